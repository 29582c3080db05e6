// sun.cu -- the twisted Wilson flow and its observables for SU(N), N = 2, 3, 4, in FP64.
//
// The paper's coupling is defined for SU(N) on the l x l x (Nl) x (Nl) box with twist
// exp(2 pi i k / N) in the short plane (Sec. 1 and Sec. 3.1); its numbers are for N = 3, and its
// outlook (Sec. 5) is larger N.  This file is the generic-N form of the flow: the same
// definitions as the SU(3) kernels (twisted staples, Z = -P_ta(U Sigma) with the 1/N trace,
// Luscher's low-storage RK3, W' = exp(X) W, the clover G = -(i/8)(C - C^+), E, q and the twisted
// plaquette), written for N x N matrices in registers.  The exponential is a Taylor polynomial of
// degree 7-11 after scaling by 2^-s, evaluated with few products, then squared s times (SU(2):
// closed form; SU(3): the Cayley-Hamilton form of the SU(3) kernels).
//
// Storage per configuration and direction: N^2 double2 planes (matrix entries, row-major) of
// Vp sites; the RK3 accumulator X holds N^2 reals per link: the imaginary parts of the N
// diagonal entries, then real and imaginary parts of the entries above the diagonal.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "expm.cuh"
#include "lattice.cuh"

namespace tgf {

namespace {

constexpr int kSunSites = 128;  // sites (threads) per block of the measurement

template <int N>
struct matN {
    cx<double> e[N][N];
};

template <int N>
__device__ __forceinline__ void zeroN(matN<N>& a) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) a.e[i][j] = {0.0, 0.0};
}

// c (+)= a b, a b^+, a^+ b
template <int N, bool ACC>
__device__ __forceinline__ void nnN(matN<N>& c, const matN<N>& a, const matN<N>& b) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double re = ACC ? c.e[i][j].re : 0.0, im = ACC ? c.e[i][j].im : 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                re = fma(a.e[i][k].re, b.e[k][j].re, re);
                re = fma(-a.e[i][k].im, b.e[k][j].im, re);
                im = fma(a.e[i][k].re, b.e[k][j].im, im);
                im = fma(a.e[i][k].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}
template <int N, bool ACC>
__device__ __forceinline__ void ndN(matN<N>& c, const matN<N>& a, const matN<N>& b) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double re = ACC ? c.e[i][j].re : 0.0, im = ACC ? c.e[i][j].im : 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                re = fma(a.e[i][k].re, b.e[j][k].re, re);
                re = fma(a.e[i][k].im, b.e[j][k].im, re);
                im = fma(a.e[i][k].im, b.e[j][k].re, im);
                im = fma(-a.e[i][k].re, b.e[j][k].im, im);
            }
            c.e[i][j] = {re, im};
        }
}
template <int N, bool ACC>
__device__ __forceinline__ void dnN(matN<N>& c, const matN<N>& a, const matN<N>& b) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            double re = ACC ? c.e[i][j].re : 0.0, im = ACC ? c.e[i][j].im : 0.0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
                re = fma(a.e[k][i].re, b.e[k][j].re, re);
                re = fma(a.e[k][i].im, b.e[k][j].im, re);
                im = fma(a.e[k][i].re, b.e[k][j].im, im);
                im = fma(-a.e[k][i].im, b.e[k][j].re, im);
            }
            c.e[i][j] = {re, im};
        }
}

template <int N>
__device__ __forceinline__ void scaleN(matN<N>& a, double zr, double zi) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double r = a.e[i][j].re, m = a.e[i][j].im;
            a.e[i][j] = {r * zr - m * zi, r * zi + m * zr};
        }
}

template <int N>
__device__ __forceinline__ void addN(matN<N>& a, const matN<N>& b) {
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            a.e[i][j].re += b.e[i][j].re;
            a.e[i][j].im += b.e[i][j].im;
        }
}

template <int N>
__device__ __forceinline__ void loadN(const double* __restrict__ base, int Vp, int dir, int s, matN<N>& u) {
    s = checked_site(s, Vp);
    const double2* q = reinterpret_cast<const double2*>(base) + (size_t)dir * N * N * Vp;
#pragma unroll
    for (int k = 0; k < N * N; ++k) {
        const double2 v = __ldg(q + (size_t)k * Vp + s);
        u.e[k / N][k % N] = {v.x, v.y};
    }
}
template <int N>
__device__ __forceinline__ void storeN(double* __restrict__ base, int Vp, int dir, int s, const matN<N>& u) {
    s = checked_site(s, Vp);
    double2* q = reinterpret_cast<double2*>(base) + (size_t)dir * N * N * Vp;
#pragma unroll
    for (int k = 0; k < N * N; ++k) q[(size_t)k * Vp + s] = make_double2(u.e[k / N][k % N].re, u.e[k / N][k % N].im);
}

// exp(2 pi i k / N)
template <int N>
__device__ __forceinline__ void centreN(int k, double& zr, double& zi) {
    sincospi(2.0 * k / N, &zi, &zr);
}

// exp(X) for anti-Hermitian X: X is scaled by 2^-s to ||Y||_F <= 1/5 and exp(Y) is replaced by
// its Taylor polynomial T_d of degree d, evaluated by Paterson and Stockmeyer's scheme (SIAM J.
// Comput. 2 (1973) 60) in blocks of B terms: with M = Y^B, T_d(Y) = B_0 + M (B_1 + M (B_2 + ...)),
// B_j = sum_{i<B} Y^i / (Bj+i)!, d = B NB - 1 for NB blocks.  B = 3 (Y^2, Y^3, then NB - 1 Horner
// products) for N <= 3; B = 2 (Y^2, then NB - 1 Horner products) for N = 4, which keeps one
// matrix fewer live.  The dropped tail is at most ||Y||^{d+1}/(d+1)! e^{||Y||}, so NB follows the
// norm: the smallest degree whose bound stays under 1.1e-17 (far below FP64 rounding of the
// unitary result):
//   B = 3:  d = 8 for ||Y|| <= 0.05,  d = 11 up to 0.2;
//   B = 2:  d = 7 for ||Y|| <= 0.028, d = 9 for <= 0.088, d = 11 up to 0.2.
// A flow step of eps = 0.01 has ||X||_F of a few 0.01, so it takes 4 matrix products where the
// plain series takes one per term (7-9); the result is then squared s times.
template <int N>
__device__ void expN(matN<N>& out, const matN<N>& X) {
    constexpr int B = N >= 4 ? 2 : 3;
    double n2 = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) n2 += X.e[i][j].re * X.e[i][j].re + X.e[i][j].im * X.e[i][j].im;
    int s = 0;
    double sc = 1.0;
    while (n2 * sc * sc > 0.04 && s < 60) {
        sc *= 0.5;
        ++s;
    }
    n2 *= sc * sc;
    // blocks and 1/d!
    int NB;
    double ctop;
    if (B == 3) {
        if (n2 <= 0.05 * 0.05) { NB = 3; ctop = 1.0 / 40320.0; }
        else { NB = 4; ctop = 1.0 / 39916800.0; }
    } else {
        if (n2 <= 0.028 * 0.028) { NB = 4; ctop = 1.0 / 5040.0; }
        else if (n2 <= 0.088 * 0.088) { NB = 5; ctop = 1.0 / 362880.0; }
        else { NB = 6; ctop = 1.0 / 39916800.0; }
    }
    matN<N> Y, Y2, Y3, t;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) Y.e[i][j] = {X.e[i][j].re * sc, X.e[i][j].im * sc};
    nnN<N, false>(Y2, Y, Y);
    if constexpr (B == 3) nnN<N, false>(Y3, Y2, Y);
    const matN<N>& M = B == 3 ? Y3 : Y2;
    // dst = B_j, given ctop = 1/(Bj+B-1)!; returns 1/(Bj)!
    auto block = [&](matN<N>& dst, int jb, double ct) {
        double c0 = ct * double(B * jb + B - 1), c1 = ct, c2 = 0.0;
        if constexpr (B == 3) {
            c2 = ct;
            c1 = c0;
            c0 = c1 * double(B * jb + 1);
        }
#pragma unroll
        for (int i = 0; i < N; ++i)
#pragma unroll
            for (int j = 0; j < N; ++j) {
                cx<double> v = {c1 * Y.e[i][j].re + (i == j ? c0 : 0.0), c1 * Y.e[i][j].im};
                if constexpr (B == 3) {
                    v.re += c2 * Y2.e[i][j].re;
                    v.im += c2 * Y2.e[i][j].im;
                }
                dst.e[i][j] = v;
            }
        return c0;
    };
    // top block, then 1/(Bj-1)! = Bj / (Bj)! going down; each Horner step forms B_j first and
    // accumulates the product M (B_{j+1} + ...) onto it in the product's own FMAs
    ctop = block(out, NB - 1, ctop) * double(B * (NB - 1));
#pragma unroll 1
    for (int jb = NB - 2; jb >= 0; --jb) {
        ctop = block(t, jb, ctop) * double(B * jb);
        nnN<N, true>(t, M, out);
        out = t;
    }
#pragma unroll 1
    for (int k = 0; k < s; ++k) {
        t = out;
        nnN<N, false>(out, t, t);
    }
}

// SU(2): closed form.  X = i tau 1 + X0 with X0 traceless anti-Hermitian, X0^2 = -theta^2 1
// (theta^2 = a^2 + |b|^2 for X0 = [[i a, b], [-b*, -i a]]), so
// exp(X) = e^{i tau} (cos theta 1 + (sin theta / theta) X0).
template <>
__device__ void expN<2>(matN<2>& out, const matN<2>& X) {
    const double tau = 0.5 * (X.e[0][0].im + X.e[1][1].im);
    const double a = X.e[0][0].im - tau;
    const double br = X.e[0][1].re, bi = X.e[0][1].im;
    const double th = sqrt(a * a + br * br + bi * bi);
    const double c = cos(th), sn = th > 1e-30 ? sin(th) / th : 1.0;
    double er, ei;
    sincos(tau, &ei, &er);
    // M = c 1 + sn X0;  out = e^{i tau} M
    const cx<double> m00 = {c, sn * a}, m11 = {c, -sn * a};
    const cx<double> m01 = {sn * br, sn * bi}, m10 = {-sn * br, sn * bi};
    out.e[0][0] = {er * m00.re - ei * m00.im, er * m00.im + ei * m00.re};
    out.e[0][1] = {er * m01.re - ei * m01.im, er * m01.im + ei * m01.re};
    out.e[1][0] = {er * m10.re - ei * m10.im, er * m10.im + ei * m10.re};
    out.e[1][1] = {er * m11.re - ei * m11.im, er * m11.im + ei * m11.re};
}

// SU(3): the Cayley-Hamilton exponential of the SU(3) kernels (expm.cuh) on the 8 parameters of
// the traceless X (the stage builds X traceless; a trace at rounding level is dropped): a few
// dozen scalar operations instead of the polynomial's 4 matrix products.
template <>
__device__ void expN<3>(matN<3>& out, const matN<3>& X) {
    alg8<double> x;
    x.v[0] = X.e[0][0].im;
    x.v[1] = X.e[1][1].im;
    x.v[2] = X.e[0][1].re;
    x.v[3] = X.e[0][1].im;
    x.v[4] = X.e[0][2].re;
    x.v[5] = X.e[0][2].im;
    x.v[6] = X.e[1][2].re;
    x.v[7] = X.e[1][2].im;
    mat3<double> m;
    expm_su3<double, false>(m, x);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) out.e[i][j] = m.e[i][j];
}

// one RK3 stage for SU(N); block = 4 warps (one per direction) x 32 sites
template <int N, int STAGE, int CAP>
__global__ void __launch_bounds__(128, 1)
k_sun_stage(const __grid_constant__ BatchT<CAP> B, const double* __restrict__ w_in, double* __restrict__ w_out,
            double* __restrict__ acc) {
    const int mu = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int blk = blockIdx.x;
    if (blk >= B.nblk) return;
    const int ci = find_cfg(B, blk);
    const CfgDesc& c = B.c[ci];
    const int s = (blk - c.blk0) * 32 + lane;
    if (s >= c.V) return;
    const uint64_t xp = pack_coords(c, s);
    const int Vp = c.Vp;
    const double* base = w_in + c.w_off;
    const int xm = coord(xp, mu), Lm = c.L[mu], Sm = c.st[mu];
    const int s_mp = step_p(s, xm, Lm, Sm);
    matN<N> sig, a, b, t;
    zeroN(sig);
#pragma unroll 1
    for (int dn = 1; dn < 4; ++dn) {
        const int nu = (mu + dn) & 3;
        const int xn = coord(xp, nu), Ln = c.L[nu], Sn = c.st[nu];
        const int s_nm = step_m(s, xn, Ln, Sn);
        const int s_mp_nm = step_p(s_nm, xm, Lm, Sm);
        const int k = c.tw[mu * 4 + nu];
        double zr = 1.0, zi = 0.0;
        if (k != 0) centreN<N>(k, zr, zi);
        // forward staple Z*_{mu nu}(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
        loadN<N>(base, Vp, nu, s_mp, a);
        loadN<N>(base, Vp, mu, step_p(s, xn, Ln, Sn), b);
        ndN<N, false>(t, a, b);
        loadN<N>(base, Vp, nu, s, a);
        if (k != 0 && xm == 0 && xn == 0) {
            ndN<N, false>(b, t, a);
            scaleN(b, zr, -zi);
            addN(sig, b);
        } else {
            ndN<N, true>(sig, t, a);
        }
        // backward staple Z_{mu nu}(n-nu) U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu)
        loadN<N>(base, Vp, mu, s_nm, a);
        loadN<N>(base, Vp, nu, s_mp_nm, b);
        nnN<N, false>(t, a, b);
        loadN<N>(base, Vp, nu, s_nm, a);
        if (k != 0 && xm == 0 && xn == 1) {
            dnN<N, false>(b, t, a);
            scaleN(b, zr, zi);
            addN(sig, b);
        } else {
            dnN<N, true>(sig, t, a);
        }
    }
    // Omega = U Sigma; Z = -P_ta(Omega) = -(Omega - Omega^+)/2 + tr(Omega - Omega^+)/(2N)
    loadN<N>(base, Vp, mu, s, a);
    nnN<N, false>(t, a, sig);
    double trim = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) trim += t.e[i][i].im;
    trim /= N;
    const double h = c.h;
    double* xb = acc + c.x_off + (size_t)mu * N * N * Vp;
    // X in N^2 reals: diag imag parts, then (re, im) above the diagonal
    double x[N * N];
    int r = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) x[r++] = -(t.e[i][i].im - trim);
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i + 1; j < N; ++j) {
            x[r++] = -0.5 * (t.e[i][j].re - t.e[j][i].re);
            x[r++] = -0.5 * (t.e[i][j].im + t.e[j][i].im);
        }
#pragma unroll
    for (int q = 0; q < N * N; ++q) {
        double v;
        if (STAGE == 1) v = 0.25 * h * x[q];
        else if (STAGE == 2) v = (8.0 / 9.0) * h * x[q] - (17.0 / 9.0) * xb[(size_t)q * Vp + s];
        else v = 0.75 * h * x[q] - xb[(size_t)q * Vp + s];
        x[q] = v;
        if (STAGE != 3) xb[(size_t)q * Vp + s] = v;
    }
    r = 0;
#pragma unroll
    for (int i = 0; i < N; ++i) b.e[i][i] = {0.0, x[r++]};
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = i + 1; j < N; ++j) {
            b.e[i][j] = {x[r], x[r + 1]};
            b.e[j][i] = {-x[r], x[r + 1]};
            r += 2;
        }
    expN<N>(t, b);
    nnN<N, false>(b, t, a);
    storeN<N>(w_out + c.w_off, Vp, mu, s, b);
}

// G = -(i/8)(C - C^+) of the plane (mu, nu) at site s, from the four twisted leaves (Sec. 3.1, eq. gmunu);
// also returns Re Tr[Z* P_{mu nu}(n)] (the first leaf)
template <int N>
__device__ void cloverN(const CfgDesc& c, const double* __restrict__ base, int s, uint64_t xp, int mu, int nu,
                        bool traceless, matN<N>& G, double& retr) {
    const int Vp = c.Vp;
    const int xm = coord(xp, mu), xn = coord(xp, nu);
    const int s_mp = step_p(s, xm, c.L[mu], c.st[mu]), s_mm = step_m(s, xm, c.L[mu], c.st[mu]);
    const int s_np = step_p(s, xn, c.L[nu], c.st[nu]), s_nm = step_m(s, xn, c.L[nu], c.st[nu]);
    const int s_nm_mp = step_p(s_nm, xm, c.L[mu], c.st[mu]);
    const int s_mm_np = step_p(s_mm, xn, c.L[nu], c.st[nu]);
    const int s_mm_nm = step_m(s_mm, xn, c.L[nu], c.st[nu]);
    const int k = c.tw[mu * 4 + nu];
    double zr = 1.0, zi = 0.0;
    if (k != 0) centreN<N>(k, zr, zi);
    matN<N> C, a, b, t, l;
    // L1 = Z*(n) U_mu(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
    loadN<N>(base, Vp, mu, s, a);
    loadN<N>(base, Vp, nu, s_mp, b);
    nnN<N, false>(t, a, b);
    loadN<N>(base, Vp, mu, s_np, a);
    ndN<N, false>(l, t, a);
    loadN<N>(base, Vp, nu, s, a);
    ndN<N, false>(C, l, a);
    if (k != 0 && xm == 0 && xn == 0) scaleN(C, zr, -zi);
    retr = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) retr += C.e[i][i].re;
    // L2 = Z*(n-nu) U_nu(n-nu)^+ U_mu(n-nu) U_nu(n-nu+mu) U_mu(n)^+
    loadN<N>(base, Vp, nu, s_nm, a);
    loadN<N>(base, Vp, mu, s_nm, b);
    dnN<N, false>(t, a, b);
    loadN<N>(base, Vp, nu, s_nm_mp, a);
    nnN<N, false>(l, t, a);
    loadN<N>(base, Vp, mu, s, a);
    ndN<N, false>(t, l, a);
    if (k != 0 && xm == 0 && xn == 1) scaleN(t, zr, -zi);
    addN(C, t);
    // L3 = Z*(n-mu) U_nu(n) U_mu(n-mu+nu)^+ U_nu(n-mu)^+ U_mu(n-mu)
    loadN<N>(base, Vp, nu, s, a);
    loadN<N>(base, Vp, mu, s_mm_np, b);
    ndN<N, false>(t, a, b);
    loadN<N>(base, Vp, nu, s_mm, a);
    ndN<N, false>(l, t, a);
    loadN<N>(base, Vp, mu, s_mm, a);
    nnN<N, false>(t, l, a);
    if (k != 0 && xm == 1 && xn == 0) scaleN(t, zr, -zi);
    addN(C, t);
    // L4 = Z*(n-mu-nu) U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu) U_nu(n-nu)
    loadN<N>(base, Vp, nu, s_mm_nm, b);
    loadN<N>(base, Vp, mu, s_mm, a);
    nnN<N, false>(t, b, a);  // U_nu(n-mu-nu) U_mu(n-mu)
    loadN<N>(base, Vp, mu, s_mm_nm, a);
    dnN<N, false>(l, t, a);  // (U_nu U_mu)^+ U_mu(n-mu-nu) = U_mu(n-mu)^+ U_nu(n-mu-nu)^+ U_mu(n-mu-nu)
    loadN<N>(base, Vp, nu, s_nm, a);
    nnN<N, false>(t, l, a);
    if (k != 0 && xm == 1 && xn == 1) scaleN(t, zr, -zi);
    addN(C, t);
    // G = -(i/8)(C - C^+): G_jk = -(i/8)(C_jk - conj(C_kj))
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const double dr = C.e[i][j].re - C.e[j][i].re, di = C.e[i][j].im + C.e[j][i].im;
            G.e[i][j] = {di / 8.0, -dr / 8.0};
        }
    if (traceless) {
        double tr = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) tr += G.e[i][i].re;
        tr /= N;
#pragma unroll
        for (int i = 0; i < N; ++i) G.e[i][i].re -= tr;
    }
}

// Re Tr[A B] for Hermitian A, B
template <int N>
__device__ __forceinline__ double retr_prod(const matN<N>& A, const matN<N>& B) {
    double v = 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k < N; ++k) v += A.e[i][k].re * B.e[k][i].re - A.e[i][k].im * B.e[k][i].im;
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// per-site E, q, p, s summed over each block of kSunSites sites (fixed order)
template <int N, int CAP>
__global__ void __launch_bounds__(kSunSites, 1)
k_sun_measure(const __grid_constant__ BatchT<CAP> B, const double* __restrict__ w, double* __restrict__ partial,
              int traceless) {
    __shared__ double red[kSunSites / 32][4];
    const int blk = blockIdx.x;
    if (blk >= B.nblk) return;
    const int ci = find_cfg(B, blk);
    const CfgDesc& c = B.c[ci];
    const int s = (blk - c.blk0) * kSunSites + threadIdx.x;
    double e = 0.0, q = 0.0, p = 0.0, sa = 0.0;
    if (s < c.V) {
        const uint64_t xp = pack_coords(c, s);
        const double* base = w + c.w_off;
        // planes in pairs (01, 23), (02, 13), (03, 12) with the signs of eq. qlatt
        const int pa[3][2] = {{0, 1}, {0, 2}, {0, 3}}, pb[3][2] = {{2, 3}, {1, 3}, {1, 2}};
        const double sg[3] = {1.0, -1.0, 1.0};
#pragma unroll 1
        for (int pr = 0; pr < 3; ++pr) {
            matN<N> Ga, Gb;
            double ra, rb;
            cloverN<N>(c, base, s, xp, pa[pr][0], pa[pr][1], traceless, Ga, ra);
            cloverN<N>(c, base, s, xp, pb[pr][0], pb[pr][1], traceless, Gb, rb);
            e += retr_prod(Ga, Ga) + retr_prod(Gb, Gb);
            q += sg[pr] * retr_prod(Ga, Gb);
            p += (ra + rb) / N;
            sa += 2.0 * N - (ra + rb);
        }
        q *= 1.0 / (4.0 * CUDART_PI * CUDART_PI);
    }
    e = warp_sum(e);
    q = warp_sum(q);
    p = warp_sum(p);
    sa = warp_sum(sa);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp][0] = e;
        red[warp][1] = q;
        red[warp][2] = p;
        red[warp][3] = sa;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int i = 0; i < kSunSites / 32; ++i) v += red[i][threadIdx.x];
        partial[(size_t)blk * 4 + threadIdx.x] = v;
    }
}

// per configuration: sum of its block partials in block order -> {t, E, Q, P, S}
template <int CAP>
__global__ void __launch_bounds__(256) k_sun_reduce(const __grid_constant__ BatchT<CAP> B, const double* __restrict__ partial,
                                                    double* __restrict__ obs) {
    __shared__ double red[4][256];
    const CfgDesc& c = B.c[blockIdx.x];
    const int nb = (c.V + kSunSites - 1) / kSunSites;
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nb; i += 256)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += partial[(size_t)(c.blk0 + i) * 4 + k];
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int wdt = 128; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt)
#pragma unroll
            for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + wdt];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* o = obs + (size_t)c.o_off * 5;
        o[0] = c.h;
        o[1] = red[0][0] / c.V;
        o[2] = red[1][0];
        o[3] = red[2][0] / (6.0 * c.V);
        o[4] = red[3][0];
    }
}

// canonical [site][mu][N][N] complex <-> storage planes
template <int N, int CAP, bool TO_STORAGE>
__global__ void k_sun_layout(const __grid_constant__ BatchT<CAP> B, double* __restrict__ canon, double* __restrict__ w) {
    const int blk = blockIdx.x;
    if (blk >= B.nblk) return;
    const int ci = find_cfg(B, blk);
    const CfgDesc& c = B.c[ci];
    const int s = (blk - c.blk0) * 128 + threadIdx.x;
    if (s >= c.V) return;
    double2* q = reinterpret_cast<double2*>(w + c.w_off);
    double2* cn = reinterpret_cast<double2*>(canon + c.m_off) + (size_t)s * 4 * N * N;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu)
#pragma unroll
        for (int k = 0; k < N * N; ++k) {
            if (TO_STORAGE) q[((size_t)mu * N * N + k) * c.Vp + s] = cn[mu * N * N + k];
            else cn[mu * N * N + k] = q[((size_t)mu * N * N + k) * c.Vp + s];
        }
}

template <int CAP>
BatchT<CAP> shrink(const Batch& B) {
    BatchT<CAP> b;
    b.ncfg = B.ncfg;
    b.nblk = B.nblk;
    for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
    return b;
}

template <int N, int CAP>
void sun_stage_cap(int stage, const Batch& B, const double* w_in, double* w_out, double* acc, cudaStream_t st) {
    const BatchT<CAP> b = shrink<CAP>(B);
    if (stage == 1) k_sun_stage<N, 1, CAP><<<B.nblk, 128, 0, st>>>(b, w_in, w_out, acc);
    else if (stage == 2) k_sun_stage<N, 2, CAP><<<B.nblk, 128, 0, st>>>(b, w_in, w_out, acc);
    else k_sun_stage<N, 3, CAP><<<B.nblk, 128, 0, st>>>(b, w_in, w_out, acc);
}

template <int N, int CAP>
void sun_measure_cap(const Batch& Bm, const Batch& Br, const double* w, double* partial, double* obs, int traceless,
                     cudaStream_t st) {
    const BatchT<CAP> bm = shrink<CAP>(Bm), br = shrink<CAP>(Br);
    k_sun_measure<N, CAP><<<Bm.nblk, kSunSites, 0, st>>>(bm, w, partial, traceless);
    k_sun_reduce<CAP><<<Br.ncfg, 256, 0, st>>>(br, partial, obs);
}

template <int N, int CAP>
void sun_layout_cap(bool to_storage, const Batch& B, double* canon, double* w, cudaStream_t st) {
    const BatchT<CAP> b = shrink<CAP>(B);
    if (to_storage) k_sun_layout<N, CAP, true><<<B.nblk, 128, 0, st>>>(b, canon, w);
    else k_sun_layout<N, CAP, false><<<B.nblk, 128, 0, st>>>(b, canon, w);
}

template <int N>
void sun_dispatch(int op, int stage, bool to_storage, const Batch& B, const Batch& B2, const double* a, double* b,
                  double* c, double* d, int flag, cudaStream_t st) {
    const bool small = B.ncfg <= kSmallCap;
    if (op == 0) {
        if (small) sun_stage_cap<N, kSmallCap>(stage, B, a, b, c, st);
        else sun_stage_cap<N, kMaxCfg>(stage, B, a, b, c, st);
    } else if (op == 1) {
        if (small) sun_measure_cap<N, kSmallCap>(B, B2, a, c, d, flag, st);
        else sun_measure_cap<N, kMaxCfg>(B, B2, a, c, d, flag, st);
    } else {
        if (small) sun_layout_cap<N, kSmallCap>(to_storage, B, c, b, st);
        else sun_layout_cap<N, kMaxCfg>(to_storage, B, c, b, st);
    }
}

void sun_any(int N, int op, int stage, bool to_storage, const Batch& B, const Batch& B2, const double* a, double* b,
             double* c, double* d, int flag, cudaStream_t st) {
    if (N == 2) sun_dispatch<2>(op, stage, to_storage, B, B2, a, b, c, d, flag, st);
    else if (N == 3) sun_dispatch<3>(op, stage, to_storage, B, B2, a, b, c, d, flag, st);
    else sun_dispatch<4>(op, stage, to_storage, B, B2, a, b, c, d, flag, st);
}

}  // namespace

void launch_sun_stage(int N, int stage, const Batch& B, const double* w_in, double* w_out, double* acc,
                      cudaStream_t st) {
    sun_any(N, 0, stage, false, B, B, w_in, w_out, acc, nullptr, 0, st);
}

void launch_sun_measure(int N, const Batch& Bm, const Batch& Br, const double* w, double* partial, double* obs,
                        int traceless, cudaStream_t st) {
    sun_any(N, 1, 0, false, Bm, Br, w, nullptr, partial, obs, traceless, st);
}

void launch_sun_layout(int N, bool to_storage, const Batch& B, double* canon, double* w, cudaStream_t st) {
    sun_any(N, 2, 0, to_storage, B, B, nullptr, w, canon, nullptr, 0, st);
}

TGF_CHECK_WORD(sun)

}  // namespace tgf
