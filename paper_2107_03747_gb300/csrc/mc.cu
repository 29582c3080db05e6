// mc.cu -- twisted hybrid Monte Carlo update of FP64 link fields: Cabibbo-Marinari heat-bath
// and over-relaxation in the three SU(2) subgroups, one checkerboard pass per launch.
//
// Ensembles of the twisted Wilson action S_W = 3b sum_n sum_{mu!=nu} Tr[1 - Z* P] (Sec. 3.1) are
// generated with one heat-bath sweep followed by L~ over-relaxation sweeps (the hybrid
// algorithm the paper cites).  With beta = 18 b the weight of one link U = U_mu(n) is
// exp((beta/3) Re Tr[U Sigma]), Sigma its twisted staple sum.  For the SU(2) block (i, j) of
// W = U Sigma, with SU(2)-proportional part k v (v in SU(2)):
//   heat-bath        R = X v^+, X drawn with density exp(alpha X0) dHaar, alpha = 2 beta k / 3
//   over-relaxation  R = (v^+)^2                      (keeps Re Tr[U Sigma])
// and U <- R U.  X0 comes from Kennedy-Pendleton's sampler (alpha > 2) or Creutz's (otherwise).
//
// Thread mapping: one thread per link (n, mu) of one parity; a launch updates every link of
// direction mu on the sites with x0+x1+x2+x3 = parity (mod 2).  Their staples contain only links
// of the other directions or of the other parity, so the in-place update is race-free and equal
// to any sequential order inside the pass.
//
// Random numbers are counter-based: draw = SplitMix64 output function of
// key + (counter + 1) * 0x9E3779B97F4A7C15, u = ((x >> 11) + 1) 2^-53 in (0, 1], with
// key = the same hash of (seed, configuration index) and counter
// (((sweep * 4 + mu) * V + site) * 3 + subgroup) * 260 + slot; slots 4a..4a+3 serve rejection
// attempt a < 64, slots 256 and 257 the direction of X.  A subgroup whose 64 attempts are all
// rejected is left unchanged.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"

namespace tgf {

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kSlots = 260;
constexpr int kAttempts = 64;
constexpr int kMcThreads = 128;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hash64(uint64_t key, uint64_t counter) { return mix64(key + (counter + 1) * kGolden); }
__device__ __forceinline__ double draw(uint64_t key, uint64_t counter) {
    return ((double)(hash64(key, counter) >> 11) + 1.0) * 0x1.0p-53;
}

struct quat {
    double a0, a1, a2, a3;
};
__device__ __forceinline__ quat qmul(const quat& a, const quat& b) {
    // (a0 + i a.s)(b0 + i b.s) = a0 b0 - a.b + i (a0 b + b0 a - a x b).s
    return {a.a0 * b.a0 - (a.a1 * b.a1 + a.a2 * b.a2 + a.a3 * b.a3),
            a.a0 * b.a1 + b.a0 * a.a1 - (a.a2 * b.a3 - a.a3 * b.a2),
            a.a0 * b.a2 + b.a0 * a.a2 - (a.a3 * b.a1 - a.a1 * b.a3),
            a.a0 * b.a3 + b.a0 * a.a3 - (a.a1 * b.a2 - a.a2 * b.a1)};
}
__device__ __forceinline__ quat qconj(const quat& a) { return {a.a0, -a.a1, -a.a2, -a.a3}; }

// X0 with density sqrt(1 - X0^2) exp(alpha X0) on [-1, 1]; false when every attempt is rejected
__device__ bool sample_x0(double alpha, uint64_t key, uint64_t c0, double& x0) {
    const bool kp = alpha > 2.0;
    const double e2a = kp ? 0.0 : exp(-2.0 * alpha);
#pragma unroll 1
    for (int a = 0; a < kAttempts; ++a) {
        const uint64_t c = c0 + 4 * a;
        const double r1 = draw(key, c), r2 = draw(key, c + 1);
        if (kp) {
            // Kennedy-Pendleton: lambda^2 = -(ln r1 + cos^2(2 pi r2) ln r3) / (2 alpha)
            const double r3 = draw(key, c + 2), r4 = draw(key, c + 3);
            const double cs = cos(2.0 * M_PI * r2);
            const double lam2 = -__dadd_rn(log(r1), __dmul_rn(__dmul_rn(cs, cs), log(r3))) / (2.0 * alpha);
            if (__dmul_rn(r4, r4) <= 1.0 - lam2) {
                x0 = 1.0 - 2.0 * lam2;
                return true;
            }
        } else {
            // Creutz: X0 = 1 + ln(e^{-2 alpha} + (1 - e^{-2 alpha}) r1) / alpha, kept with probability sqrt(1 - X0^2)
            const double xc = alpha < 1e-8 ? 2.0 * r1 - 1.0
                                           : 1.0 + log(__dadd_rn(e2a, __dmul_rn(1.0 - e2a, r1))) / alpha;
            if (__dmul_rn(r2, r2) <= 1.0 - __dmul_rn(xc, xc)) {
                x0 = xc;
                return true;
            }
        }
    }
    return false;
}

// twisted staple sum Sigma_mu(n): Re Tr[U_mu(n) Sigma] = sum of Re Tr[Z* P] over the six
// plaquettes that contain U_mu(n)
__device__ void staple_sum(const double* __restrict__ base, int Vp, const CfgDesc& c, int s, uint64_t xp, int mu,
                           mat3<double>& sig) {
    using S = Store<P64>;
    auto link = [&](int dir, int site, mat3<double>& u) { S::load(base + (size_t)dir * 18 * Vp, Vp, site, u); };
    mat3<double> a, b, t, f;
    set_zero(sig);
    const int xm = coord(xp, mu);
    const int s_mp = step_p(s, xm, c.L[mu], c.st[mu]);
#pragma unroll 1
    for (int dn = 1; dn < 4; ++dn) {
        const int nu = (mu + dn) & 3;
        const int xn = coord(xp, nu);
        const int s_np = step_p(s, xn, c.L[nu], c.st[nu]);
        const int s_nm = step_m(s, xn, c.L[nu], c.st[nu]);
        const int s_mp_nm = step_p(s_nm, xm, c.L[mu], c.st[mu]);
        const int k = c.tw[mu * 4 + nu];
        double zr = 1.0, zi = 0.0;
        if (k != 0) centre<double>(k, zr, zi);
        // forward: Z*_{mu nu}(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
        link(nu, s_mp, a);
        link(mu, s_np, b);
        mul_nd(t, a, b);
        link(nu, s, a);
        mul_nd(f, t, a);
        if (k != 0 && xm == 0 && xn == 0) scale_cx(f, zr, -zi);
        add_to(sig, f);
        // backward: Z_{mu nu}(n-nu) U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu)
        link(mu, s_nm, a);
        link(nu, s_mp_nm, b);
        mul_nn(t, a, b);
        link(nu, s_nm, a);
        mul_dn(f, t, a);
        if (k != 0 && xm == 0 && xn == 1) scale_cx(f, zr, zi);
        add_to(sig, f);
    }
}

template <int OVERRELAX, int CAP>
__global__ void __launch_bounds__(kMcThreads) k_mc(const __grid_constant__ BatchT<CAP> B, double* __restrict__ w,
                                                   int mu, int parity, double beta, uint64_t seed, uint64_t sweep) {
    const int blk = blockIdx.x;
    if (blk >= B.nblk) return;
    const int ci = find_cfg(B, blk);
    const CfgDesc& c = B.c[ci];
    const int t = (blk - c.blk0) * kMcThreads + threadIdx.x;
    if (t >= c.V / 2) return;
    // t -> the t-th site of this parity (every extent even): x0 = 2j + ((x1 + x2 + x3 + parity) & 1)
    int x[4];
    const int h0 = c.L[0] / 2;
    int r = t / h0;
    const int j = t - r * h0;
    x[1] = r % c.L[1];
    r /= c.L[1];
    x[2] = r % c.L[2];
    x[3] = r / c.L[2];
    x[0] = 2 * j + ((x[1] + x[2] + x[3] + parity) & 1);
    const int s = x[0] + c.st[1] * x[1] + c.st[2] * x[2] + c.st[3] * x[3];
    const int Vp = c.Vp;
    double* base = w + c.w_off;

    mat3<double> sig, u, wm;
    const uint64_t xp = (uint64_t)x[0] | ((uint64_t)x[1] << 16) | ((uint64_t)x[2] << 32) | ((uint64_t)x[3] << 48);
    staple_sum(base, Vp, c, s, xp, mu, sig);
    Store<P64>::load(base + (size_t)mu * 18 * Vp, Vp, s, u);
    mul_nn(wm, u, sig);
    const uint64_t key = hash64(seed, (uint64_t)ci);
    const int sub[3][2] = {{0, 1}, {0, 2}, {1, 2}};
#pragma unroll
    for (int g = 0; g < 3; ++g) {
        const int i = sub[g][0], jj = sub[g][1];
        // SU(2)-proportional part of the block (i, jj) of W
        quat xq = {0.5 * (wm.e[i][i].re + wm.e[jj][jj].re), 0.5 * (wm.e[i][jj].im + wm.e[jj][i].im),
                   0.5 * (wm.e[i][jj].re - wm.e[jj][i].re), 0.5 * (wm.e[i][i].im - wm.e[jj][jj].im)};
        const double k = sqrt(xq.a0 * xq.a0 + xq.a1 * xq.a1 + xq.a2 * xq.a2 + xq.a3 * xq.a3);
        const bool live = k > 1e-300;
        const quat v = live ? quat{xq.a0 / k, xq.a1 / k, xq.a2 / k, xq.a3 / k} : quat{1.0, 0.0, 0.0, 0.0};
        quat R = {1.0, 0.0, 0.0, 0.0};
        if (OVERRELAX) {
            if (live) R = qmul(qconj(v), qconj(v));
        } else {
            const uint64_t c0 = ((((uint64_t)sweep * 4 + (uint64_t)mu) * (uint64_t)c.V + (uint64_t)s) * 3 + g) * kSlots;
            double x0;
            if (sample_x0(2.0 * beta * k / 3.0, key, c0, x0)) {
                const double cth = 2.0 * draw(key, c0 + 256) - 1.0;
                const double phi = 2.0 * M_PI * draw(key, c0 + 257);
                const double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
                const double rr = sqrt(fmax(0.0, 1.0 - x0 * x0));
                const quat X = {x0, rr * sth * cos(phi), rr * sth * sin(phi), rr * cth};
                R = qmul(X, qconj(v));
            }
        }
        // R as a 2x2 matrix [[R0 + i R3, R2 + i R1], [-R2 + i R1, R0 - i R3]] acting on rows i, jj
        const cx<double> r00 = {R.a0, R.a3}, r01 = {R.a2, R.a1}, r10 = {-R.a2, R.a1}, r11 = {R.a0, -R.a3};
        auto rot = [&](mat3<double>& m) {
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                const cx<double> p = m.e[i][col], q = m.e[jj][col];
                m.e[i][col] = {r00.re * p.re - r00.im * p.im + (r01.re * q.re - r01.im * q.im),
                               r00.re * p.im + r00.im * p.re + (r01.re * q.im + r01.im * q.re)};
                m.e[jj][col] = {r10.re * p.re - r10.im * p.im + (r11.re * q.re - r11.im * q.im),
                                r10.re * p.im + r10.im * p.re + (r11.re * q.im + r11.im * q.re)};
            }
        };
        rot(u);
        rot(wm);
    }
    Store<P64>::store(base + (size_t)mu * 18 * Vp, Vp, s, u);
}

template <int OVERRELAX, int CAP>
void launch_cap(const Batch& B, double* w, int mu, int parity, double beta, uint64_t seed, uint64_t sweep,
                cudaStream_t st) {
    if constexpr (CAP == kMaxCfg) {
        k_mc<OVERRELAX, kMaxCfg><<<B.nblk, kMcThreads, 0, st>>>(B, w, mu, parity, beta, seed, sweep);
    } else {
        BatchT<CAP> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_mc<OVERRELAX, CAP><<<B.nblk, kMcThreads, 0, st>>>(b, w, mu, parity, beta, seed, sweep);
    }
}

}  // namespace

void launch_mc(int overrelax, const Batch& B, double* w, int mu, int parity, double beta, uint64_t seed,
               uint64_t sweep, cudaStream_t st) {
    if (B.ncfg <= kSmallCap) {
        if (overrelax) launch_cap<1, kSmallCap>(B, w, mu, parity, beta, seed, sweep, st);
        else launch_cap<0, kSmallCap>(B, w, mu, parity, beta, seed, sweep, st);
    } else {
        if (overrelax) launch_cap<1, kMaxCfg>(B, w, mu, parity, beta, seed, sweep, st);
        else launch_cap<0, kMaxCfg>(B, w, mu, parity, beta, seed, sweep, st);
    }
}

TGF_CHECK_WORD(mc)

}  // namespace tgf
