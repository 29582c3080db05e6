// stage.cu -- one stage of the RK3 Wilson-flow step: twisted staples -> force -> X update ->
// exact exponential -> W' = exp(X) W, fused in one kernel per stage.
//
// Thread mapping: a block covers SPB consecutive sites of one configuration; each of its
// 4*SPB threads owns one link (site, mu), warps grouped by mu so that every load of a
// component plane is a contiguous, 16-byte-vectorised warp access.  Neighbour links are
// read through the read-only data path (L1/L2 absorb the 19-fold reuse of each link).
#include <cuda_runtime.h>

#include "expm.cuh"
#include "lattice.cuh"

namespace tgf {

// Gram-Schmidt re-projection onto SU(3) in FP64 registers: rows 0, 1 orthonormalised,
// row 2 = conj(row0 x row1).
template <class T>
__device__ __forceinline__ void reunitarize(mat3<T>& u) {
    mat3<double> d;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) d.e[i][j] = {(double)u.e[i][j].re, (double)u.e[i][j].im};
    double n0 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n0 += d.e[0][j].re * d.e[0][j].re + d.e[0][j].im * d.e[0][j].im;
    n0 = rsqrt(n0);
#pragma unroll
    for (int j = 0; j < 3; ++j) { d.e[0][j].re *= n0; d.e[0][j].im *= n0; }
    // r1 -= (r0^+ r1) r0
    double pr = 0, pi = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        pr += d.e[0][j].re * d.e[1][j].re + d.e[0][j].im * d.e[1][j].im;
        pi += d.e[0][j].re * d.e[1][j].im - d.e[0][j].im * d.e[1][j].re;
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        d.e[1][j].re -= pr * d.e[0][j].re - pi * d.e[0][j].im;
        d.e[1][j].im -= pr * d.e[0][j].im + pi * d.e[0][j].re;
    }
    double n1 = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) n1 += d.e[1][j].re * d.e[1][j].re + d.e[1][j].im * d.e[1][j].im;
    n1 = rsqrt(n1);
#pragma unroll
    for (int j = 0; j < 3; ++j) { d.e[1][j].re *= n1; d.e[1][j].im *= n1; }
    rebuild_row2(d);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) u.e[i][j] = {(T)d.e[i][j].re, (T)d.e[i][j].im};
}

template <int P, int STAGE, int SPB, int CAP>
__global__ void __launch_bounds__(4 * SPB)
k_stage(const __grid_constant__ BatchT<CAP> B, const typename Store<P>::T* __restrict__ w_in,
        typename Store<P>::T* __restrict__ w_out, typename Store<P>::T* __restrict__ acc, int reunit) {
    using T = typename Store<P>::T;
    using S = Store<P>;
    constexpr int R = S::reals;
    constexpr int WPD = SPB / 32;  // warps per direction
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mu = warp / WPD;

    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int s = (blk - c.blk0) * SPB + (warp % WPD) * 32 + lane;
        if (s >= c.V) continue;
        Site p;
        make_site(p, c, s);
        const int Vp = c.Vp;
        const T* base = w_in + c.w_off;
        auto link = [&](int dir, int site, mat3<T>& u) { S::load(base + (size_t)dir * R * Vp, Vp, site, u); };

        mat3<T> sig, a, b, t;
        set_zero(sig);
        const int smu_p = nb(p, s, p.x[mu], mu, +1);
#pragma unroll
        for (int dn = 1; dn < 4; ++dn) {
            const int nu = (mu + dn) & 3;
            const int snu_p = nb(p, s, p.x[nu], nu, +1);
            const int snu_m = nb(p, s, p.x[nu], nu, -1);
            const int k = c.tw[mu * 4 + nu];
            // forward staple Z*_{mu nu}(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+
            link(nu, smu_p, a);
            link(mu, snu_p, b);
            mul_nd(t, a, b);
            link(nu, s, a);
            if (k != 0 && p.x[mu] == 0 && p.x[nu] == 0) {
                mul_nd(b, t, a);
                T zr, zi;
                centre<T>(k, zr, zi);
                scale_cx(b, zr, -zi);
                add_to(sig, b);
            } else {
                mul_nd_acc(sig, t, a);
            }
            // backward staple Z_{mu nu}(n-nu) U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu)
            const int smu_p_nu_m = nb(p, snu_m, p.x[mu], mu, +1);
            link(mu, snu_m, a);
            link(nu, smu_p_nu_m, b);
            mul_nn(t, a, b);
            link(nu, snu_m, a);
            if (k != 0 && p.x[mu] == 0 && p.x[nu] == 1) {
                mul_dn(b, t, a);
                T zr, zi;
                centre<T>(k, zr, zi);
                scale_cx(b, zr, zi);
                add_to(sig, b);
            } else {
                mul_dn_acc(sig, t, a);
            }
        }
        // Omega = U_mu(n) Sigma, Z = -P_ta(Omega)
        link(mu, s, a);
        mul_nn(t, a, sig);
        alg8<T> z;
        minus_proj_ta(z, t);
        const T h = (T)c.h;
        alg8<T> x;
        T* xb = acc + c.x_off + (size_t)mu * 8 * Vp;
        if (STAGE == 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = T(0.25) * h * z.v[i];
            AccStore<T>::store(xb, Vp, s, x);
        } else if (STAGE == 2) {
            AccStore<T>::load(xb, Vp, s, x);
            const T c1 = T(8) / T(9), c2 = T(17) / T(9);
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = c1 * h * z.v[i] - c2 * x.v[i];
            AccStore<T>::store(xb, Vp, s, x);
        } else {
            AccStore<T>::load(xb, Vp, s, x);
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = T(0.75) * h * z.v[i] - x.v[i];
        }
        expm_su3(b, x);
        mul_nn(t, b, a);
        if (STAGE == 3 && P != P64 && reunit) reunitarize(t);
        S::store(w_out + c.w_off + (size_t)mu * R * Vp, Vp, s, t);
    }
}

template <int P, int STAGE, int SPB, int CAP>
static void launch_cap(const Batch& B, const void* w_in, void* w_out, void* acc, int reunit, cudaStream_t st) {
    using T = typename Store<P>::T;
    BatchT<CAP> b;
    b.ncfg = B.ncfg;
    b.nblk = B.nblk;
    for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
    k_stage<P, STAGE, SPB, CAP><<<B.nblk, 4 * SPB, 0, st>>>(b, (const T*)w_in, (T*)w_out, (T*)acc, reunit);
}

template <int P, int STAGE, int SPB>
static void launch_p(const Batch& B, const void* w_in, void* w_out, void* acc, int reunit, cudaStream_t st) {
    if (B.ncfg <= kSmallCap)
        launch_cap<P, STAGE, SPB, kSmallCap>(B, w_in, w_out, acc, reunit, st);
    else
        launch_cap<P, STAGE, SPB, kMaxCfg>(B, w_in, w_out, acc, reunit, st);
}

template <int P>
static void launch_stage_p(int stage, int reunit, const Batch& B, const void* w_in, void* w_out, void* acc,
                           cudaStream_t st) {
    switch (stage) {
        case 1: launch_p<P, 1, 32>(B, w_in, w_out, acc, reunit, st); break;
        case 2: launch_p<P, 2, 32>(B, w_in, w_out, acc, reunit, st); break;
        default: launch_p<P, 3, 32>(B, w_in, w_out, acc, reunit, st); break;
    }
}

void launch_stage(int prec, int stage, int reunit, const Batch& B, const void* w_in, void* w_out, void* acc,
                  int sites_per_block, cudaStream_t st) {
    (void)sites_per_block;
    if (prec == P64) launch_stage_p<P64>(stage, reunit, B, w_in, w_out, acc, st);
    else if (prec == P32) launch_stage_p<P32>(stage, reunit, B, w_in, w_out, acc, st);
    else launch_stage_p<P32R12>(stage, reunit, B, w_in, w_out, acc, st);
}

}  // namespace tgf
