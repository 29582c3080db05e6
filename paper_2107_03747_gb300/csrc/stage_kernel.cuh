// stage_kernel.cuh -- one stage of the RK3 Wilson-flow step: twisted staples -> force -> X update
// -> exact exponential -> W' = exp(X) W, fused in one kernel per stage (included by stage.cu for
// the default tile and by stage_tiles.cu for the other tiles of the launch tuner).
//
// Thread mapping: a block covers SPB consecutive sites of one configuration; each of its
// 4*SPB threads owns one link (site, mu), warps grouped by mu so that every load of a
// component plane is a contiguous, 32-byte-vectorised warp access.  Neighbour links are
// read through the read-only data path (L1/L2 absorb the 19-fold reuse of each link).
#pragma once

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

// Launch tiles of the stage kernel (chosen per workload by the launch tuner, flag TGF_TUNE_TILE):
//   0  32 sites per block, one warp per direction, 4 resident blocks per SM in the FP32 forms
//      (at most 128 registers per thread), 2 in FP64
//   1  64 sites per block, two warps per direction (a block spans two 32-site rows), 2 resident
//      blocks of 256 threads per SM (at most 128 registers)
//   2  32 sites per block as a 4 x 2 x 2 x 2 hypercube (x0 x1 x2 x3) instead of 32 consecutive
//      sites: a run of 4 sites along x0 is one full 128-byte line of a 32-byte plane, and more of
//      the neighbours along x1, x2, x3 fall inside the block (used where L0 is a multiple of 4
//      and L1, L2, L3 are even; other configurations of the launch keep the consecutive order)
//   3  as 0, and in the unmeasured stages the block's direction warps share the forward-staple
//      corners T_ab in pairs through shared memory (below)
//   4  as 0 with a tighter register cap in the unmeasured stages: 5 resident blocks per SM (at
//      most 102 registers; the measured stage 1 keeps 4), more warps to cover latency
// Tiles 1 to 4 exist for the FP32 forms only.  Tiles 0, 1, 2 and 4 compute the same flow bit for
// bit; tile 3 forms the shared staples as (Z T_ba)^+ U^+ instead of Z* T_ab U^+, equal up to
// rounding.
template <int TILE>
struct StageTile {
    static constexpr int spb = TILE == 1 ? 64 : 32;
    static constexpr int minb32 = TILE == 1 ? 2 : TILE == 4 ? 5 : 4;
    static constexpr bool cube = TILE == 2;
    static constexpr bool pair = TILE == 3;
};

// Site of lane `lane` in block `b` (index within its configuration) of a hypercube tile: the
// block's origin (4 h0, 2 h1, 2 h2, 2 h3) from the multiply-shift constants of the fine strides,
// floor(b / (L0/4)) = floor(4b / L0) etc. (exact: L0/4, L1/2, L2/2 are integers); lanes cover
// dx0 = lane & 3, dx1..dx3 = the next three bits.  Returns false if the extents do not allow it.
__device__ __forceinline__ bool cube_site(const CfgDesc& c, int b, int lane, int& s, int (&x)[4]) {
    if ((c.L[0] & 3) | (c.L[1] & 1) | (c.L[2] & 1) | (c.L[3] & 1)) return false;
    const unsigned u = (unsigned)b;
    const int q1 = (int)(__umulhi(u << 6, c.dmul[0]) >> c.dsh[0]);  // b / (L0/4)
    const int q2 = (int)(__umulhi(u << 7, c.dmul[1]) >> c.dsh[1]);  // b / (L0 L1/8)
    const int q3 = (int)(__umulhi(u << 8, c.dmul[2]) >> c.dsh[2]);  // b / (L0 L1 L2/16)
    x[0] = 4 * (b - q1 * (c.L[0] >> 2)) + (lane & 3);
    x[1] = 2 * (q1 - q2 * (c.L[1] >> 1)) + ((lane >> 2) & 1);
    x[2] = 2 * (q2 - q3 * (c.L[2] >> 1)) + ((lane >> 3) & 1);
    x[3] = 2 * q3 + (lane >> 4);
    s = x[0] + x[1] * c.st[1] + x[2] * c.st[2] + x[3] * c.st[3];
    return true;
}

// Tile 3: forward-staple corners shared in pairs.  T_ab(n) = U_b(n+a) U_a(n+b)^+ serves link (n, a)
// (staple T_ab U_b(n)^+) and link (n, b) (staple T_ab^+ U_a(n)^+ = T_ba U_a(n)^+), so of the two
// direction warps of a plane one forms T and the other reads it from shared memory.  The
// producer signals with bar.arrive on the plane's named barrier (64 threads: both warps) and goes
// on; the consumer waits with bar.sync.  Order of nu per warp mu and which planes it forms: every
// warp forms its planes before it reads any, so no wait can close a cycle, and every plane is
// read at a later position of the reader's order than the one at which its producer forms it,
// so a consumer rarely finds its corner not yet written:
//   mu 0: nu 1 (forms 01), 3 (reads 03), 2 (reads 02)
//   mu 1: nu 2 (forms 12), 3 (forms 13), 0 (reads 01)
//   mu 2: nu 3 (forms 23), 0 (forms 02), 1 (reads 12)
//   mu 3: nu 0 (forms 03), 2 (reads 23), 1 (reads 13)
static __constant__ int8_t c_pair_nu[4][3] = {{1, 3, 2}, {2, 3, 0}, {3, 0, 1}, {0, 2, 1}};
static __constant__ int8_t c_pair_own[4][4] = {{0, 1, 0, 0}, {0, 0, 1, 1}, {1, 0, 0, 1}, {1, 0, 0, 0}};
__device__ __forceinline__ void bar_arrive(int id, int nthreads) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void bar_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// the measured stage 1 (MODE 1: clover halves too) needs more registers: at most 4 blocks per SM
template <int P, int TILE, int MODE>
constexpr int stage_min_blocks() {
    return P == P64 ? 2 : (MODE != 0 && StageTile<TILE>::minb32 > 4) ? 4 : StageTile<TILE>::minb32;
}

// Plane index of (mu, nu), mu < nu, in the order 01, 23, 02, 13, 03, 12 (consecutive planes
// pair up in the topological charge); -1 for mu >= nu.
static __constant__ int8_t c_plane_of[4][4] = {{-1, 0, 2, 4}, {-1, -1, 5, 3}, {-1, -1, -1, 1}, {-1, -1, -1, -1}};
static __constant__ int8_t c_pair[6][2] = {{0, 1}, {2, 3}, {0, 2}, {1, 3}, {0, 3}, {1, 2}};
// Which direction's warp builds the clover halves of each plane: 01, 02 by warp 0; 12, 13 by
// warp 1; 23 by warp 2; 03 by warp 3 -- two planes at most per warp instead of 3, 2, 1, 0.
static __constant__ int8_t c_clover_owner[4][4] = {{0, 1, 1, 0}, {0, 0, 1, 1}, {0, 0, 0, 1}, {1, 0, 0, 0}};

// The anti-Hermitian part D - D^+ of a 3x3 matrix as 9 reals (2 Im D_jj; D_jk - conj(D_kj), j<k),
// written to one slot of the clover scratch (AhStore).
template <class T>
__device__ __forceinline__ void store_ah(T* __restrict__ p, int Vp, int s, const mat3<T>& d) {
    const T v[9] = {T(2) * d.e[0][0].im,           T(2) * d.e[1][1].im,           T(2) * d.e[2][2].im,
                    d.e[0][1].re - d.e[1][0].re, d.e[0][1].im + d.e[1][0].im, d.e[0][2].re - d.e[2][0].re,
                    d.e[0][2].im + d.e[2][0].im, d.e[1][2].re - d.e[2][1].re, d.e[1][2].im + d.e[2][1].im};
    AhStore<T>::store(p, Vp, s, v);
}

// MODE 0: the RK3 stage.  MODE 1: the stage, and from the same staples of the input field the
// clover halves used by the measurement.  MODE 2: the clover halves only.
//
// Clover from staples.  With F, B the forward and backward twisted staples of link U_mu(n) in
// direction nu (below), the four leaves of eq. (gmunu) are L1 = U F, L2 = B^+ U^+ (both from
// link (n, mu)) and L3 = F' U', L4 = U'^+ B'^+ (from link (n - mu, mu), primed), so
//   C - C^+ = [D1 - D1^+] + [D2 - D2^+],  D1 = U (F - B) at n,  D2 = (F' - B') U' carried to n.
// Thread (n, mu) writes D1 - D1^+ to site n and D2 - D2^+ to site n + mu for the planes its warp
// builds (c_clover_owner), plus 3 - Re Tr(U F) (the twisted plaquette at n).
template <int P, int STAGE, int MODE, int TILE, int CAP>
__global__ void __launch_bounds__(4 * StageTile<TILE>::spb, (stage_min_blocks<P, TILE, MODE>()))
k_stage(const __grid_constant__ BatchT<CAP> B, const typename Store<P>::T* __restrict__ w_in,
        typename Store<P>::T* __restrict__ w_out, typename Store<P>::T* __restrict__ acc,
        typename Store<P>::T* __restrict__ clov, int reunit) {
    using T = typename Store<P>::T;
    using S = Store<P>;
    constexpr int R = S::reals;
    constexpr int SPB = StageTile<TILE>::spb;
    static_assert(P != P64 || TILE == 0, "FP64 shares the block's forward-staple corners: tile 0 only");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mu = warp & 3;
    const int row = warp >> 2;  // which 32-site row of the block
    // T_{ab}(n) = U_b(n+a) U_a(n+b)^+ of the six planes a < b: the forward staple of link (n, a) in
    // direction b is T_ab U_b(n)^+, that of link (n, b) in direction a is T_ab^+ U_a(n)^+, so in
    // FP64 (bound by the FP64 pipe) each is computed once per site by one warp of the block and
    // shared behind one block barrier (42 instead of 48 staple products per site).  The FP32 forms,
    // bound by latency, share them only in launch tile 3, in pairs of warps without a block barrier.
    constexpr bool SHARE = (P == P64);
    __shared__ cx<T> sT[SHARE ? 6 : 1][9][32];
    // tile 3 (FP32 forms, unmeasured stages): corners shared in pairs; every lane of the block's four
    // warps takes part in the named barriers, lanes past the configuration's end on site 0 with
    // their results discarded
    constexpr bool PAIR = (P != P64) && StageTile<TILE>::pair && MODE == 0;
    __shared__ cx<T> sP[PAIR ? 6 : 1][9][32];

    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        int s_raw = (blk - c.blk0) * SPB + row * 32 + lane;
        int xc[4];
        bool have_x = false;
        if constexpr (StageTile<TILE>::cube) have_x = cube_site(c, blk - c.blk0, lane, s_raw, xc);
        const bool valid = s_raw < c.V;
        const int s = (PAIR && !valid) ? 0 : s_raw;
        if (!have_x) site_coords(c, valid ? s : 0, xc);
        const unsigned eb = edge_bits(c, xc);  // boundary flags (lattice.cuh)
        const int Vp = c.Vp;
        const T* base = w_in + c.w_off;
        auto link = [&](int dir, int site, mat3<T>& u) { S::load(base + (size_t)dir * R * Vp, Vp, site, u); };
        // Two-row storage: the first factor of a link-by-link product is read without its third
        // row, the product's rows 0 and 1 are formed and its row 2 is rebuilt once (an SU(3)
        // product), which saves rebuilding that factor's row on load.
        constexpr bool TWO_ROW = (P == P32R12);
        // out = U_da(sa) U_db(sb)^+ (prod_nd) or U_da(sa) U_db(sb) (prod_nn); fa, fb receive the factors
        auto prod_nd = [&](mat3<T>& out, int da, int sa, int db, int sb, mat3<T>& fa, mat3<T>& fb) {
            if constexpr (TWO_ROW) {
                Store<P32R12>::load_top(base + (size_t)da * R * Vp, Vp, sa, fa);
                link(db, sb, fb);
                mul_nd_top(out, fa, fb);
                rebuild_row2(out);
            } else {
                link(da, sa, fa);
                link(db, sb, fb);
                mul_nd(out, fa, fb);
            }
        };
        auto prod_nn = [&](mat3<T>& out, int da, int sa, int db, int sb, mat3<T>& fa, mat3<T>& fb) {
            if constexpr (TWO_ROW) {
                Store<P32R12>::load_top(base + (size_t)da * R * Vp, Vp, sa, fa);
                link(db, sb, fb);
                mul_nn_top(out, fa, fb);
                rebuild_row2(out);
            } else {
                link(da, sa, fa);
                link(db, sb, fb);
                mul_nn(out, fa, fb);
            }
        };
        mat3<T> sig, a, b, t;
        if constexpr (SHARE) {
            // phase 1: warp w builds T of planes w and w + 4 (pair order 01, 23, 02, 13, 03, 12)
            for (int pr = warp; pr < 6; pr += 4) {
                if (!valid) break;
                const int pa = c_pair[pr][0], pb = c_pair[pr][1];
                link(pb, fwd(c, eb, s, pa), a);
                link(pa, fwd(c, eb, s, pb), b);
                mul_nd(t, a, b);
#pragma unroll
                for (int k = 0; k < 9; ++k) sT[pr][k][lane] = t.e[k / 3][k % 3];
            }
            __syncthreads();
        }
        auto link_body = [&]() {
        const int s_mp = fwd(c, eb, s, mu);
        const bool at_mu0 = (eb >> mu) & 1u;  // x_mu = 0: the twisted plaquettes' corner row
        if (MODE != 2) set_zero(sig);
#pragma unroll 1
        for (int dn = 1; dn < 4; ++dn) {
            const int nu = PAIR ? (int)c_pair_nu[mu][dn - 1] : (mu + dn) & 3;
            const bool clover = MODE != 0 && c_clover_owner[mu][nu];
            if (MODE == 2 && !clover) continue;
            const int s_nm = bwd(c, eb, s, nu);
            const int s_mp_nm = fwd(c, eb, s_nm, mu);  // x_mu(n - nu) = x_mu(n)
            const int k = c.tw[mu * 4 + nu];
            T zr = T(1), zi = T(0);
            if (k != 0) centre<T>(k, zr, zi);
            // forward staple F = Z*_{mu nu}(n) U_nu(n+mu) U_mu(n+nu)^+ U_nu(n)^+ = Z* T_{mu nu} U_nu(n)^+
            const bool tw_f = k != 0 && at_mu0 && ((eb >> nu) & 1u);
            mat3<T> f;
            bool fwd_done = false;  // tile 3: a consumer's shared staple is already in sig
            if constexpr (SHARE) {
                // T_{mu nu} = T_{nu mu}^+ from the block's shared T of the plane
                const int pl_f = c_plane_of[mu < nu ? mu : nu][mu < nu ? nu : mu];
#pragma unroll
                for (int kk = 0; kk < 9; ++kk) t.e[kk / 3][kk % 3] = sT[pl_f][kk][lane];
            } else if constexpr (PAIR) {
                const int pl_f = c_plane_of[mu < nu ? mu : nu][mu < nu ? nu : mu];
                if (c_pair_own[mu][nu]) {
                    prod_nd(t, nu, s_mp, mu, fwd(c, eb, s, nu), a, b);  // T_{mu nu}
#pragma unroll
                    for (int kk = 0; kk < 9; ++kk) sP[pl_f][kk][lane] = t.e[kk / 3][kk % 3];
                    bar_arrive(1 + pl_f, 64);
                } else {
                    // F = Z*_{mu nu} T_{nu mu}^+ U_nu(n)^+ = (Z_{mu nu} T_{nu mu})^+ U_nu(n)^+
                    bar_sync(1 + pl_f, 64);
#pragma unroll
                    for (int kk = 0; kk < 9; ++kk) t.e[kk / 3][kk % 3] = sP[pl_f][kk][lane];
                    link(nu, s, a);
                    if (tw_f) scale_cx(t, zr, zi);
                    mul_dd_acc(sig, t, a);
                    fwd_done = true;
                }
            } else {
                prod_nd(t, nu, s_mp, mu, fwd(c, eb, s, nu), a, b);  // T = U_nu(n+mu) U_mu(n+nu)^+
            }
            if (!fwd_done) {
            link(nu, s, a);
            if (!SHARE || nu > mu) {
                if (clover) {
                    mul_nd(f, t, a);
                    if (tw_f) scale_cx(f, zr, -zi);
                    if (MODE != 2) add_to(sig, f);
                } else {
                    // the centre factor scales T before the accumulating product (Z* T U^+), so a
                    // twisted corner needs no separate staple matrix
                    if (tw_f) scale_cx(t, zr, -zi);
                    mul_nd_acc(sig, t, a);
                }
            } else {
                // F = T_{nu mu}^+ U_nu(n)^+ = (U_nu(n) T_{nu mu})^+
                mul_nn(b, a, t);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) f.e[i][j] = {b.e[j][i].re, -b.e[j][i].im};
                if (tw_f) scale_cx(f, zr, -zi);
                add_to(sig, f);
            }
            }
            // backward staple B = Z_{mu nu}(n-nu) U_nu(n+mu-nu)^+ U_mu(n-nu)^+ U_nu(n-nu)
            prod_nn(t, mu, s_nm, nu, s_mp_nm, a, b);  // U_mu(n-nu) U_nu(n+mu-nu)
            link(nu, s_nm, a);
            const bool tw_b = k != 0 && at_mu0 && ((eb >> (8 + nu)) & 1u);
            if (clover) {
                mul_dn(b, t, a);
                if (tw_b) scale_cx(b, zr, zi);
                if (MODE != 2) add_to(sig, b);
            } else {
                if (tw_b) scale_cx(t, zr, -zi);  // Z t^+ a = (Z* t)^+ a
                mul_dn_acc(sig, t, a);
            }
            if (clover) {
                const int pl = c_plane_of[mu < nu ? mu : nu][mu < nu ? nu : mu];
                T* cb = clov + c.m_off;
                link(mu, s, a);  // U = U_mu(n)
                // 3 - Re Tr(U F): the twisted plaquette Z* P_{mu nu}(n) as its deviation from the
                // unit matrix (exact subtraction for traces in [1.5, 6])
                T rt = T(0);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        rt = fma(a.e[i][j].re, f.e[j][i].re, fma(-a.e[i][j].im, f.e[j][i].im, rt));
                cb[(size_t)(108 + pl) * Vp + s] = T(3) - rt;
                // K = F - B; D1 = U K (site n), D2 = K U (site n + mu).  A plane built through its
                // second direction (nu < mu) takes K = B - F: the leaves of the plane (mu, nu) are the
                // Hermitian conjugates of those of (nu, mu), so its C - C^+ changes sign.
                const T sg = nu > mu ? T(1) : T(-1);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        f.e[i][j].re = sg * (f.e[i][j].re - b.e[i][j].re);
                        f.e[i][j].im = sg * (f.e[i][j].im - b.e[i][j].im);
                    }
                mul_nn(t, a, f);
                store_ah(cb + (size_t)(pl * 2 + 0) * 9 * Vp, Vp, s, t);
                mul_nn(t, f, a);
                store_ah(cb + (size_t)(pl * 2 + 1) * 9 * Vp, Vp, s_mp, t);
            }
        }
        if (MODE == 2) return;
        // Omega = U_mu(n) Sigma, Z = -P_ta(Omega)
        mat3<T> u;
        link(mu, s, u);
        mul_nn(t, u, sig);
        alg8<T> z;
        minus_proj_ta(z, t);
        const T h = (T)c.h;
        alg8<T> x;
        T* xb = acc + c.x_off + (size_t)mu * 8 * Vp;
        if (STAGE == 1) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = T(0.25) * h * z.v[i];
            if (valid) AccStore<T>::store(xb, Vp, s, x);
        } else if (STAGE == 2) {
            AccStore<T>::load(xb, Vp, s, x);
            const T c1 = T(8) / T(9), c2 = T(17) / T(9);
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = c1 * h * z.v[i] - c2 * x.v[i];
            if (valid) AccStore<T>::store(xb, Vp, s, x);
        } else {
            AccStore<T>::load(xb, Vp, s, x);
#pragma unroll
            for (int i = 0; i < 8; ++i) x.v[i] = T(0.75) * h * z.v[i] - x.v[i];
        }
        // W' = W + (exp(X) - 1) W: the update rounds once on top of W instead of through a full
        // product, which keeps the FP32 forms' drift off SU(3) small between re-projections (W must
        // not enter the product's accumulators: their roundings would then be relative to W)
        expm_su3<T, true>(b, x);
        if constexpr (TWO_ROW) mul_nn_plus_top(t, b, u, u);  // only rows 0 and 1 are stored
        else mul_nn_plus(t, b, u, u);
        if (STAGE == 3 && P != P64 && reunit) reunitarize(t);
        if (valid) S::store(w_out + c.w_off + (size_t)mu * R * Vp, Vp, s, t);
        };
        if (valid || PAIR) link_body();
        // sT / sP are rewritten by the next block of the grid-stride loop
        if constexpr (SHARE || PAIR) __syncthreads();
    }
}

template <int P, int STAGE, int MODE, int TILE, int CAP>
static void launch_cap(const Batch& B, const void* w_in, void* w_out, void* acc, void* clov, int reunit,
                       cudaStream_t st, int grid) {
    using T = typename Store<P>::T;
    constexpr int SPB = StageTile<TILE>::spb;
    const int g = (grid > 0 && grid < B.nblk) ? grid : B.nblk;
    if constexpr (CAP == kMaxCfg) {
        k_stage<P, STAGE, MODE, TILE, kMaxCfg><<<g, 4 * SPB, 0, st>>>(B, (const T*)w_in, (T*)w_out, (T*)acc,
                                                                     (T*)clov, reunit);
    } else {
        BatchT<CAP> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_stage<P, STAGE, MODE, TILE, CAP><<<g, 4 * SPB, 0, st>>>(b, (const T*)w_in, (T*)w_out, (T*)acc,
                                                                 (T*)clov, reunit);
    }
}

template <int P, int STAGE, int MODE, int TILE>
static void launch_m(const Batch& B, const void* w_in, void* w_out, void* acc, void* clov, int reunit,
                     cudaStream_t st, int grid) {
    if (B.ncfg <= kSmallCap)
        launch_cap<P, STAGE, MODE, TILE, kSmallCap>(B, w_in, w_out, acc, clov, reunit, st, grid);
    else
        launch_cap<P, STAGE, MODE, TILE, kMaxCfg>(B, w_in, w_out, acc, clov, reunit, st, grid);
}

template <int P, int TILE>
static void launch_stage_p(int stage, int mode, int reunit, const Batch& B, const void* w_in, void* w_out,
                           void* acc, void* clov, cudaStream_t st, int grid) {
    if constexpr (TILE == 0)
        if (mode == 2) return launch_m<P, 1, 2, 0>(B, w_in, w_out, acc, clov, reunit, st, grid);
    switch (stage) {
        case 1:
            if (mode == 1) launch_m<P, 1, 1, TILE>(B, w_in, w_out, acc, clov, reunit, st, grid);
            else launch_m<P, 1, 0, TILE>(B, w_in, w_out, acc, clov, reunit, st, grid);
            break;
        case 2: launch_m<P, 2, 0, TILE>(B, w_in, w_out, acc, clov, reunit, st, grid); break;
        default: launch_m<P, 3, 0, TILE>(B, w_in, w_out, acc, clov, reunit, st, grid); break;
    }
}

}  // namespace tgf
