// measure.cu -- clover field strength and the observables E, Q, P of every configuration.
//
// k_measure: one thread per site builds, for each of the six planes, the four twisted
// clover leaves (eq. gmunu) and A = C - C^+ (so G = -(i/8) A), and accumulates per site
//   e(n) = sum_{mu<nu} |A_{mu nu}|_F^2            (Tr G^2 = |A|^2 / 64)
//   q(n) = <A01,A23> - <A02,A13> + <A03,A12>       (Tr G_a G_b = <A_a,A_b> / 64, <X,Y> = Re sum X conj(Y))
//   p(n) = sum_{mu<nu} Re Tr[Z* P_{mu nu}(n)]
// in the working precision, then reduces them over the block in FP64 (warp shuffles, fixed
// order) to one partial per block.  k_reduce sums each configuration's partials in block order
// and writes {t, E, Q, P, S} with E = sum e/(64 V), Q = sum q/(256 pi^2), P = sum p/(18 V),
// S = 18 V - sum p.  Both orders are fixed: results are bitwise reproducible.
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace tgf {

// anti-Hermitian A = C - C^+ stored as 9 reals: Im A_jj (3) and A_01, A_02, A_12 (complex)
template <class T>
struct ah9 {
    T d[3];
    cx<T> o[3];
};

template <class T>
__device__ __forceinline__ void antiherm(ah9<T>& A, const mat3<T>& C, bool traceless) {
    A.d[0] = T(2) * C.e[0][0].im;
    A.d[1] = T(2) * C.e[1][1].im;
    A.d[2] = T(2) * C.e[2][2].im;
    if (traceless) {
        T tr = (A.d[0] + A.d[1] + A.d[2]) / T(3);
        A.d[0] -= tr; A.d[1] -= tr; A.d[2] -= tr;
    }
    A.o[0] = {C.e[0][1].re - C.e[1][0].re, C.e[0][1].im + C.e[1][0].im};
    A.o[1] = {C.e[0][2].re - C.e[2][0].re, C.e[0][2].im + C.e[2][0].im};
    A.o[2] = {C.e[1][2].re - C.e[2][1].re, C.e[1][2].im + C.e[2][1].im};
}

// <A, B> = Re sum_ij A_ij conj(B_ij) (lower triangle doubles the upper one)
template <class T>
__device__ __forceinline__ T ah_dot(const ah9<T>& A, const ah9<T>& B) {
    T d = A.d[0] * B.d[0] + A.d[1] * B.d[1] + A.d[2] * B.d[2];
    T o = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) o += A.o[k].re * B.o[k].re + A.o[k].im * B.o[k].im;
    return d + T(2) * o;
}

template <int P, int CAP>
struct Clover {
    using T = typename Store<P>::T;
    using S = Store<P>;
    const T* base;
    int Vp;
    const Site& p;
    const CfgDesc& c;

    __device__ __forceinline__ void link(int dir, int site, mat3<T>& u) const {
        S::load(base + (size_t)dir * S::reals * Vp, Vp, site, u);
    }

    // leaf += z* M for a leaf whose base plaquette sits at a twisted corner
    __device__ __forceinline__ static void add_leaf(mat3<T>& C, mat3<T>& M, int k, bool at_corner) {
        if (k != 0 && at_corner) {
            T zr, zi;
            centre<T>(k, zr, zi);
            scale_cx(M, zr, -zi);
        }
        add_to(C, M);
    }

    // C_{mu nu}(n) (sum of the four twisted leaves) and Re Tr of the first leaf
    __device__ __forceinline__ void clover(int mu, int nu, mat3<T>& C, T& re_tr_p) const {
        const int s = p.s;
        const int k = c.tw[mu * 4 + nu];
        const int xm = p.x[mu], xn = p.x[nu];
        const int smp = nb(p, s, xm, mu, +1), smm = nb(p, s, xm, mu, -1);
        const int snp = nb(p, s, xn, nu, +1), snm = nb(p, s, xn, nu, -1);
        const int smm_np = nb(p, smm, xn, nu, +1);   // n - mu + nu
        const int smp_nm = nb(p, snm, xm, mu, +1);   // n + mu - nu
        const int smm_nm = nb(p, smm, xn, nu, -1);   // n - mu - nu
        const int xm_m = (xm == 0) ? p.L[mu] - 1 : xm - 1;
        const int xn_m = (xn == 0) ? p.L[nu] - 1 : xn - 1;
        mat3<T> a, b, t, l;
        // L1 = Z*(n) U_mu(n) U_nu(n+mu) [U_nu(n) U_mu(n+nu)]^+
        link(mu, s, a);
        link(nu, smp, b);
        mul_nn(t, a, b);
        link(nu, s, a);
        link(mu, snp, b);
        mul_nn(l, a, b);
        mul_nd(C, t, l);
        if (k != 0 && xm == 0 && xn == 0) {
            T zr, zi;
            centre<T>(k, zr, zi);
            scale_cx(C, zr, -zi);
        }
        re_tr_p = C.e[0][0].re + C.e[1][1].re + C.e[2][2].re;
        // L2 = Z*(n-nu) U_nu(n-nu)^+ [U_mu(n-nu) U_nu(n-nu+mu)] U_mu(n)^+
        link(mu, snm, a);
        link(nu, smp_nm, b);
        mul_nn(t, a, b);
        link(mu, s, a);
        mul_nd(l, t, a);
        link(nu, snm, a);
        mul_dn(t, a, l);
        add_leaf(C, t, k, xm == 0 && xn_m == 0);
        // L3 = Z*(n-mu) U_nu(n) [U_nu(n-mu) U_mu(n-mu+nu)]^+ U_mu(n-mu)
        link(nu, smm, a);
        link(mu, smm_np, b);
        mul_nn(t, a, b);
        link(nu, s, a);
        mul_nd(l, a, t);
        link(mu, smm, a);
        mul_nn(t, l, a);
        add_leaf(C, t, k, xm_m == 0 && xn == 0);
        // L4 = Z*(n-mu-nu) [U_nu(n-mu-nu) U_mu(n-mu)]^+ [U_mu(n-mu-nu) U_nu(n-nu)]
        link(nu, smm_nm, a);
        link(mu, smm, b);
        mul_nn(t, a, b);
        link(mu, smm_nm, a);
        link(nu, snm, b);
        mul_nn(l, a, b);
        mul_dn(a, t, l);
        add_leaf(C, a, k, xm_m == 0 && xn_m == 0);
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int P, int CAP>
__global__ void __launch_bounds__(kMeasureSites)
k_measure(const __grid_constant__ BatchT<CAP> B, const typename Store<P>::T* __restrict__ w,
          double* __restrict__ partial, int traceless) {
    using T = typename Store<P>::T;
    __shared__ double red[kMeasureSites / 32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int s = (blk - c.blk0) * kMeasureSites + threadIdx.x;
        double e = 0, q = 0, pl = 0;
        if (s < c.V) {
            Site p;
            make_site(p, c, s);
            Clover<P, CAP> cl{w + c.w_off, c.Vp, p, c};
            mat3<T> C;
            ah9<T> A0, A1;
            T rt, te = T(0), tq = T(0), tp = T(0);
            // (01, 23), (02, 13), (03, 12) with signs +, -, +
            const int pa[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                cl.clover(pa[r][0], pa[r][1], C, rt);
                tp += rt;
                antiherm(A0, C, traceless != 0);
                cl.clover(pa[r][2], pa[r][3], C, rt);
                tp += rt;
                antiherm(A1, C, traceless != 0);
                te += ah_dot(A0, A0) + ah_dot(A1, A1);
                const T d = ah_dot(A0, A1);
                tq += (r == 1) ? -d : d;
            }
            e = (double)te;
            q = (double)tq;
            pl = (double)tp;
        }
        e = warp_sum(e);
        q = warp_sum(q);
        pl = warp_sum(pl);
        if (lane == 0) {
            red[warp][0] = e;
            red[warp][1] = q;
            red[warp][2] = pl;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double se = 0, sq = 0, sp = 0;
#pragma unroll
            for (int i = 0; i < kMeasureSites / 32; ++i) {
                se += red[i][0];
                sq += red[i][1];
                sp += red[i][2];
            }
            double* o = partial + (size_t)blk * kPartials;
            o[0] = se;
            o[1] = sq;
            o[2] = sp;
            o[3] = 0.0;
        }
        __syncthreads();
    }
}

// One block per configuration of the launch: fixed-order sum of its partials.
template <int CAP>
__global__ void __launch_bounds__(256)
k_reduce(const __grid_constant__ BatchT<CAP> B, const double* __restrict__ partial, double* __restrict__ obs) {
    __shared__ double red[3][256];
    const CfgDesc& c = B.c[blockIdx.x];
    const int nb_cfg = (c.V + kMeasureSites - 1) / kMeasureSites;
    double e = 0, q = 0, p = 0;
    for (int i = threadIdx.x; i < nb_cfg; i += 256) {
        const double* o = partial + (size_t)(c.blk0 + i) * kPartials;
        e += o[0];
        q += o[1];
        p += o[2];
    }
    red[0][threadIdx.x] = e;
    red[1][threadIdx.x] = q;
    red[2][threadIdx.x] = p;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
            red[2][threadIdx.x] += red[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double V = (double)c.V;
        const double pi = 3.14159265358979323846;
        double* o = obs + (size_t)c.o_off * 5;
        o[0] = c.h;                                   // t
        o[1] = red[0][0] / (64.0 * V);               // E
        o[2] = red[1][0] / (256.0 * pi * pi);        // Q
        o[3] = red[2][0] / (18.0 * V);               // P
        o[4] = 18.0 * V - red[2][0];                 // S
    }
}

template <int P, int CAP>
static void measure_cap(unsigned flags, const Batch& B, const void* w, double* partial, cudaStream_t st) {
    using T = typename Store<P>::T;
    BatchT<CAP> b;
    b.ncfg = B.ncfg;
    b.nblk = B.nblk;
    for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
    k_measure<P, CAP><<<B.nblk, kMeasureSites, 0, st>>>(b, (const T*)w, partial, (int)(flags & 1u));
}

template <int P>
static void measure_p(unsigned flags, const Batch& B, const void* w, double* partial, cudaStream_t st) {
    if (B.ncfg <= kSmallCap) measure_cap<P, kSmallCap>(flags, B, w, partial, st);
    else measure_cap<P, kMaxCfg>(flags, B, w, partial, st);
}

void launch_measure(int prec, unsigned flags, const Batch& B, const void* w, double* partial, cudaStream_t st) {
    if (prec == P64) measure_p<P64>(flags, B, w, partial, st);
    else if (prec == P32) measure_p<P32>(flags, B, w, partial, st);
    else measure_p<P32R12>(flags, B, w, partial, st);
}

void launch_reduce(const Batch& B, const double* partial, double* obs, cudaStream_t st) {
    if (B.ncfg <= kSmallCap) {
        BatchT<kSmallCap> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_reduce<kSmallCap><<<B.ncfg, 256, 0, st>>>(b, partial, obs);
    } else {
        k_reduce<kMaxCfg><<<B.ncfg, 256, 0, st>>>(B, partial, obs);
    }
}

}  // namespace tgf
