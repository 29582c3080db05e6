// pack.cu -- canonical FP64 link layout <-> device storage planes.
//
// Canonical: per configuration [site][mu][row][col][re,im] doubles (x0 fastest within site).
// For these launches CfgDesc::x_off is the configuration's offset in the canonical buffer
// (doubles) and blocks cover 32 sites x 4 directions (one thread per link).
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace tgf {

template <int P, int CAP>
__global__ void __launch_bounds__(128)
k_pack(const __grid_constant__ BatchT<CAP> B, const double* __restrict__ canon, typename Store<P>::T* __restrict__ w) {
    using T = typename Store<P>::T;
    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int mu = threadIdx.x >> 5;
        const int s = (blk - c.blk0) * 32 + (threadIdx.x & 31);
        if (s >= c.V) continue;
        const double* src = canon + c.x_off + ((size_t)s * 4 + mu) * 18;
        mat3<T> u;
#pragma unroll
        for (int k = 0; k < 9; ++k) u.e[k / 3][k % 3] = {(T)src[2 * k], (T)src[2 * k + 1]};
        Store<P>::store(w + c.w_off + (size_t)mu * Store<P>::reals * c.Vp, c.Vp, s, u);
    }
}

template <int P, int CAP>
__global__ void __launch_bounds__(128)
k_unpack(const __grid_constant__ BatchT<CAP> B, const typename Store<P>::T* __restrict__ w, double* __restrict__ canon) {
    using T = typename Store<P>::T;
    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int mu = threadIdx.x >> 5;
        const int s = (blk - c.blk0) * 32 + (threadIdx.x & 31);
        if (s >= c.V) continue;
        mat3<T> u;
        Store<P>::load(w + c.w_off + (size_t)mu * Store<P>::reals * c.Vp, c.Vp, s, u);
        double* dst = canon + c.x_off + ((size_t)s * 4 + mu) * 18;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            dst[2 * k] = (double)u.e[k / 3][k % 3].re;
            dst[2 * k + 1] = (double)u.e[k / 3][k % 3].im;
        }
    }
}

template <int P>
static void pack_p(const Batch& B, const double* canon, void* w, cudaStream_t st) {
    using T = typename Store<P>::T;
    if (B.ncfg <= kSmallCap) {
        BatchT<kSmallCap> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_pack<P, kSmallCap><<<B.nblk, 128, 0, st>>>(b, canon, (T*)w);
    } else {
        k_pack<P, kMaxCfg><<<B.nblk, 128, 0, st>>>(B, canon, (T*)w);
    }
}

template <int P>
static void unpack_p(const Batch& B, const void* w, double* canon, cudaStream_t st) {
    using T = typename Store<P>::T;
    if (B.ncfg <= kSmallCap) {
        BatchT<kSmallCap> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_unpack<P, kSmallCap><<<B.nblk, 128, 0, st>>>(b, (const T*)w, canon);
    } else {
        k_unpack<P, kMaxCfg><<<B.nblk, 128, 0, st>>>(B, (const T*)w, canon);
    }
}

void launch_pack(int prec, const Batch& B, const double* canon, void* w, cudaStream_t st) {
    if (prec == P64) pack_p<P64>(B, canon, w, st);
    else if (prec == P32) pack_p<P32>(B, canon, w, st);
    else pack_p<P32R12>(B, canon, w, st);
}

void launch_unpack(int prec, const Batch& B, const void* w, double* canon, cudaStream_t st) {
    if (prec == P64) unpack_p<P64>(B, w, canon, st);
    else if (prec == P32) unpack_p<P32>(B, w, canon, st);
    else unpack_p<P32R12>(B, w, canon, st);
}

TGF_CHECK_WORD(pack)

}  // namespace tgf
