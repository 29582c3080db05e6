// measure.cu -- observables E, Q, P of every configuration from the clover halves.
//
// The stage kernel (modes 1 and 2) leaves, per site and plane, the two halves of the clover's
// anti-Hermitian part A = C - C^+ (so G = -(i/8) A, eq. gmunu) and the twisted plaquette
// trace.  k_clover_sum adds the halves and accumulates per site
//   e(n) = sum_{mu<nu} |A_{mu nu}|_F^2            (Tr G^2 = |A|^2 / 64)
//   q(n) = <A01,A23> - <A02,A13> + <A03,A12>       (Tr G_a G_b = <A_a,A_b> / 64, <X,Y> = Re sum X conj(Y))
//   s(n) = sum_{mu<nu} (3 - Re Tr[Z* P_{mu nu}(n)])
// in the working precision (the stage kernel stores each plane's 3 - Re Tr[Z* P], so the small
// deviations are summed, not six numbers near 3), then reduces them over the block in FP64 (warp
// shuffles, fixed order) to one partial per block.  k_reduce sums each configuration's partials in
// block order and writes {t, E, Q, P, S} with E = sum e/(64 V), Q = sum q/(256 pi^2) (eq. qlatt
// with Gt_{mu nu} = eps_{mu nu rho sigma} G_{rho sigma}/2), S = sum s, P = 1 - S/(18 V).
// Both orders are fixed: results are bitwise reproducible.
#include <cuda_runtime.h>

#include "lattice.cuh"

namespace tgf {

// First observable slot (o_off + 1) whose record came out non-finite since the host last read
// the word; 0 if none.  Read and cleared by nonfinite_read_and_clear().
__device__ unsigned long long g_nonfinite;

unsigned long long nonfinite_read_and_clear(cudaStream_t st, cudaError_t* err) {
    unsigned long long v = 0, z = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_nonfinite, sizeof v, 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_nonfinite, &z, sizeof z, 0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *err = e;
    return e == cudaSuccess ? v : 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <class T, int CAP>
__global__ void __launch_bounds__(kMeasureSites)
k_clover_sum(const __grid_constant__ BatchT<CAP> B, const T* __restrict__ clov, double* __restrict__ partial,
             int traceless) {
    __shared__ double red[kMeasureSites / 32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int s = (blk - c.blk0) * kMeasureSites + threadIdx.x;
        double e = 0, q = 0, pl = 0;
        if (s < c.V) {
            const T* cb = clov + c.m_off;
            const size_t Vp = (size_t)c.Vp;
            T te = T(0), tq = T(0), tp = T(0);
            T a0[9];
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                T a[9], a1[9];
                AhStore<T>::load(cb + (size_t)(p * 2) * 9 * Vp, (int)Vp, s, a);
                AhStore<T>::load(cb + (size_t)(p * 2 + 1) * 9 * Vp, (int)Vp, s, a1);
#pragma unroll
                for (int k = 0; k < 9; ++k) a[k] += a1[k];
                if (traceless) {
                    const T tr = (a[0] + a[1] + a[2]) * (T(1) / T(3));
                    a[0] -= tr; a[1] -= tr; a[2] -= tr;
                }
                te += a[0] * a[0] + a[1] * a[1] + a[2] * a[2] +
                      T(2) * (a[3] * a[3] + a[4] * a[4] + a[5] * a[5] + a[6] * a[6] + a[7] * a[7] + a[8] * a[8]);
                if (p & 1) {
                    const T d = a0[0] * a[0] + a0[1] * a[1] + a0[2] * a[2] +
                                T(2) * (a0[3] * a[3] + a0[4] * a[4] + a0[5] * a[5] + a0[6] * a[6] + a0[7] * a[7] + a0[8] * a[8]);
                    tq += (p == 3) ? -d : d;
                } else {
#pragma unroll
                    for (int k = 0; k < 9; ++k) a0[k] = a[k];
                }
                tp += __ldg(cb + (size_t)(108 + p) * Vp + s);
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
        const double E = red[0][0] / (64.0 * V), Q = red[1][0] / (256.0 * pi * pi), S = red[2][0];
        o[0] = c.h;                                   // t
        o[1] = E;
        o[2] = Q;
        o[3] = 1.0 - S / (18.0 * V);                  // P = (1/(18V)) sum Re Tr[Z* P]
        o[4] = S;                                     // S = sum (3 - Re Tr[Z* P])
        // a non-finite record (non-finite links in, or an overflow) is reported to the host
        if (!isfinite(E) || !isfinite(Q) || !isfinite(S))
            atomicCAS(&g_nonfinite, 0ull, (unsigned long long)c.o_off + 1ull);
    }
}

// q(x0, t) (Sec. 4): the charge density summed over the slab x_dir = x of each configuration,
// one block per (configuration, slab), FP64 sums in a fixed order.  The launch descriptor has
// L[dir] blocks per configuration; q_out[cfg_index * q_stride + x] with cfg_index = c.o_off.
template <class T, int CAP>
__global__ void __launch_bounds__(256)
k_slice_charge(const __grid_constant__ BatchT<CAP> B, const T* __restrict__ clov, int dir, double* __restrict__ q_out,
               int q_stride, int traceless) {
    __shared__ double red[256];
    for (int blk = blockIdx.x; blk < B.nblk; blk += gridDim.x) {
        const int ci = find_cfg(B, blk);
        const CfgDesc& c = B.c[ci];
        const int x = blk - c.blk0;
        const int n_slab = c.V / c.L[dir];
        const T* cb = clov + c.m_off;
        const size_t Vp = (size_t)c.Vp;
        double acc = 0.0;
        for (int j = threadIdx.x; j < n_slab; j += 256) {
            int r = j, s = x * c.st[dir];
#pragma unroll
            for (int d = 0; d < 4; ++d) {
                if (d == dir) continue;
                s += (r % c.L[d]) * c.st[d];
                r /= c.L[d];
            }
            T a0[9], tq = T(0);
#pragma unroll
            for (int p = 0; p < 6; ++p) {
                T a[9], a1[9];
                AhStore<T>::load(cb + (size_t)(p * 2) * 9 * Vp, (int)Vp, s, a);
                AhStore<T>::load(cb + (size_t)(p * 2 + 1) * 9 * Vp, (int)Vp, s, a1);
#pragma unroll
                for (int k = 0; k < 9; ++k) a[k] += a1[k];
                if (traceless) {
                    const T tr = (a[0] + a[1] + a[2]) * (T(1) / T(3));
                    a[0] -= tr; a[1] -= tr; a[2] -= tr;
                }
                if (p & 1) {
                    const T d = a0[0] * a[0] + a0[1] * a[1] + a0[2] * a[2] +
                                T(2) * (a0[3] * a[3] + a0[4] * a[4] + a0[5] * a[5] + a0[6] * a[6] + a0[7] * a[7] + a0[8] * a[8]);
                    tq += (p == 3) ? -d : d;
                } else {
#pragma unroll
                    for (int k = 0; k < 9; ++k) a0[k] = a[k];
                }
            }
            acc += (double)tq;
        }
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double pi = 3.14159265358979323846;
            q_out[(size_t)c.o_off * q_stride + x] = red[0] / (256.0 * pi * pi);
        }
        __syncthreads();
    }
}

template <class T, int CAP>
static void slices_cap(const Batch& B, const void* clov, int dir, double* q, int q_stride, unsigned flags,
                       cudaStream_t st) {
    if constexpr (CAP == kMaxCfg) {
        k_slice_charge<T, kMaxCfg><<<B.nblk, 256, 0, st>>>(B, (const T*)clov, dir, q, q_stride, (int)(flags & 1u));
    } else {
        BatchT<CAP> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_slice_charge<T, CAP><<<B.nblk, 256, 0, st>>>(b, (const T*)clov, dir, q, q_stride, (int)(flags & 1u));
    }
}

void launch_slice_charge(int prec, unsigned flags, const Batch& B, const void* clov, int dir, double* q, int q_stride,
                         cudaStream_t st) {
    const bool small = B.ncfg <= kSmallCap;
    if (prec == P64) small ? slices_cap<double, kSmallCap>(B, clov, dir, q, q_stride, flags, st)
                           : slices_cap<double, kMaxCfg>(B, clov, dir, q, q_stride, flags, st);
    else small ? slices_cap<float, kSmallCap>(B, clov, dir, q, q_stride, flags, st)
               : slices_cap<float, kMaxCfg>(B, clov, dir, q, q_stride, flags, st);
}

template <class T, int CAP>
static void sum_cap(unsigned flags, const Batch& B, const void* clov, double* partial, cudaStream_t st) {
    if constexpr (CAP == kMaxCfg) {
        k_clover_sum<T, kMaxCfg><<<B.nblk, kMeasureSites, 0, st>>>(B, (const T*)clov, partial, (int)(flags & 1u));
    } else {
        BatchT<CAP> b;
        b.ncfg = B.ncfg;
        b.nblk = B.nblk;
        for (int i = 0; i < B.ncfg; ++i) b.c[i] = B.c[i];
        k_clover_sum<T, CAP><<<B.nblk, kMeasureSites, 0, st>>>(b, (const T*)clov, partial, (int)(flags & 1u));
    }
}

template <class T>
static void sum_t(unsigned flags, const Batch& B, const void* clov, double* partial, cudaStream_t st) {
    if (B.ncfg <= kSmallCap) sum_cap<T, kSmallCap>(flags, B, clov, partial, st);
    else sum_cap<T, kMaxCfg>(flags, B, clov, partial, st);
}

void launch_clover_sum(int prec, unsigned flags, const Batch& B, const void* clov, double* partial,
                       cudaStream_t st) {
    if (prec == P64) sum_t<double>(flags, B, clov, partial, st);
    else sum_t<float>(flags, B, clov, partial, st);
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

TGF_CHECK_WORD(measure)

}  // namespace tgf
