// lattice.cuh -- batch descriptors, device storage layouts and neighbour indexing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "su3.cuh"

namespace tgf {

constexpr int kMaxCfg = 256;     // TGF_MAX_CFG
constexpr int kSiteAlign = 32;   // Vp = V rounded up to a multiple of this

enum Prec { P64 = 0, P32 = 1, P32R12 = 2 };

// One configuration of a launch.  Offsets are in reals of the storage type.
struct CfgDesc {
    int L[4];
    int st[4];        // strides 1, L0, L0 L1, L0 L1 L2
    int V;            // sites
    int Vp;           // padded plane length
    int blk0;         // first block of this configuration in the launch
    int rec;          // measurement record index (tgf_measure)
    int64_t w_off;    // link storage offset (reals)
    int64_t x_off;    // accumulator offset (reals)
    int64_t o_off;    // observable slot (records) = cfg * obs_stride + rec
    int64_t m_off;    // clover-halves offset in the scratch buffer (reals of the storage type)
    double h;         // step size (stages) or flow time t (measure)
    int8_t tw[16];    // n_{mu nu} mod 3 in {0,1,2}, row-major 4x4, antisymmetric mod 3
};

// Launch descriptor passed by value as a kernel parameter; CAP = 16 or kMaxCfg keeps the
// parameter block small for the common few-configuration launches.
template <int CAP>
struct BatchT {
    int ncfg;
    int nblk;         // total blocks of the launch
    CfgDesc c[CAP];
};
using Batch = BatchT<kMaxCfg>;
constexpr int kSmallCap = 16;

// Block -> configuration by binary search over blk0 (ascending).
template <int CAP>
__device__ __forceinline__ int find_cfg(const BatchT<CAP>& B, int blk) {
    int lo = 0, hi = B.ncfg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.c[mid].blk0 <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// The four coordinates of a site packed in 16-bit fields of one 64-bit register; extents and
// strides are read from the launch descriptor (parameter bank), so a direction chosen at run
// time costs a shift, not a local-memory array access.
__device__ __forceinline__ uint64_t pack_coords(const CfgDesc& c, int s) {
    int t = s;
    const uint64_t x0 = (uint64_t)(t % c.L[0]); t /= c.L[0];
    const uint64_t x1 = (uint64_t)(t % c.L[1]); t /= c.L[1];
    const uint64_t x2 = (uint64_t)(t % c.L[2]);
    const uint64_t x3 = (uint64_t)(t / c.L[2]);
    return x0 | (x1 << 16) | (x2 << 32) | (x3 << 48);
}
__device__ __forceinline__ int coord(uint64_t xp, int d) { return (int)((xp >> (16 * d)) & 0xFFFFu); }

// site index of n +- one step along a direction with coordinate x, extent L, stride st (periodic)
__device__ __forceinline__ int step_p(int s, int x, int L, int st) { return x == L - 1 ? s - (L - 1) * st : s + st; }
__device__ __forceinline__ int step_m(int s, int x, int L, int st) { return x == 0 ? s + (L - 1) * st : s - st; }

// exp(2 pi i k / 3) for k in {1, 2}
template <class T>
__device__ __forceinline__ void centre(int k, T& zr, T& zi) {
    zr = T(-0.5);
    zi = (k == 1) ? T(0.86602540378443864676) : T(-0.86602540378443864676);
}

// ---------------------------------------------------------------------------------------------
// self-checking builds (-DTGF_CHECK): every link, accumulator and clover access checks its site
// index against the plane length.  A violation sets bit 0 of the translation unit's check word
// and the access goes to site 0 instead, so nothing faults; tgf_check_errors() reads and clears
// the words.  Without TGF_CHECK the checks compile to nothing.
// ---------------------------------------------------------------------------------------------

#ifdef TGF_CHECK
static __device__ unsigned int g_tgf_check;
__device__ __forceinline__ int checked_site(int s, int n) {
    if ((unsigned)s < (unsigned)n) return s;
    atomicOr(&g_tgf_check, 1u);
    return 0;
}
// host: this translation unit's check word, cleared after reading (~0u if the copy fails)
static inline unsigned check_word_read_and_clear() {
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_tgf_check, sizeof v) != cudaSuccess) return ~0u;
    if (cudaMemcpyToSymbol(g_tgf_check, &z, sizeof z) != cudaSuccess) return ~0u;
    return v;
}
#define TGF_CHECK_WORD(name) \
    unsigned check_word_##name() { return check_word_read_and_clear(); }
#else
__device__ __forceinline__ int checked_site(int s, int) { return s; }
#define TGF_CHECK_WORD(name)
#endif

// per translation unit check words of a self-checking build
unsigned check_word_stage();
unsigned check_word_measure();
unsigned check_word_pack();
unsigned check_word_mc();
unsigned check_word_sun();

// ---------------------------------------------------------------------------------------------
// storage traits: load / store a link of direction mu at site s
// ---------------------------------------------------------------------------------------------

template <int P>
struct Store;

template <>
struct Store<P64> {
    using T = double;
    static constexpr int reals = 18;
    static __device__ __forceinline__ void load(const double* __restrict__ base, int Vp, int s, mat3<double>& u) {
        s = checked_site(s, Vp);
        const double2* q = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = __ldg(q + (size_t)k * Vp + s);
            u.e[k / 3][k % 3] = {v.x, v.y};
        }
    }
    static __device__ __forceinline__ void store(double* __restrict__ base, int Vp, int s, const mat3<double>& u) {
        s = checked_site(s, Vp);
        double2* q = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int k = 0; k < 9; ++k) q[(size_t)k * Vp + s] = make_double2(u.e[k / 3][k % 3].re, u.e[k / 3][k % 3].im);
    }
};

template <>
struct Store<P32> {
    using T = float;
    static constexpr int reals = 18;
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, mat3<float>& u) {
        s = checked_site(s, Vp);
        const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            float4 v = __ldg(q + (size_t)g * Vp + s);
            u.e[(2 * g) / 3][(2 * g) % 3] = {v.x, v.y};
            u.e[(2 * g + 1) / 3][(2 * g + 1) % 3] = {v.z, v.w};
        }
        float2 w = __ldg(reinterpret_cast<const float2*>(base + (size_t)16 * Vp) + s);
        u.e[2][2] = {w.x, w.y};
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const mat3<float>& u) {
        s = checked_site(s, Vp);
        float4* q = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int g = 0; g < 4; ++g)
            q[(size_t)g * Vp + s] = make_float4(u.e[(2 * g) / 3][(2 * g) % 3].re, u.e[(2 * g) / 3][(2 * g) % 3].im,
                                                u.e[(2 * g + 1) / 3][(2 * g + 1) % 3].re,
                                                u.e[(2 * g + 1) / 3][(2 * g + 1) % 3].im);
        reinterpret_cast<float2*>(base + (size_t)16 * Vp)[s] = make_float2(u.e[2][2].re, u.e[2][2].im);
    }
};

template <>
struct Store<P32R12> {
    using T = float;
    static constexpr int reals = 12;
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, mat3<float>& u) {
        s = checked_site(s, Vp);
        const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int g = 0; g < 3; ++g) {
            float4 v = __ldg(q + (size_t)g * Vp + s);
            u.e[(2 * g) / 3][(2 * g) % 3] = {v.x, v.y};
            u.e[(2 * g + 1) / 3][(2 * g + 1) % 3] = {v.z, v.w};
        }
        rebuild_row2(u);
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const mat3<float>& u) {
        s = checked_site(s, Vp);
        float4* q = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int g = 0; g < 3; ++g)
            q[(size_t)g * Vp + s] = make_float4(u.e[(2 * g) / 3][(2 * g) % 3].re, u.e[(2 * g) / 3][(2 * g) % 3].im,
                                                u.e[(2 * g + 1) / 3][(2 * g + 1) % 3].re,
                                                u.e[(2 * g + 1) / 3][(2 * g + 1) % 3].im);
    }
};

// accumulator X: 8 reals per link as two (FP32: float4) or four (FP64: double2) planes
template <class T>
struct AccStore;

template <>
struct AccStore<double> {
    static __device__ __forceinline__ void load(const double* __restrict__ base, int Vp, int s, alg8<double>& x) {
        s = checked_site(s, Vp);
        const double2* q = reinterpret_cast<const double2*>(base);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            double2 v = q[(size_t)g * Vp + s];
            x.v[2 * g] = v.x;
            x.v[2 * g + 1] = v.y;
        }
    }
    static __device__ __forceinline__ void store(double* __restrict__ base, int Vp, int s, const alg8<double>& x) {
        s = checked_site(s, Vp);
        double2* q = reinterpret_cast<double2*>(base);
#pragma unroll
        for (int g = 0; g < 4; ++g) q[(size_t)g * Vp + s] = make_double2(x.v[2 * g], x.v[2 * g + 1]);
    }
};

template <>
struct AccStore<float> {
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, alg8<float>& x) {
        s = checked_site(s, Vp);
        const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float4 v = q[(size_t)g * Vp + s];
            x.v[4 * g] = v.x;
            x.v[4 * g + 1] = v.y;
            x.v[4 * g + 2] = v.z;
            x.v[4 * g + 3] = v.w;
        }
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const alg8<float>& x) {
        s = checked_site(s, Vp);
        float4* q = reinterpret_cast<float4*>(base);
#pragma unroll
        for (int g = 0; g < 2; ++g)
            q[(size_t)g * Vp + s] = make_float4(x.v[4 * g], x.v[4 * g + 1], x.v[4 * g + 2], x.v[4 * g + 3]);
    }
};

// ---------------------------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------------------------

// Record a failure message for tgf_last_error() and return `st` (host, printf-style).
int set_error(int st, const char* fmt, ...);

// mode: 0 = RK3 stage only; 1 = stage and clover halves of the input field; 2 = halves only
// grid > 0 launches that many blocks (a grid-stride loop covers B.nblk tiles); 0 = one block per tile
void launch_stage(int prec, int stage, int mode, int reunit, const Batch& B, const void* w_in, void* w_out,
                  void* acc, void* clov, cudaStream_t st, int grid = 0);
void launch_clover_sum(int prec, unsigned flags, const Batch& B, const void* clov, double* partial,
                       cudaStream_t st);
void launch_reduce(const Batch& B, const double* partial, double* obs, cudaStream_t st);
// per-slab sums of the charge density along `dir`; the batch has L[dir] blocks per configuration
void launch_slice_charge(int prec, unsigned flags, const Batch& B, const void* clov, int dir, double* q, int q_stride,
                         cudaStream_t st);
void launch_pack(int prec, const Batch& B, const double* canon, void* w, cudaStream_t st);
// SU(N) forms (N = 2, 3, 4; FP64): one RK3 stage (batch of 32-site blocks), the measurement
// (measure batch of 128-site blocks with o_off / h set; partial holds 4 doubles per block), and
// canonical <-> storage layout (batch of 128-site blocks, m_off = canonical offset in doubles)
void launch_sun_stage(int N, int stage, const Batch& B, const double* w_in, double* w_out, double* acc,
                      cudaStream_t st);
void launch_sun_measure(int N, const Batch& Bm, const Batch& Br, const double* w, double* partial, double* obs,
                        int traceless, cudaStream_t st);
void launch_sun_layout(int N, bool to_storage, const Batch& B, double* canon, double* w, cudaStream_t st);
// one checkerboard pass of the Monte Carlo update (FP64 storage): links of direction mu on the
// sites of the given parity; heat-bath (overrelax = 0) or over-relaxation; the batch has
// ceil(V / 256) blocks of 128 threads per configuration
void launch_mc(int overrelax, const Batch& B, double* w, int mu, int parity, double beta, uint64_t seed,
               uint64_t sweep, cudaStream_t st);
void launch_unpack(int prec, const Batch& B, const void* w, double* canon, cudaStream_t st);

constexpr int kMeasureSites = 128;  // sites (threads) per block of the measurement kernel
constexpr int kPartials = 4;        // doubles per block partial: E, q, p, pad
// clover scratch per site: 6 planes x 2 halves x 9 reals (anti-Hermitian parts) + 6 plaquette traces
constexpr int kClovReals = 6 * 2 * 9 + 6;

}  // namespace tgf
