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
    int st[5];        // strides 1, L0, L0 L1, L0 L1 L2 and V (so st[d+1] - st[d] = (L_d - 1) st_d)
    int V;            // sites
    int Vp;           // padded plane length
    int blk0;         // first block of this configuration in the launch
    unsigned dmul[3]; // s / st[d+1] = umulhi(16 s, dmul[d]) >> dsh[d] for every site s < 2^28
    uint8_t dsh[4];
    int64_t w_off;    // link storage offset (reals)
    int64_t x_off;    // accumulator offset (reals)
    int64_t o_off;    // observable slot (records) = cfg * obs_stride + rec; slice charge: cfg index
    int64_t m_off;    // clover-halves offset in the scratch buffer (reals of the storage type)
    double h;         // step size (stages) or flow time t (measure)
    int8_t tw[16];    // n_{mu nu} mod 3 in {0,1,2}, row-major 4x4, antisymmetric mod 3
};
static_assert(sizeof(CfgDesc) == 120, "launch descriptor layout");

// Host: extents, strides and the division constants of a descriptor.  For a divisor d <= 2^28
// with l = ceil(log2 d) and m = ceil(2^(28+l) / d) < 2^29, floor(n/d) = floor(16 n m / 2^(32+l))
// for every n < 2^28: the error term n (m - 2^(28+l)/d) / 2^(28+l) stays below n / 2^28 < 1 in
// units of 1/d, so it never reaches the next multiple (Granlund and Montgomery, PLDI 1994, with
// the four spare bits of n taking the place of the 33rd bit of the multiplier).
inline void set_geometry(CfgDesc& d, const int L[4]) {
    for (int mu = 0; mu < 4; ++mu) d.L[mu] = L[mu];
    d.st[0] = 1;
    for (int mu = 1; mu <= 4; ++mu) d.st[mu] = d.st[mu - 1] * L[mu - 1];
    d.V = d.st[4];
    for (int k = 0; k < 3; ++k) {
        const uint64_t dv = (uint64_t)d.st[k + 1];
        int l = 0;
        while ((uint64_t(1) << l) < dv) ++l;
        d.dmul[k] = (unsigned)(((uint64_t(1) << (28 + l)) + dv - 1) / dv);
        d.dsh[k] = (uint8_t)l;
    }
    d.dsh[3] = 0;
}

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

// The four coordinates of site s: three independent multiply-shift divisions by the strides
// (constants from set_geometry) instead of a chain of integer divisions.
__device__ __forceinline__ void site_coords(const CfgDesc& c, int s, int (&x)[4]) {
    const unsigned u = (unsigned)s << 4;
    const int q1 = (int)(__umulhi(u, c.dmul[0]) >> c.dsh[0]);  // s / L0
    const int q2 = (int)(__umulhi(u, c.dmul[1]) >> c.dsh[1]);  // s / (L0 L1)
    const int q3 = (int)(__umulhi(u, c.dmul[2]) >> c.dsh[2]);  // s / (L0 L1 L2)
    x[0] = s - q1 * c.L[0];
    x[1] = q1 - q2 * c.L[1];
    x[2] = q2 - q3 * c.L[2];
    x[3] = q3;
}

// The four coordinates packed in 16-bit fields of one 64-bit register, so that a direction
// chosen at run time costs a shift, not a local-memory array access.
__device__ __forceinline__ uint64_t pack_coords(const CfgDesc& c, int s) {
    int x[4];
    site_coords(c, s, x);
    return (uint64_t)x[0] | ((uint64_t)x[1] << 16) | ((uint64_t)x[2] << 32) | ((uint64_t)x[3] << 48);
}
__device__ __forceinline__ int coord(uint64_t xp, int d) { return (int)((xp >> (16 * d)) & 0xFFFFu); }

// site index of n +- one step along a direction with coordinate x, extent L, stride st (periodic)
__device__ __forceinline__ int step_p(int s, int x, int L, int st) { return x == L - 1 ? s - (L - 1) * st : s + st; }
__device__ __forceinline__ int step_m(int s, int x, int L, int st) { return x == 0 ? s + (L - 1) * st : s - st; }

// Boundary flags of a site in one word: bit d  x_d == 0,  bit 4+d  x_d == L_d - 1,  bit 8+d
// x_d == 1.  With them a neighbour costs a bit test and a select for a direction chosen at run
// time; the wrap distance (L_d - 1) st_d is st[d+1] - st[d].
__device__ __forceinline__ unsigned edge_bits(const CfgDesc& c, const int (&x)[4]) {
    unsigned m = 0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        m |= (unsigned)(x[d] == 0) << d;
        m |= (unsigned)(x[d] == c.L[d] - 1) << (4 + d);
        m |= (unsigned)(x[d] == 1) << (8 + d);
    }
    return m;
}
__device__ __forceinline__ int fwd(const CfgDesc& c, unsigned m, int s, int d) {
    return ((m >> (4 + d)) & 1u) ? s - (c.st[d + 1] - c.st[d]) : s + c.st[d];
}
__device__ __forceinline__ int bwd(const CfgDesc& c, unsigned m, int s, int d) {
    return ((m >> d) & 1u) ? s + (c.st[d + 1] - c.st[d]) : s - c.st[d];
}

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
unsigned check_word_stage_tiles();
unsigned check_word_measure();
unsigned check_word_pack();
unsigned check_word_mc();
unsigned check_word_sun();

// ---------------------------------------------------------------------------------------------
// 32-byte vector access.  A warp moving one 32-byte element per lane touches 1 KB of contiguous
// memory in one instruction (ld/st .v8.f32 / .v4.f64 of sm_100+), so a link takes 3 loads in FP32
// (32 + 32 + 8 bytes) and 5 in FP64 instead of 5 and 9 with 16-byte vectors.  Addresses must be
// 32-byte aligned: every plane below starts at a multiple of 32 bytes (Vp is a multiple of 32
// sites and the caller's buffers are 256-byte aligned).  The .nc form reads through the
// non-coherent (read-only) path and is used only for data no thread of the kernel writes.
// ---------------------------------------------------------------------------------------------

__device__ __forceinline__ void ld8_nc(const float* p, float (&v)[8]) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}
__device__ __forceinline__ void ld8(const float* p, float (&v)[8]) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st8(float* p, const float (&v)[8]) {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]), "f"(v[2]),
                 "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
}
__device__ __forceinline__ void ld4d_nc(const double* p, double (&v)[4]) {
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
}
__device__ __forceinline__ void ld4d(const double* p, double (&v)[4]) {
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
                 : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                 : "l"(p)
                 : "memory");
}
__device__ __forceinline__ void st4d(double* p, const double (&v)[4]) {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
                 : "memory");
}

// ---------------------------------------------------------------------------------------------
// storage traits: load / store a link of direction mu at site s.  `base` points at the
// direction's planes (reals of the storage type); plane p of site s sits at
// base + p * (plane reals) * Vp + s * (plane reals).
//   FP64     (144 B/site): planes 0-3 hold entries (0,1), (2,3), (4,5), (6,7) as 4 doubles
//                          (32 B per site), plane 4 entry 8 (16 B per site)
//   FP32     ( 72 B/site): plane 0 entries 0-3, plane 1 entries 4-7 (8 floats, 32 B per site),
//                          plane 2 entry 8 (8 B per site)
//   FP32_R12 ( 48 B/site): plane 0 entries 0-3 (32 B per site), plane 1 entries 4-5 (16 B per
//                          site); row 2 = conj(row0 x row1) is rebuilt on every load
// (entries numbered row-major, each a complex (re, im)).
// ---------------------------------------------------------------------------------------------

template <int P>
struct Store;

template <>
struct Store<P64> {
    using T = double;
    static constexpr int reals = 18;
    static __device__ __forceinline__ void load(const double* __restrict__ base, int Vp, int s, mat3<double>& u) {
        s = checked_site(s, Vp);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            double v[4];
            ld4d_nc(base + (size_t)g * 4 * Vp + (size_t)s * 4, v);
            u.e[(2 * g) / 3][(2 * g) % 3] = {v[0], v[1]};
            u.e[(2 * g + 1) / 3][(2 * g + 1) % 3] = {v[2], v[3]};
        }
        const double2 w = __ldg(reinterpret_cast<const double2*>(base + (size_t)16 * Vp) + s);
        u.e[2][2] = {w.x, w.y};
    }
    static __device__ __forceinline__ void store(double* __restrict__ base, int Vp, int s, const mat3<double>& u) {
        s = checked_site(s, Vp);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const cx<double> a = u.e[(2 * g) / 3][(2 * g) % 3], b = u.e[(2 * g + 1) / 3][(2 * g + 1) % 3];
            const double v[4] = {a.re, a.im, b.re, b.im};
            st4d(base + (size_t)g * 4 * Vp + (size_t)s * 4, v);
        }
        reinterpret_cast<double2*>(base + (size_t)16 * Vp)[s] = make_double2(u.e[2][2].re, u.e[2][2].im);
    }
};

template <>
struct Store<P32> {
    using T = float;
    static constexpr int reals = 18;
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, mat3<float>& u) {
        s = checked_site(s, Vp);
        float a[8], b[8];
        ld8_nc(base + (size_t)s * 8, a);
        ld8_nc(base + (size_t)8 * Vp + (size_t)s * 8, b);
        const float2 w = __ldg(reinterpret_cast<const float2*>(base + (size_t)16 * Vp) + s);
        u.e[0][0] = {a[0], a[1]}; u.e[0][1] = {a[2], a[3]}; u.e[0][2] = {a[4], a[5]}; u.e[1][0] = {a[6], a[7]};
        u.e[1][1] = {b[0], b[1]}; u.e[1][2] = {b[2], b[3]}; u.e[2][0] = {b[4], b[5]}; u.e[2][1] = {b[6], b[7]};
        u.e[2][2] = {w.x, w.y};
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const mat3<float>& u) {
        s = checked_site(s, Vp);
        const float a[8] = {u.e[0][0].re, u.e[0][0].im, u.e[0][1].re, u.e[0][1].im,
                            u.e[0][2].re, u.e[0][2].im, u.e[1][0].re, u.e[1][0].im};
        const float b[8] = {u.e[1][1].re, u.e[1][1].im, u.e[1][2].re, u.e[1][2].im,
                            u.e[2][0].re, u.e[2][0].im, u.e[2][1].re, u.e[2][1].im};
        st8(base + (size_t)s * 8, a);
        st8(base + (size_t)8 * Vp + (size_t)s * 8, b);
        reinterpret_cast<float2*>(base + (size_t)16 * Vp)[s] = make_float2(u.e[2][2].re, u.e[2][2].im);
    }
};

template <>
struct Store<P32R12> {
    using T = float;
    static constexpr int reals = 12;
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, mat3<float>& u) {
        s = checked_site(s, Vp);
        float a[8];
        ld8_nc(base + (size_t)s * 8, a);
        const float4 b = __ldg(reinterpret_cast<const float4*>(base + (size_t)8 * Vp) + s);
        u.e[0][0] = {a[0], a[1]}; u.e[0][1] = {a[2], a[3]}; u.e[0][2] = {a[4], a[5]}; u.e[1][0] = {a[6], a[7]};
        u.e[1][1] = {b.x, b.y}; u.e[1][2] = {b.z, b.w};
        rebuild_row2(u);
    }
    // rows 0 and 1 only (row 2 of u left as it was)
    static __device__ __forceinline__ void load_top(const float* __restrict__ base, int Vp, int s, mat3<float>& u) {
        s = checked_site(s, Vp);
        float a[8];
        ld8_nc(base + (size_t)s * 8, a);
        const float4 b = __ldg(reinterpret_cast<const float4*>(base + (size_t)8 * Vp) + s);
        u.e[0][0] = {a[0], a[1]}; u.e[0][1] = {a[2], a[3]}; u.e[0][2] = {a[4], a[5]}; u.e[1][0] = {a[6], a[7]};
        u.e[1][1] = {b.x, b.y}; u.e[1][2] = {b.z, b.w};
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const mat3<float>& u) {
        s = checked_site(s, Vp);
        const float a[8] = {u.e[0][0].re, u.e[0][0].im, u.e[0][1].re, u.e[0][1].im,
                            u.e[0][2].re, u.e[0][2].im, u.e[1][0].re, u.e[1][0].im};
        st8(base + (size_t)s * 8, a);
        reinterpret_cast<float4*>(base + (size_t)8 * Vp)[s] =
            make_float4(u.e[1][1].re, u.e[1][1].im, u.e[1][2].re, u.e[1][2].im);
    }
};

// accumulator X: 8 reals per link -- FP32 one plane of 8 floats (32 B per site), FP64 two planes
// of 4 doubles.  Read and written by the same thread in one kernel: coherent loads.
template <class T>
struct AccStore;

template <>
struct AccStore<double> {
    static __device__ __forceinline__ void load(const double* __restrict__ base, int Vp, int s, alg8<double>& x) {
        s = checked_site(s, Vp);
        double a[4], b[4];
        ld4d(base + (size_t)s * 4, a);
        ld4d(base + (size_t)4 * Vp + (size_t)s * 4, b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x.v[k] = a[k];
            x.v[4 + k] = b[k];
        }
    }
    static __device__ __forceinline__ void store(double* __restrict__ base, int Vp, int s, const alg8<double>& x) {
        s = checked_site(s, Vp);
        const double a[4] = {x.v[0], x.v[1], x.v[2], x.v[3]}, b[4] = {x.v[4], x.v[5], x.v[6], x.v[7]};
        st4d(base + (size_t)s * 4, a);
        st4d(base + (size_t)4 * Vp + (size_t)s * 4, b);
    }
};

template <>
struct AccStore<float> {
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, alg8<float>& x) {
        s = checked_site(s, Vp);
        ld8(base + (size_t)s * 8, x.v);
    }
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const alg8<float>& x) {
        s = checked_site(s, Vp);
        st8(base + (size_t)s * 8, x.v);
    }
};

// The anti-Hermitian part D - D^+ of a 3x3 matrix as 9 reals {2 Im D_00, 2 Im D_11, 2 Im D_22,
// (D_01 - conj D_10) re/im, (D_02 - conj D_20) re/im, (D_12 - conj D_21) re/im} in the clover
// scratch: reals 0-7 as one 8-real vector per site (32 B in FP32, two 32-byte halves in FP64),
// real 8 in a plane of its own; a slot takes 9 Vp reals.
template <class T>
struct AhStore;

template <>
struct AhStore<float> {
    static __device__ __forceinline__ void store(float* __restrict__ base, int Vp, int s, const float (&v)[9]) {
        s = checked_site(s, Vp);
        const float a[8] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7]};
        st8(base + (size_t)s * 8, a);
        base[(size_t)8 * Vp + s] = v[8];
    }
    static __device__ __forceinline__ void load(const float* __restrict__ base, int Vp, int s, float (&v)[9]) {
        s = checked_site(s, Vp);
        float a[8];
        ld8_nc(base + (size_t)s * 8, a);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = a[k];
        v[8] = __ldg(base + (size_t)8 * Vp + s);
    }
};

template <>
struct AhStore<double> {
    static __device__ __forceinline__ void store(double* __restrict__ base, int Vp, int s, const double (&v)[9]) {
        s = checked_site(s, Vp);
        const double a[4] = {v[0], v[1], v[2], v[3]}, b[4] = {v[4], v[5], v[6], v[7]};
        st4d(base + (size_t)s * 8, a);
        st4d(base + (size_t)s * 8 + 4, b);
        base[(size_t)8 * Vp + s] = v[8];
    }
    static __device__ __forceinline__ void load(const double* __restrict__ base, int Vp, int s, double (&v)[9]) {
        s = checked_site(s, Vp);
        double a[4], b[4];
        ld4d_nc(base + (size_t)s * 8, a);
        ld4d_nc(base + (size_t)s * 8 + 4, b);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = a[k];
            v[4 + k] = b[k];
        }
        v[8] = __ldg(base + (size_t)8 * Vp + s);
    }
};

// ---------------------------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------------------------

// Record a failure message for tgf_last_error() and return `st` (host, printf-style).
int set_error(int st, const char* fmt, ...);

// mode: 0 = RK3 stage only; 1 = stage and clover halves of the input field; 2 = halves only
// grid > 0 launches that many blocks (a grid-stride loop covers B.nblk tiles); 0 = one block per tile
// tile: the launch tile of the FP32 forms (stage_kernel.cuh; 0 for FP64 and mode 2); the batch must
// have been built with tile_sites(tile) sites per block
void launch_stage(int prec, int stage, int mode, int reunit, const Batch& B, const void* w_in, void* w_out,
                  void* acc, void* clov, cudaStream_t st, int grid = 0, int tile = 0);
void launch_stage_tile(int tile, int prec, int stage, int mode, int reunit, const Batch& B, const void* w_in,
                       void* w_out, void* acc, void* clov, cudaStream_t st, int grid);
constexpr int kTiles = 5;
inline int tile_sites(int tile) { return tile == 1 ? 64 : 32; }
void launch_clover_sum(int prec, unsigned flags, const Batch& B, const void* clov, double* partial,
                       cudaStream_t st);
void launch_reduce(const Batch& B, const double* partial, double* obs, cudaStream_t st);
// Host: the first observable slot + 1 whose record came out non-finite since the last call (0 if
// none), read and cleared on `st` (synchronises `st`).
unsigned long long nonfinite_read_and_clear(cudaStream_t st, cudaError_t* err);
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
