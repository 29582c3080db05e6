// api.cu -- the C ABI of libtgf (declared in include/tgf.h): argument checks, batch
// descriptors, and the flow driver that sequences the stage / measure / reduce kernels
// and captures a whole flow into one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <list>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/tgf.h"
#include "lattice.cuh"

using namespace tgf;

namespace {

thread_local std::string g_err;

// NVTX range over one ABI call (visible in Nsight Systems / Compute timelines; no cost without a tool)
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

tgf_status fail(tgf_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

}  // namespace

int tgf::set_error(int st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

namespace {

#define TGF_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return fail(TGF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

int reals_of(int prec) { return prec == TGF_FP32_R12 ? 12 : 18; }
size_t real_size(int prec) { return prec == TGF_FP64 ? 8 : 4; }

int64_t padded(int64_t V) { return (V + kSiteAlign - 1) / kSiteAlign * kSiteAlign; }

int64_t sites(const tgf_lattice& l) { return (int64_t)l.L[0] * l.L[1] * l.L[2] * l.L[3]; }

tgf_status check_prec(int prec) {
    if (prec != TGF_FP64 && prec != TGF_FP32 && prec != TGF_FP32_R12)
        return fail(TGF_EINVAL, "unknown precision %d", prec);
    return TGF_OK;
}

// Extents, size limits and the box of the paper (Sec. 3.1): L = (l, l, N l, N l) with the twisted
// plane first, unless the configuration sets TGF_ANY_EXTENTS.
tgf_status check_lat(const tgf_lattice* lat, int ncfg, int N = 3) {
    if (!lat) return fail(TGF_EINVAL, "lattice array is NULL");
    if (ncfg < 1 || ncfg > TGF_MAX_CFG) return fail(TGF_EINVAL, "ncfg = %d outside 1..%d", ncfg, TGF_MAX_CFG);
    for (int c = 0; c < ncfg; ++c) {
        const int* L = lat[c].L;
        for (int mu = 0; mu < 4; ++mu)
            if (L[mu] < 2 || L[mu] > 4096)
                return fail(TGF_EINVAL, "configuration %d: extent L[%d] = %d outside 2..4096", c, mu, L[mu]);
        if (sites(lat[c]) > (int64_t(1) << 28))
            return fail(TGF_EINVAL, "configuration %d: %lld sites exceed 2^28", c, (long long)sites(lat[c]));
        if (lat[c].flags & ~TGF_ANY_EXTENTS)
            return fail(TGF_EINVAL, "configuration %d: unknown lattice flags 0x%x", c, lat[c].flags);
        if (!(lat[c].flags & TGF_ANY_EXTENTS) && (L[1] != L[0] || L[2] != N * L[0] || L[3] != N * L[0]))
            return fail(TGF_EINVAL,
                        "configuration %d: extents %dx%dx%dx%d are not the twisted box l x l x %dl x %dl "
                        "(set TGF_ANY_EXTENTS in the lattice's flags to allow other extents)",
                        c, L[0], L[1], L[2], L[3], N, N);
    }
    return TGF_OK;
}

// ---- host-side fault injection (TGF_FAULT) ---------------------------------------------------
// TGF_FAULT=alloc: tgf_create fails as if cudaMalloc had (TGF_ENOMEM), allocating nothing;
// TGF_FAULT=nan: tgf_upload and tgf_set_links plant a NaN in the first real of the first
// configuration they copy (in the device staging copy; the caller's buffer is untouched);
// TGF_FAULT=badarg: the argument checks of the hot-path calls fail (TGF_EINVAL).
// Read at every call, so a test can set and clear it in-process.  Nothing faults on the GPU.
bool fault_is(const char* what) {
    const char* v = std::getenv("TGF_FAULT");
    return v && std::strcmp(v, what) == 0;
}

// TGF_EKERNEL if a record written since the last read on this device came out non-finite
// (synchronises `st`); `stride` decodes the slot into configuration and record.
tgf_status check_nonfinite(cudaStream_t st, size_t stride, const char* call) {
    cudaError_t e = cudaSuccess;
    const unsigned long long v = nonfinite_read_and_clear(st, &e);
    if (e != cudaSuccess) return fail(TGF_ECUDA, "%s: reading the kernel status: %s", call, cudaGetErrorString(e));
    if (v) {
        const unsigned long long slot = v - 1, sd = stride ? stride : 1;
        return fail(TGF_EKERNEL, "%s: the record of configuration %llu, record %llu (observable slot %llu) is not finite "
                    "(non-finite links or an overflow)", call, slot / sd, slot % sd, slot);
    }
    return TGF_OK;
}

tgf_status injected_badarg(const char* call) {
    if (fault_is("badarg")) return fail(TGF_EINVAL, "%s: argument check failed (fault injected by TGF_FAULT=badarg)", call);
    return TGF_OK;
}

// n_{mu nu} mod 3 table from the six upper entries
void twist_table(const tgf_lattice& l, int8_t tw[16]) {
    const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    std::memset(tw, 0, 16);
    for (int i = 0; i < 6; ++i) {
        int k = ((l.twist[i] % 3) + 3) % 3;
        int mu = pairs[i][0], nu = pairs[i][1];
        tw[mu * 4 + nu] = (int8_t)k;
        tw[nu * 4 + mu] = (int8_t)((3 - k) % 3);
    }
}

struct Layout {
    std::vector<int64_t> w_off, x_off, c_off, m_off;  // reals / reals / canonical doubles / reals
    std::vector<int64_t> meas_blk0;                   // first measure block of each config in a full launch
    int64_t w_total = 0, x_total = 0, m_total = 0, meas_blocks = 0;
    // scratch: [partials: meas_blocks x kPartials doubles][pad to 256 B][clover halves: m_total reals]
    size_t partial_bytes() const { return ((size_t)meas_blocks * kPartials * sizeof(double) + 255) / 256 * 256; }
    size_t scratch_bytes(int prec) const;
};

size_t Layout::scratch_bytes(int prec) const { return partial_bytes() + (size_t)m_total * real_size(prec); }

Layout layout(int prec, const tgf_lattice* lat, int ncfg) {
    Layout L;
    int64_t w = 0, x = 0, cc = 0, mb = 0, m = 0;
    for (int c = 0; c < ncfg; ++c) {
        int64_t V = sites(lat[c]), Vp = padded(V);
        L.w_off.push_back(w);
        L.x_off.push_back(x);
        L.c_off.push_back(cc);
        L.m_off.push_back(m);
        L.meas_blk0.push_back(mb);
        w += 4 * (int64_t)reals_of(prec) * Vp;
        x += 4 * 8 * Vp;
        cc += V * 72;
        m += (int64_t)kClovReals * Vp;
        mb += (V + kMeasureSites - 1) / kMeasureSites;
    }
    L.w_total = w;
    L.x_total = x;
    L.m_total = m;
    L.meas_blocks = mb;
    return L;
}

// Descriptor of a launch over the configurations `which`, `spb` sites per block.
Batch make_batch(const tgf_lattice* lat, const Layout& Ly, const std::vector<int>& which, int spb) {
    Batch B;
    B.ncfg = (int)which.size();
    int blk = 0;
    for (int i = 0; i < B.ncfg; ++i) {
        const int c = which[i];
        CfgDesc& d = B.c[i];
        set_geometry(d, lat[c].L);
        d.Vp = (int)padded(d.V);
        d.blk0 = blk;
        d.w_off = Ly.w_off[c];
        d.x_off = Ly.x_off[c];
        d.m_off = Ly.m_off[c];
        d.o_off = 0;
        d.h = 0.0;
        twist_table(lat[c], d.tw);
        blk += (d.V + spb - 1) / spb;
    }
    B.nblk = blk;
    return B;
}

std::vector<int> all_cfgs(int ncfg) {
    std::vector<int> v(ncfg);
    for (int i = 0; i < ncfg; ++i) v[i] = i;
    return v;
}

tgf_status last_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(TGF_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
    return TGF_OK;
}

void* clover_base(void* scratch, const Layout& Ly) { return (char*)scratch + Ly.partial_bytes(); }

// clover-sum + reduce over `which` (halves already written), record r_c at time t_c
tgf_status enqueue_sum(int prec, unsigned flags, const tgf_lattice* lat, const Layout& Ly,
                       const std::vector<int>& which, const std::vector<int>& rec, const std::vector<double>& t,
                       size_t obs_stride, double* scratch, tgf_obs* obs, cudaStream_t st) {
    Batch B = make_batch(lat, Ly, which, kMeasureSites);
    for (int i = 0; i < B.ncfg; ++i) {
        B.c[i].h = t[i];
        B.c[i].o_off = (int64_t)which[i] * (int64_t)obs_stride + rec[i];
    }
    launch_clover_sum(prec, flags, B, clover_base(scratch, Ly), scratch, st);
    tgf_status s = last_launch("clover sum");
    if (s) return s;
    launch_reduce(B, scratch, reinterpret_cast<double*>(obs), st);
    return last_launch("reduce");
}

// full measurement of `which` from the field w: clover halves, their sum, the reduction
tgf_status enqueue_measure(int prec, unsigned flags, const tgf_lattice* lat, const Layout& Ly,
                           const std::vector<int>& which, const std::vector<int>& rec, const std::vector<double>& t,
                           size_t obs_stride, const void* w, double* scratch, tgf_obs* obs, cudaStream_t st) {
    Batch B = make_batch(lat, Ly, which, 32);
    launch_stage(prec, 1, 2, 0, B, w, nullptr, nullptr, clover_base(scratch, Ly), st);
    tgf_status s = last_launch("clover halves");
    if (s) return s;
    return enqueue_sum(prec, flags, lat, Ly, which, rec, t, obs_stride, scratch, obs, st);
}

tgf_status check_ptr(const void* p, const char* name) {
    if (!p) return fail(TGF_EINVAL, "%s is NULL", name);
    if (reinterpret_cast<uintptr_t>(p) % 256 != 0) return fail(TGF_EINVAL, "%s is not 256-byte aligned", name);
    return TGF_OK;
}

void flow_counts(double eps, double t_end, int64_t& n, double& rest) {
    n = (int64_t)std::floor(t_end / eps + 1e-9);
    rest = t_end - (double)n * eps;
    if (rest <= 1e-12 * eps) rest = 0.0;
}

int64_t records_of(int64_t n, double rest, int measure_every) {
    int64_t total = n + (rest > 0 ? 1 : 0);
    return (total + measure_every - 1) / measure_every + 1;
}

// ---- graph cache ----------------------------------------------------------------------------

struct GraphEntry {
    std::string key;
    int device;
    cudaGraphExec_t exec;
};
std::mutex g_graph_mu;
std::list<GraphEntry> g_graphs;  // most recent first
constexpr size_t kGraphCache = 8;
cudaStream_t g_capture[64] = {};

// Side branch of a flow: the clover sum + reduction of a measured step (HBM-bound) runs on this
// stream while stages 2 and 3 (FP-pipe-bound) run on the main one; captured into the same graph
// as parallel nodes.  Every enqueue_flow call creates its own stream and events and releases them
// when it returns (CUDA releases them once the enqueued work is done), so flows enqueued at the
// same time from several host threads never share a fork or join event.
struct SideBranch {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    SideBranch() = default;
    SideBranch(const SideBranch&) = delete;
    SideBranch& operator=(const SideBranch&) = delete;
    ~SideBranch() {
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (s) cudaStreamDestroy(s);
    }
    tgf_status create() {
        TGF_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        TGF_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        TGF_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        return TGF_OK;
    }
};

}  // namespace

extern "C" {

const char* tgf_last_error(void) { return g_err.c_str(); }

const char* tgf_status_string(int status) {
    switch (status) {
        case TGF_OK: return "ok";
        case TGF_EINVAL: return "invalid argument";
        case TGF_ENOMEM: return "out of device memory";
        case TGF_ECUDA: return "CUDA error";
        case TGF_EKERNEL: return "non-finite result";
        case TGF_ESTATE: return "no configuration kept";
        case TGF_EIO: return "checkpoint file error";
        default: return "unknown status";
    }
}

const char* tgf_version(void) { return "1.1.0"; }

tgf_status tgf_links_bytes(int prec, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    *bytes = (size_t)layout(prec, lat, ncfg).w_total * real_size(prec);
    return TGF_OK;
}

tgf_status tgf_accum_bytes(int prec, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    *bytes = (size_t)layout(prec, lat, ncfg).x_total * real_size(prec);
    return TGF_OK;
}

tgf_status tgf_scratch_bytes(int prec, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    *bytes = layout(prec, lat, ncfg).scratch_bytes(prec);
    return TGF_OK;
}

tgf_status tgf_canonical_bytes(const tgf_lattice* lat, size_t* bytes) {
    tgf_status s;
    if ((s = check_lat(lat, 1))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    *bytes = (size_t)sites(*lat) * 72 * sizeof(double);
    return TGF_OK;
}

tgf_status tgf_pack(int prec, const tgf_lattice* lat, int ncfg, const double* canon_dev, void* links, void* stream) {
    Range range_("tgf_pack");
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(canon_dev, "canon_dev")) ||
        (s = check_ptr(links, "links")))
        return s;
    Layout Ly = layout(prec, lat, ncfg);
    Batch B = make_batch(lat, Ly, all_cfgs(ncfg), 32);
    for (int i = 0; i < ncfg; ++i) B.c[i].x_off = Ly.c_off[i];
    launch_pack(prec, B, canon_dev, links, (cudaStream_t)stream);
    return last_launch("pack");
}

tgf_status tgf_unpack(int prec, const tgf_lattice* lat, int ncfg, const void* links, double* canon_dev, void* stream) {
    Range range_("tgf_unpack");
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(canon_dev, "canon_dev")) ||
        (s = check_ptr(links, "links")))
        return s;
    Layout Ly = layout(prec, lat, ncfg);
    Batch B = make_batch(lat, Ly, all_cfgs(ncfg), 32);
    for (int i = 0; i < ncfg; ++i) B.c[i].x_off = Ly.c_off[i];
    launch_unpack(prec, B, links, canon_dev, (cudaStream_t)stream);
    return last_launch("unpack");
}

static tgf_status check_staging(const tgf_lattice* lat, int ncfg, const double* staging, size_t staging_bytes) {
    tgf_status s;
    if ((s = check_ptr(staging, "staging_dev"))) return s;
    for (int c = 0; c < ncfg; ++c)
        if ((size_t)sites(lat[c]) * 72 * sizeof(double) > staging_bytes)
            return fail(TGF_EINVAL, "staging buffer of %zu bytes too small for configuration %d", staging_bytes, c);
    return TGF_OK;
}

tgf_status tgf_upload(int prec, const tgf_lattice* lat, int ncfg, const double* canon_host, double* staging_dev,
                      size_t staging_bytes, void* links, void* stream) {
    Range range_("tgf_upload");
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links")) ||
        (s = check_staging(lat, ncfg, staging_dev, staging_bytes)))
        return s;
    if (!canon_host) return fail(TGF_EINVAL, "canon_host is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    Layout Ly = layout(prec, lat, ncfg);
    static const double kNaN = std::numeric_limits<double>::quiet_NaN();
    const bool plant_nan = fault_is("nan");
    for (int c = 0; c < ncfg; ++c) {
        TGF_CUDA(cudaMemcpyAsync(staging_dev, canon_host + Ly.c_off[c], (size_t)sites(lat[c]) * 72 * sizeof(double),
                                 cudaMemcpyHostToDevice, st));
        if (plant_nan && c == 0)
            TGF_CUDA(cudaMemcpyAsync(staging_dev, &kNaN, sizeof kNaN, cudaMemcpyHostToDevice, st));
        Batch B = make_batch(lat, Ly, std::vector<int>{c}, 32);
        B.c[0].x_off = 0;
        launch_pack(prec, B, staging_dev, links, st);
        if ((s = last_launch("pack"))) return s;
    }
    return TGF_OK;
}

tgf_status tgf_download(int prec, const tgf_lattice* lat, int ncfg, const void* links, double* staging_dev,
                        size_t staging_bytes, double* canon_host, void* stream) {
    Range range_("tgf_download");
    tgf_status s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links")) ||
        (s = check_staging(lat, ncfg, staging_dev, staging_bytes)))
        return s;
    if (!canon_host) return fail(TGF_EINVAL, "canon_host is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    Layout Ly = layout(prec, lat, ncfg);
    for (int c = 0; c < ncfg; ++c) {
        Batch B = make_batch(lat, Ly, std::vector<int>{c}, 32);
        B.c[0].x_off = 0;
        launch_unpack(prec, B, links, staging_dev, st);
        if ((s = last_launch("unpack"))) return s;
        TGF_CUDA(cudaMemcpyAsync(canon_host + Ly.c_off[c], staging_dev, (size_t)sites(lat[c]) * 72 * sizeof(double),
                                 cudaMemcpyDeviceToHost, st));
        TGF_CUDA(cudaStreamSynchronize(st));
    }
    return TGF_OK;
}

tgf_status tgf_stage(int prec, const tgf_lattice* lat, int ncfg, const void* w_in, void* w_out, void* accum, int stage,
                     double eps, int reunit, unsigned flags, void* stream) {
    Range range_("tgf_stage");
    tgf_status s;
    if ((s = injected_badarg("tgf_stage"))) return s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(w_in, "w_in")) ||
        (s = check_ptr(w_out, "w_out")) || (s = check_ptr(accum, "accum")))
        return s;
    if (stage < 1 || stage > 3) return fail(TGF_EINVAL, "stage %d outside 1..3", stage);
    if (!(std::isfinite(eps)) || eps == 0.0) return fail(TGF_EINVAL, "eps = %g must be finite and non-zero", eps);
    if (w_in == w_out) return fail(TGF_EINVAL, "w_in and w_out must be distinct buffers");
    if (flags & ~(0x7u << 13)) return fail(TGF_EINVAL, "tgf_stage: unknown flags 0x%x (only TGF_TUNE_TILE)", flags);
    const int tile = prec == TGF_FP64 ? 0 : (int)((flags >> 13) & 0x7u);
    if (tile >= kTiles) return fail(TGF_EINVAL, "tgf_stage: launch tile %d outside 0..%d", tile, kTiles - 1);
    Layout Ly = layout(prec, lat, ncfg);
    Batch B = make_batch(lat, Ly, all_cfgs(ncfg), tile_sites(tile));
    for (int i = 0; i < ncfg; ++i) B.c[i].h = eps;
    launch_stage(prec, stage, 0, reunit, B, w_in, w_out, accum, nullptr, (cudaStream_t)stream, 0, tile);
    return last_launch("stage");
}

tgf_status tgf_measure(int prec, const tgf_lattice* lat, int ncfg, const void* links, double* scratch,
                       size_t scratch_bytes, tgf_obs* obs_dev, size_t obs_stride, int rec, double t, unsigned flags,
                       void* stream) {
    Range range_("tgf_measure");
    tgf_status s;
    if ((s = injected_badarg("tgf_measure"))) return s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links")) ||
        (s = check_ptr(scratch, "scratch")) || (s = check_ptr(obs_dev, "obs_dev")))
        return s;
    Layout Ly = layout(prec, lat, ncfg);
    if (scratch_bytes < Ly.scratch_bytes(prec))
        return fail(TGF_EINVAL, "scratch of %zu bytes too small (need %zu)", scratch_bytes, Ly.scratch_bytes(prec));
    if (rec < 0 || (ncfg > 1 && (size_t)rec >= obs_stride))
        return fail(TGF_EINVAL, "record %d outside the stride %zu", rec, obs_stride);
    if (flags & ~(TGF_CLOVER_TRACELESS | TGF_SYNC)) return fail(TGF_EINVAL, "tgf_measure: unknown flags 0x%x", flags);
    std::vector<int> which = all_cfgs(ncfg), recs(ncfg, rec);
    std::vector<double> ts(ncfg, t);
    if ((s = enqueue_measure(prec, flags, lat, Ly, which, recs, ts, obs_stride, links, scratch, obs_dev,
                             (cudaStream_t)stream)))
        return s;
    if (flags & TGF_SYNC) return check_nonfinite((cudaStream_t)stream, obs_stride, "tgf_measure");
    return TGF_OK;
}

tgf_status tgf_kernel_status(void* stream) {
    Range range_("tgf_kernel_status");
    return check_nonfinite((cudaStream_t)stream, 0, "tgf_kernel_status");
}

// ---- self-checking builds ------------------------------------------------------------------

tgf_status tgf_check_errors(unsigned* bits) {
    if (!bits) return fail(TGF_EINVAL, "bits is NULL");
#ifdef TGF_CHECK
    TGF_CUDA(cudaDeviceSynchronize());
    const unsigned w[6] = {check_word_stage(), check_word_measure(), check_word_pack(), check_word_mc(),
                           check_word_sun(), check_word_stage_tiles()};
    unsigned b = 0;
    for (int i = 0; i < 6; ++i)
        if (w[i]) b |= 1u << i;
    *bits = b;
    return TGF_OK;
#else
    *bits = 0;
    return fail(TGF_EINVAL, "not a self-checking build (compile the library with -DTGF_CHECK)");
#endif
}

// ---- checkpoints ---------------------------------------------------------------------------

namespace {

// CRC-32 of IEEE 802.3 (reflected polynomial 0xEDB88320, initial value and final xor 0xFFFFFFFF)
uint32_t crc32_update(uint32_t crc, const unsigned char* p, size_t n) {
    static uint32_t table[256];
    static std::once_flag once;
    std::call_once(once, [] {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : c >> 1;
            table[i] = c;
        }
    });
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xFFu] ^ (crc >> 8);
    return crc;
}

constexpr char kMagic[8] = {'T', 'G', 'F', 'C', 'K', 'P', 'T', '1'};

struct CkptHeader {
    char magic[8];
    uint32_t version;
    uint32_t ncfg;
    int32_t precision;
    int32_t reserved;
    double t;
    int64_t step;
    uint64_t seed;
};
static_assert(sizeof(CkptHeader) == 48, "checkpoint header layout");

struct CkptLattice {
    int32_t L[4];
    int32_t twist[6];
};

}  // namespace

uint32_t tgf_crc32(const void* data, size_t n) {
    return crc32_update(0xFFFFFFFFu, static_cast<const unsigned char*>(data), n) ^ 0xFFFFFFFFu;
}

tgf_status tgf_save(const char* path, int prec, const tgf_lattice* lat, int ncfg, const void* links, double* staging_dev,
                    size_t staging_bytes, double t, long long step, unsigned long long seed, void* stream) {
    Range range_("tgf_save");
    tgf_status s;
    if (!path) return fail(TGF_EINVAL, "path is NULL");
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links"))) return s;
    size_t total = 0;
    for (int c = 0; c < ncfg; ++c) total += (size_t)sites(lat[c]) * 72;
    std::vector<double> canon(total);
    if ((s = tgf_download(prec, lat, ncfg, links, staging_dev, staging_bytes, canon.data(), stream))) return s;
    CkptHeader h{};
    std::memcpy(h.magic, kMagic, 8);
    h.version = 1;
    h.ncfg = (uint32_t)ncfg;
    h.precision = prec;
    h.t = t;
    h.step = (int64_t)step;
    h.seed = (uint64_t)seed;
    std::vector<CkptLattice> lt(ncfg);
    for (int c = 0; c < ncfg; ++c) {
        for (int m = 0; m < 4; ++m) lt[c].L[m] = lat[c].L[m];
        for (int i = 0; i < 6; ++i) lt[c].twist[i] = lat[c].twist[i];
    }
    uint32_t crc = 0xFFFFFFFFu;
    crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(&h), sizeof h);
    crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(lt.data()), lt.size() * sizeof(CkptLattice));
    crc = crc32_update(crc, reinterpret_cast<const unsigned char*>(canon.data()), canon.size() * sizeof(double));
    crc ^= 0xFFFFFFFFu;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(TGF_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 &&
              std::fwrite(lt.data(), sizeof(CkptLattice), lt.size(), f) == lt.size() &&
              std::fwrite(canon.data(), sizeof(double), canon.size(), f) == canon.size() &&
              std::fwrite(&crc, sizeof crc, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(TGF_EIO, "write to %s failed", path);
    return TGF_OK;
}

tgf_status tgf_load(const char* path, int prec, const tgf_lattice* lat, int ncfg, void* links, double* staging_dev,
                    size_t staging_bytes, double* t, long long* step, unsigned long long* seed, void* stream) {
    Range range_("tgf_load");
    tgf_status s;
    if (!path) return fail(TGF_EINVAL, "path is NULL");
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links"))) return s;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(TGF_EIO, "cannot open %s", path);
    std::vector<unsigned char> buf;
    unsigned char chunk[1 << 16];
    size_t n;
    while ((n = std::fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + n);
    std::fclose(f);
    if (buf.size() < sizeof(CkptHeader) + sizeof(uint32_t)) return fail(TGF_EIO, "%s: too short for a checkpoint", path);
    CkptHeader h;
    std::memcpy(&h, buf.data(), sizeof h);
    if (std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 1) return fail(TGF_EIO, "%s: not a libtgf checkpoint", path);
    uint32_t stored;
    std::memcpy(&stored, buf.data() + buf.size() - sizeof stored, sizeof stored);
    if (tgf_crc32(buf.data(), buf.size() - sizeof stored) != stored) return fail(TGF_EIO, "%s: CRC mismatch", path);
    if ((int)h.ncfg != ncfg) return fail(TGF_EINVAL, "%s holds %u configurations, the call %d", path, h.ncfg, ncfg);
    const unsigned char* p = buf.data() + sizeof h;
    size_t total = 0;
    for (int c = 0; c < ncfg; ++c) {
        CkptLattice l;
        std::memcpy(&l, p + c * sizeof l, sizeof l);
        for (int m = 0; m < 4; ++m)
            if (l.L[m] != lat[c].L[m])
                return fail(TGF_EINVAL, "%s: configuration %d has L[%d] = %d, the call %d", path, c, m, l.L[m],
                            lat[c].L[m]);
        for (int i = 0; i < 6; ++i)
            if (((l.twist[i] - lat[c].twist[i]) % 3 + 3) % 3 != 0)
                return fail(TGF_EINVAL, "%s: configuration %d has another twist", path, c);
        total += (size_t)sites(lat[c]) * 72;
    }
    const size_t data_off = sizeof h + (size_t)ncfg * sizeof(CkptLattice);
    if (buf.size() != data_off + total * sizeof(double) + sizeof(uint32_t))
        return fail(TGF_EIO, "%s: size does not match its lattices", path);
    std::vector<double> canon(total);
    std::memcpy(canon.data(), buf.data() + data_off, total * sizeof(double));
    if ((s = tgf_upload(prec, lat, ncfg, canon.data(), staging_dev, staging_bytes, links, stream))) return s;
    TGF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (t) *t = h.t;
    if (step) *step = (long long)h.step;
    if (seed) *seed = (unsigned long long)h.seed;
    return TGF_OK;
}

// ---- SU(N) forms (FP64) -------------------------------------------------------------------

namespace {

constexpr int kSunMeasureSites = 128;

tgf_status check_n(int N) {
    if (N < 2 || N > 4) return fail(TGF_EINVAL, "N = %d outside the supported 2..4", N);
    return TGF_OK;
}

// per-configuration offsets in doubles: links (4 N^2 complex planes of Vp), X (4 N^2 reals of Vp),
// canonical (V x 4 x N^2 complex); blocks of `spb` sites
Batch make_sun_batch(int N, const tgf_lattice* lat, int ncfg, int spb) {
    Batch B;
    B.ncfg = ncfg;
    int blk = 0;
    int64_t w = 0, x = 0, cc = 0;
    for (int c = 0; c < ncfg; ++c) {
        CfgDesc& d = B.c[c];
        set_geometry(d, lat[c].L);
        d.Vp = (int)padded(d.V);
        d.blk0 = blk;
        d.w_off = w;
        d.x_off = x;
        d.m_off = cc;
        d.o_off = 0;
        d.h = 0.0;
        const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
        std::memset(d.tw, 0, 16);
        for (int i = 0; i < 6; ++i) {
            const int k = ((lat[c].twist[i] % N) + N) % N;
            d.tw[pairs[i][0] * 4 + pairs[i][1]] = (int8_t)k;
            d.tw[pairs[i][1] * 4 + pairs[i][0]] = (int8_t)((N - k) % N);
        }
        w += (int64_t)4 * N * N * 2 * d.Vp;
        x += (int64_t)4 * N * N * d.Vp;
        cc += (int64_t)d.V * 4 * N * N * 2;
        blk += (d.V + spb - 1) / spb;
    }
    B.nblk = blk;
    return B;
}

size_t sun_scratch(const tgf_lattice* lat, int ncfg) {
    size_t nb = 0;
    for (int c = 0; c < ncfg; ++c) nb += (size_t)((sites(lat[c]) + kSunMeasureSites - 1) / kSunMeasureSites);
    return (nb * 4 * sizeof(double) + 255) / 256 * 256;
}

}  // namespace

tgf_status tgf_sun_links_bytes(int N, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    size_t b = 0;
    for (int c = 0; c < ncfg; ++c) b += (size_t)4 * N * N * 16 * (size_t)padded(sites(lat[c]));
    *bytes = b;
    return TGF_OK;
}

tgf_status tgf_sun_accum_bytes(int N, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    size_t b = 0;
    for (int c = 0; c < ncfg; ++c) b += (size_t)4 * N * N * 8 * (size_t)padded(sites(lat[c]));
    *bytes = b;
    return TGF_OK;
}

tgf_status tgf_sun_scratch_bytes(int N, const tgf_lattice* lat, int ncfg, size_t* bytes) {
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N))) return s;
    if (!bytes) return fail(TGF_EINVAL, "bytes is NULL");
    *bytes = sun_scratch(lat, ncfg);
    return TGF_OK;
}

tgf_status tgf_sun_pack(int N, const tgf_lattice* lat, int ncfg, const double* canon_dev, void* links, void* stream) {
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N)) || (s = check_ptr(canon_dev, "canon_dev")) ||
        (s = check_ptr(links, "links")))
        return s;
    Batch B = make_sun_batch(N, lat, ncfg, 128);
    launch_sun_layout(N, true, B, const_cast<double*>(canon_dev), static_cast<double*>(links), (cudaStream_t)stream);
    return last_launch("SU(N) pack");
}

tgf_status tgf_sun_unpack(int N, const tgf_lattice* lat, int ncfg, const void* links, double* canon_dev, void* stream) {
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N)) || (s = check_ptr(canon_dev, "canon_dev")) ||
        (s = check_ptr(links, "links")))
        return s;
    Batch B = make_sun_batch(N, lat, ncfg, 128);
    launch_sun_layout(N, false, B, canon_dev, const_cast<double*>(static_cast<const double*>(links)),
                      (cudaStream_t)stream);
    return last_launch("SU(N) unpack");
}

tgf_status tgf_sun_stage(int N, const tgf_lattice* lat, int ncfg, const void* w_in, void* w_out, void* accum, int stage,
                         double eps, void* stream) {
    Range range_("tgf_sun_stage");
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N)) || (s = check_ptr(w_in, "w_in")) ||
        (s = check_ptr(w_out, "w_out")) || (s = check_ptr(accum, "accum")))
        return s;
    if (stage < 1 || stage > 3) return fail(TGF_EINVAL, "stage %d outside 1..3", stage);
    if (!(std::isfinite(eps)) || eps == 0.0) return fail(TGF_EINVAL, "eps = %g must be finite and non-zero", eps);
    if (w_in == w_out) return fail(TGF_EINVAL, "w_in and w_out must be distinct buffers");
    Batch B = make_sun_batch(N, lat, ncfg, 32);
    for (int i = 0; i < ncfg; ++i) B.c[i].h = eps;
    launch_sun_stage(N, stage, B, static_cast<const double*>(w_in), static_cast<double*>(w_out),
                     static_cast<double*>(accum), (cudaStream_t)stream);
    return last_launch("SU(N) stage");
}

tgf_status tgf_sun_measure(int N, const tgf_lattice* lat, int ncfg, const void* links, double* scratch,
                           size_t scratch_bytes, tgf_obs* obs_dev, size_t obs_stride, int rec, double t, unsigned flags,
                           void* stream) {
    Range range_("tgf_sun_measure");
    tgf_status s;
    if ((s = check_n(N)) || (s = check_lat(lat, ncfg, N)) || (s = check_ptr(links, "links")) ||
        (s = check_ptr(scratch, "scratch")) || (s = check_ptr(obs_dev, "obs_dev")))
        return s;
    if (scratch_bytes < sun_scratch(lat, ncfg))
        return fail(TGF_EINVAL, "scratch of %zu bytes too small (need %zu)", scratch_bytes, sun_scratch(lat, ncfg));
    if (rec < 0 || (ncfg > 1 && (size_t)rec >= obs_stride))
        return fail(TGF_EINVAL, "record %d outside the stride %zu", rec, obs_stride);
    Batch B = make_sun_batch(N, lat, ncfg, kSunMeasureSites);
    for (int i = 0; i < ncfg; ++i) {
        B.c[i].h = t;
        B.c[i].o_off = (int64_t)i * (int64_t)obs_stride + rec;
    }
    launch_sun_measure(N, B, B, static_cast<const double*>(links), scratch, reinterpret_cast<double*>(obs_dev),
                       (flags & TGF_CLOVER_TRACELESS) ? 1 : 0, (cudaStream_t)stream);
    return last_launch("SU(N) measure");
}

tgf_status tgf_mc_sweeps(int prec, const tgf_lattice* lat, int ncfg, void* links, double beta, int n_hybrid, int n_or,
                         unsigned long long seed, unsigned long long first_sweep, void* stream) {
    Range range_("tgf_mc_sweeps");
    tgf_status s;
    if ((s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links"))) return s;
    if (prec != TGF_FP64) return fail(TGF_EINVAL, "the Monte Carlo update needs TGF_FP64 storage (got precision %d)", prec);
    for (int c = 0; c < ncfg; ++c)
        for (int mu = 0; mu < 4; ++mu)
            if (lat[c].L[mu] % 2)
                return fail(TGF_EINVAL, "configuration %d: extent L[%d] = %d is odd (checkerboard update)", c, mu,
                            lat[c].L[mu]);
    if (!(std::isfinite(beta) && beta > 0.0)) return fail(TGF_EINVAL, "beta = %g must be finite and positive", beta);
    if (n_hybrid < 0 || n_or < 0) return fail(TGF_EINVAL, "n_hybrid = %d and n_or = %d must be >= 0", n_hybrid, n_or);
    Layout Ly = layout(prec, lat, ncfg);
    Batch B = make_batch(lat, Ly, all_cfgs(ncfg), 256);
    cudaStream_t st = (cudaStream_t)stream;
    for (int h = 0; h < n_hybrid; ++h) {
        for (int o = -1; o < n_or; ++o) {
            const int overrelax = o >= 0;
            for (int mu = 0; mu < 4; ++mu)
                for (int parity = 0; parity < 2; ++parity) {
                    launch_mc(overrelax, B, static_cast<double*>(links), mu, parity, beta, (uint64_t)seed,
                              (uint64_t)(first_sweep + (unsigned long long)h), st);
                    if ((s = last_launch(overrelax ? "over-relaxation" : "heat-bath"))) return s;
                }
        }
    }
    return TGF_OK;
}

tgf_status tgf_measure_slices(int prec, const tgf_lattice* lat, int ncfg, const void* links, double* scratch,
                              size_t scratch_bytes, int dir, double* q_dev, size_t q_stride, unsigned flags,
                              void* stream) {
    Range range_("tgf_measure_slices");
    tgf_status s;
    if ((s = injected_badarg("tgf_measure_slices"))) return s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(links, "links")) ||
        (s = check_ptr(scratch, "scratch")) || (s = check_ptr(q_dev, "q_dev")))
        return s;
    if (dir < 0 || dir > 3) return fail(TGF_EINVAL, "direction %d outside 0..3", dir);
    Layout Ly = layout(prec, lat, ncfg);
    if (scratch_bytes < Ly.scratch_bytes(prec))
        return fail(TGF_EINVAL, "scratch of %zu bytes too small (need %zu)", scratch_bytes, Ly.scratch_bytes(prec));
    for (int c = 0; c < ncfg; ++c)
        if ((size_t)lat[c].L[dir] > q_stride)
            return fail(TGF_EINVAL, "q_stride %zu < extent %d of configuration %d", q_stride, lat[c].L[dir], c);
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> which = all_cfgs(ncfg);
    Batch H = make_batch(lat, Ly, which, 32);
    launch_stage(prec, 1, 2, 0, H, links, nullptr, nullptr, clover_base(scratch, Ly), st);
    if ((s = last_launch("clover halves"))) return s;
    // one block per (configuration, slab)
    Batch Q = make_batch(lat, Ly, which, 1);
    int blk = 0;
    for (int c = 0; c < ncfg; ++c) {
        Q.c[c].blk0 = blk;
        Q.c[c].o_off = c;
        blk += lat[c].L[dir];
    }
    Q.nblk = blk;
    launch_slice_charge(prec, flags, Q, clover_base(scratch, Ly), dir, q_dev, (int)q_stride, st);
    return last_launch("slice charge");
}

tgf_status tgf_flow_records(double eps, double t_end, int measure_every, int* n_records) {
    if (!(eps > 0) || !std::isfinite(eps)) return fail(TGF_EINVAL, "eps = %g must be positive", eps);
    if (!(t_end >= 0) || !std::isfinite(t_end)) return fail(TGF_EINVAL, "t_end = %g must be >= 0", t_end);
    if (measure_every < 1) return fail(TGF_EINVAL, "measure_every = %d must be >= 1", measure_every);
    if (!n_records) return fail(TGF_EINVAL, "n_records is NULL");
    if (t_end / eps > 1e8) return fail(TGF_EINVAL, "t_end/eps = %g steps is too many", t_end / eps);
    int64_t n;
    double rest;
    flow_counts(eps, t_end, n, rest);
    *n_records = (int)records_of(n, rest, measure_every);
    return TGF_OK;
}

static tgf_status enqueue_flow(int prec, const tgf_lattice* lat, int ncfg, const Layout& Ly, void* w, void* w_tmp,
                               void* accum, double* scratch, double eps, const std::vector<int64_t>& n,
                               const std::vector<double>& rest, int measure_every, int reunit_every, unsigned flags,
                               tgf_obs* obs, size_t obs_cap, cudaStream_t st) {
    tgf_status s;
    std::vector<int64_t> total(ncfg);
    int64_t maxT = 0;
    for (int c = 0; c < ncfg; ++c) {
        total[c] = n[c] + (rest[c] > 0 ? 1 : 0);
        maxT = std::max(maxT, total[c]);
    }
    std::vector<int> rec(ncfg, 0);
    // tuning (flags): a persistent grid of k x SMs x resident blocks, configurations by size
    int grid = 0;
    if (const int k = (int)((flags >> 8) & 0xFu)) {
        int dev = 0, sms = 0;
        TGF_CUDA(cudaGetDevice(&dev));
        TGF_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const unsigned t = (flags >> 13) & 0x7u;  // resident blocks per SM of the tile
        grid = k * sms * (prec == TGF_FP64 ? 2 : t == 1 ? 2 : 4);
    }
    const bool by_size = (flags & TGF_TUNE_SIZE_ORDER) != 0;
    // launch tile of the FP32 forms' stage kernels (FP64 has one tile)
    const int tile = prec == TGF_FP64 ? 0 : (int)((flags >> 13) & 0x7u);
    if (tile >= kTiles) return fail(TGF_EINVAL, "tgf_flow: launch tile %d outside 0..%d", tile, kTiles - 1);
    void* cur = w;
    void* alt = w_tmp;
    SideBranch side;
    if ((s = side.create())) return s;
    SideBranch* sb = &side;
    bool pending = false;  // a side-branch sum still reads the clover halves / writes the partials
    auto join = [&]() -> tgf_status {
        if (pending) {
            TGF_CUDA(cudaStreamWaitEvent(st, sb->join, 0));
            pending = false;
        }
        return TGF_OK;
    };
    // configurations with nothing to integrate: one record at t = 0
    {
        std::vector<int> which, r;
        std::vector<double> t;
        for (int c = 0; c < ncfg; ++c)
            if (total[c] == 0) { which.push_back(c); r.push_back(rec[c]++); t.push_back(0.0); }
        if (!which.empty() &&
            (s = enqueue_measure(prec, flags, lat, Ly, which, r, t, obs_cap, cur, scratch, obs, st)))
            return s;
    }
    for (int64_t i = 0; i < maxT; ++i) {
        std::vector<int> act, mw, mr;
        std::vector<double> mt;
        for (int c = 0; c < ncfg; ++c) {
            if (i >= total[c]) continue;
            act.push_back(c);
            if (i % measure_every == 0) { mw.push_back(c); mr.push_back(rec[c]++); mt.push_back((double)i * eps); }
        }
        // every active configuration starts at step 0, so either all of them are measured now or none
        const int mode1 = mw.empty() ? 0 : 1;
        if (by_size)
            std::stable_sort(act.begin(), act.end(), [&](int a, int b) { return sites(lat[a]) > sites(lat[b]); });
        Batch B = make_batch(lat, Ly, act, tile_sites(tile));
        for (int k = 0; k < B.ncfg; ++k) {
            const int c = act[k];
            B.c[k].h = (i < n[c]) ? eps : rest[c];
        }
        const int ru = (prec != TGF_FP64 && reunit_every > 0 && (i + 1) % reunit_every == 0) ? 1 : 0;
        if (mode1 && (s = join())) return s;  // stage 1 is about to rewrite the halves
        launch_stage(prec, 1, mode1, 0, B, cur, alt, accum, clover_base(scratch, Ly), st, grid, tile);
        if ((s = last_launch("stage 1"))) return s;
        if (mode1) {
            TGF_CUDA(cudaEventRecord(sb->fork, st));
            TGF_CUDA(cudaStreamWaitEvent(sb->s, sb->fork, 0));
            if ((s = enqueue_sum(prec, flags, lat, Ly, mw, mr, mt, obs_cap, scratch, obs, sb->s))) return s;
            TGF_CUDA(cudaEventRecord(sb->join, sb->s));
            pending = true;
        }
        launch_stage(prec, 2, 0, 0, B, alt, cur, accum, nullptr, st, grid, tile);
        if ((s = last_launch("stage 2"))) return s;
        launch_stage(prec, 3, 0, ru, B, cur, alt, accum, nullptr, st, grid, tile);
        if ((s = last_launch("stage 3"))) return s;
        std::swap(cur, alt);
        std::vector<int> fw, fr;
        std::vector<double> ft;
        for (int c : act)
            if (total[c] == i + 1) { fw.push_back(c); fr.push_back(rec[c]++); ft.push_back((double)n[c] * eps + rest[c]); }
        if (!fw.empty()) {
            if ((s = join())) return s;
            if ((s = enqueue_measure(prec, flags, lat, Ly, fw, fr, ft, obs_cap, cur, scratch, obs, st))) return s;
        }
    }
    if ((s = join())) return s;
    // configurations that finished after an odd number of steps hold their field in w_tmp
    const size_t rs = real_size(prec);
    for (int c = 0; c < ncfg; ++c) {
        if (total[c] % 2 == 1) {
            const size_t off = (size_t)Ly.w_off[c] * rs;
            const size_t bytes = (size_t)4 * reals_of(prec) * padded(sites(lat[c])) * rs;
            TGF_CUDA(cudaMemcpyAsync((char*)w + off, (const char*)w_tmp + off, bytes, cudaMemcpyDeviceToDevice, st));
        }
    }
    return TGF_OK;
}

tgf_status tgf_flow(int prec, const tgf_lattice* lat, int ncfg, void* w, void* w_tmp, void* accum, double* scratch,
                    size_t scratch_bytes, double eps, const double* t_end, int measure_every, int reunit_every,
                    unsigned flags, tgf_obs* obs_dev, size_t obs_cap, int* n_records, void* stream) {
    Range range_("tgf_flow");
    tgf_status s;
    if ((s = injected_badarg("tgf_flow"))) return s;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg)) || (s = check_ptr(w, "w")) ||
        (s = check_ptr(w_tmp, "w_tmp")) || (s = check_ptr(accum, "accum")) || (s = check_ptr(scratch, "scratch")) ||
        (s = check_ptr(obs_dev, "obs_dev")))
        return s;
    if (w == w_tmp) return fail(TGF_EINVAL, "w and w_tmp must be distinct buffers");
    if (!t_end) return fail(TGF_EINVAL, "t_end is NULL");
    if (!n_records) return fail(TGF_EINVAL, "n_records is NULL");
    if (reunit_every < 0) return fail(TGF_EINVAL, "reunit_every = %d must be >= 0", reunit_every);
    Layout Ly = layout(prec, lat, ncfg);
    if (scratch_bytes < Ly.scratch_bytes(prec))
        return fail(TGF_EINVAL, "scratch of %zu bytes too small (need %zu)", scratch_bytes, Ly.scratch_bytes(prec));
    std::vector<int64_t> n(ncfg);
    std::vector<double> rest(ncfg);
    for (int c = 0; c < ncfg; ++c) {
        int nr;
        if ((s = tgf_flow_records(eps, t_end[c], measure_every, &nr))) return s;
        if ((size_t)nr > obs_cap) return fail(TGF_EINVAL, "configuration %d needs %d records, obs_cap = %zu", c, nr, obs_cap);
        flow_counts(eps, t_end[c], n[c], rest[c]);
        n_records[c] = nr;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const bool sync = (flags & TGF_SYNC) != 0;
    flags &= ~TGF_SYNC;
    if (flags & TGF_NO_GRAPH) {
        if ((s = enqueue_flow(prec, lat, ncfg, Ly, w, w_tmp, accum, scratch, eps, n, rest, measure_every, reunit_every,
                              flags, obs_dev, obs_cap, st)))
            return s;
        return sync ? check_nonfinite(st, obs_cap, "tgf_flow") : TGF_OK;
    }

    // ---- one CUDA graph per distinct call, cached -----------------------------------------
    int dev = 0;
    TGF_CUDA(cudaGetDevice(&dev));
    std::string key;
    auto put = [&key](const void* p, size_t b) { key.append((const char*)p, b); };
    put(&dev, sizeof dev); put(&prec, sizeof prec); put(&ncfg, sizeof ncfg);
    put(lat, sizeof(tgf_lattice) * ncfg);
    put(&w, sizeof w); put(&w_tmp, sizeof w_tmp); put(&accum, sizeof accum); put(&scratch, sizeof scratch);
    put(&eps, sizeof eps); put(t_end, sizeof(double) * ncfg);
    put(&measure_every, sizeof measure_every); put(&reunit_every, sizeof reunit_every); put(&flags, sizeof flags);
    put(&obs_dev, sizeof obs_dev); put(&obs_cap, sizeof obs_cap);

    std::lock_guard<std::mutex> lock(g_graph_mu);
    cudaGraphExec_t exec = nullptr;
    for (auto it = g_graphs.begin(); it != g_graphs.end(); ++it) {
        if (it->device == dev && it->key == key) {
            exec = it->exec;
            g_graphs.splice(g_graphs.begin(), g_graphs, it);
            break;
        }
    }
    if (!exec) {
        if (dev < 0 || dev >= 64) return fail(TGF_EINVAL, "device %d out of range", dev);
        if (!g_capture[dev]) TGF_CUDA(cudaStreamCreateWithFlags(&g_capture[dev], cudaStreamNonBlocking));
        cudaStream_t cs = g_capture[dev];
        TGF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        s = enqueue_flow(prec, lat, ncfg, Ly, w, w_tmp, accum, scratch, eps, n, rest, measure_every, reunit_every,
                         flags, obs_dev, obs_cap, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cs, &graph);
        if (s) {
            if (graph) cudaGraphDestroy(graph);
            return s;
        }
        if (ce != cudaSuccess) return fail(TGF_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(TGF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ce));
        g_graphs.push_front(GraphEntry{key, dev, exec});
        while (g_graphs.size() > kGraphCache) {
            cudaGraphExecDestroy(g_graphs.back().exec);
            g_graphs.pop_back();
        }
    }
    TGF_CUDA(cudaGraphLaunch(exec, st));
    return sync ? check_nonfinite(st, obs_cap, "tgf_flow") : TGF_OK;
}

}  // extern "C"

// ---- library-owned context (the stateful form of the calls above) -------------------------------

namespace {

// Makes `dev` current for the lifetime of the guard and restores the caller's device after.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

tgf_status alloc_dev(void** p, size_t bytes, const char* what) {
    const cudaError_t e = cudaMalloc(p, bytes < 256 ? 256 : bytes);
    if (e == cudaSuccess) return TGF_OK;
    *p = nullptr;
    cudaGetLastError();  // a failed cudaMalloc leaves its error as the thread's last error: clear it
    if (e == cudaErrorMemoryAllocation)
        return fail(TGF_ENOMEM, "tgf_create: cudaMalloc of %zu bytes for %s failed: out of device memory", bytes, what);
    return fail(TGF_ECUDA, "tgf_create: cudaMalloc of %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
}

}  // namespace

struct tgf_ctx {
    int device = 0, prec = 0, ncfg = 0, reunit_every = 0;
    unsigned flags = 0;
    std::vector<tgf_lattice> lat;
    void* links = nullptr;
    void* links_tmp = nullptr;
    void* accum = nullptr;
    void* scratch = nullptr;
    double* staging = nullptr;
    tgf_obs* obs = nullptr;
    size_t scratch_bytes = 0, staging_bytes = 0, obs_records = 0;
    ~tgf_ctx() {
        DeviceGuard g(device);
        for (void* p : {links, links_tmp, accum, scratch, (void*)staging, (void*)obs})
            if (p) cudaFree(p);
    }
};

namespace {

tgf_status check_ctx(const tgf_ctx* ctx, int cfg, const char* call) {
    if (!ctx) return fail(TGF_EINVAL, "%s: ctx is NULL", call);
    if (cfg < -1 || cfg >= ctx->ncfg) return fail(TGF_EINVAL, "%s: configuration %d outside 0..%d", call, cfg, ctx->ncfg - 1);
    return TGF_OK;
}

tgf_status check_guard(const DeviceGuard& g, int dev) {
    if (g.err != cudaSuccess) return fail(TGF_ECUDA, "cannot make device %d current: %s", dev, cudaGetErrorString(g.err));
    return TGF_OK;
}

// device records of at least n slots, grown on demand
tgf_status ctx_obs(tgf_ctx* ctx, size_t n) {
    if (ctx->obs_records >= n) return TGF_OK;
    if (ctx->obs) cudaFree(ctx->obs);
    ctx->obs = nullptr;
    ctx->obs_records = 0;
    tgf_status s = alloc_dev(reinterpret_cast<void**>(&ctx->obs), n * sizeof(tgf_obs), "the observable records");
    if (s) return s;
    ctx->obs_records = n;
    return TGF_OK;
}

}  // namespace

extern "C" {

tgf_status tgf_create(tgf_ctx** out, int device, int prec, int ncfg, const tgf_lattice* lat, int reunit_every,
                      unsigned flags) {
    Range range_("tgf_create");
    tgf_status s;
    if (!out) return fail(TGF_EINVAL, "tgf_create: out is NULL");
    *out = nullptr;
    if ((s = check_prec(prec)) || (s = check_lat(lat, ncfg))) return s;
    if (reunit_every < 0) return fail(TGF_EINVAL, "tgf_create: reunit_every = %d must be >= 0", reunit_every);
    if (flags & ~(TGF_CLOVER_TRACELESS | TGF_NO_GRAPH)) return fail(TGF_EINVAL, "tgf_create: unknown flags 0x%x", flags);
    if (fault_is("alloc"))
        return fail(TGF_ENOMEM, "tgf_create: device allocation failed (fault injected by TGF_FAULT=alloc)");
    int ndev = 0;
    TGF_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(TGF_EINVAL, "tgf_create: device %d outside 0..%d", device, ndev - 1);
    DeviceGuard g(device);
    if ((s = check_guard(g, device))) return s;
    std::unique_ptr<tgf_ctx> c(new tgf_ctx);
    c->device = device;
    c->prec = prec;
    c->ncfg = ncfg;
    c->reunit_every = reunit_every;
    c->flags = flags;
    c->lat.assign(lat, lat + ncfg);
    const Layout Ly = layout(prec, lat, ncfg);
    const size_t lb = (size_t)Ly.w_total * real_size(prec), ab = (size_t)Ly.x_total * real_size(prec);
    c->scratch_bytes = Ly.scratch_bytes(prec);
    for (int i = 0; i < ncfg; ++i) c->staging_bytes = std::max(c->staging_bytes, (size_t)sites(lat[i]) * 72 * sizeof(double));
    if ((s = alloc_dev(&c->links, lb, "the links")) || (s = alloc_dev(&c->links_tmp, lb, "the second link buffer")) ||
        (s = alloc_dev(&c->accum, ab, "the RK3 accumulator")) || (s = alloc_dev(&c->scratch, c->scratch_bytes, "the scratch")) ||
        (s = alloc_dev(reinterpret_cast<void**>(&c->staging), c->staging_bytes, "the staging buffer")) ||
        (s = ctx_obs(c.get(), (size_t)ncfg)))
        return s;
    TGF_CUDA(cudaMemset(c->links, 0, lb));
    *out = c.release();
    return TGF_OK;
}

void tgf_destroy(tgf_ctx* ctx) { delete ctx; }

tgf_status tgf_set_links(tgf_ctx* ctx, int cfg, const double* host_canon, size_t n_doubles) {
    Range range_("tgf_set_links");
    tgf_status s;
    if ((s = check_ctx(ctx, cfg, "tgf_set_links"))) return s;
    if (cfg < 0) return fail(TGF_EINVAL, "tgf_set_links: configuration %d outside 0..%d", cfg, ctx->ncfg - 1);
    if (!host_canon) return fail(TGF_EINVAL, "tgf_set_links: host_canon is NULL");
    const size_t need = (size_t)sites(ctx->lat[cfg]) * 72;
    if (n_doubles != need) return fail(TGF_EINVAL, "tgf_set_links: %zu doubles given, configuration %d has %zu", n_doubles, cfg, need);
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    static const double kNaN = std::numeric_limits<double>::quiet_NaN();
    TGF_CUDA(cudaMemcpy(ctx->staging, host_canon, need * sizeof(double), cudaMemcpyHostToDevice));
    if (fault_is("nan")) TGF_CUDA(cudaMemcpy(ctx->staging, &kNaN, sizeof kNaN, cudaMemcpyHostToDevice));
    const Layout Ly = layout(ctx->prec, ctx->lat.data(), ctx->ncfg);
    Batch B = make_batch(ctx->lat.data(), Ly, std::vector<int>{cfg}, 32);
    B.c[0].x_off = 0;
    launch_pack(ctx->prec, B, ctx->staging, ctx->links, nullptr);
    if ((s = last_launch("pack"))) return s;
    TGF_CUDA(cudaStreamSynchronize(nullptr));
    return TGF_OK;
}

tgf_status tgf_set_links_device(tgf_ctx* ctx, int cfg, const double* canon_dev, size_t n_doubles, void* stream) {
    Range range_("tgf_set_links_device");
    tgf_status s;
    if ((s = check_ctx(ctx, cfg, "tgf_set_links_device")) || (s = check_ptr(canon_dev, "canon_dev"))) return s;
    if (cfg < 0) return fail(TGF_EINVAL, "tgf_set_links_device: configuration %d outside 0..%d", cfg, ctx->ncfg - 1);
    const size_t need = (size_t)sites(ctx->lat[cfg]) * 72;
    if (n_doubles != need)
        return fail(TGF_EINVAL, "tgf_set_links_device: %zu doubles given, configuration %d has %zu", n_doubles, cfg, need);
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    const Layout Ly = layout(ctx->prec, ctx->lat.data(), ctx->ncfg);
    Batch B = make_batch(ctx->lat.data(), Ly, std::vector<int>{cfg}, 32);
    B.c[0].x_off = 0;
    launch_pack(ctx->prec, B, canon_dev, ctx->links, (cudaStream_t)stream);
    return last_launch("pack");
}

tgf_status tgf_get_links(tgf_ctx* ctx, int cfg, double* host_canon, size_t n_doubles) {
    Range range_("tgf_get_links");
    tgf_status s;
    if ((s = check_ctx(ctx, cfg, "tgf_get_links"))) return s;
    if (cfg < 0) return fail(TGF_EINVAL, "tgf_get_links: configuration %d outside 0..%d", cfg, ctx->ncfg - 1);
    if (!host_canon) return fail(TGF_EINVAL, "tgf_get_links: host_canon is NULL");
    const size_t need = (size_t)sites(ctx->lat[cfg]) * 72;
    if (n_doubles != need) return fail(TGF_EINVAL, "tgf_get_links: %zu doubles given, configuration %d has %zu", n_doubles, cfg, need);
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    const Layout Ly = layout(ctx->prec, ctx->lat.data(), ctx->ncfg);
    Batch B = make_batch(ctx->lat.data(), Ly, std::vector<int>{cfg}, 32);
    B.c[0].x_off = 0;
    launch_unpack(ctx->prec, B, ctx->links, ctx->staging, nullptr);
    if ((s = last_launch("unpack"))) return s;
    TGF_CUDA(cudaMemcpy(host_canon, ctx->staging, need * sizeof(double), cudaMemcpyDeviceToHost));
    return TGF_OK;
}

tgf_status tgf_ctx_measure(tgf_ctx* ctx, double t, tgf_obs* out, void* stream) {
    Range range_("tgf_ctx_measure");
    tgf_status s;
    if ((s = check_ctx(ctx, -1, "tgf_ctx_measure"))) return s;
    if (!out) return fail(TGF_EINVAL, "tgf_ctx_measure: out is NULL");
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    if ((s = tgf_measure(ctx->prec, ctx->lat.data(), ctx->ncfg, ctx->links, static_cast<double*>(ctx->scratch),
                         ctx->scratch_bytes, ctx->obs, 1, 0, t, (ctx->flags & TGF_CLOVER_TRACELESS) | TGF_SYNC, stream)))
        return s;
    TGF_CUDA(cudaMemcpyAsync(out, ctx->obs, (size_t)ctx->ncfg * sizeof(tgf_obs), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    TGF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TGF_OK;
}

tgf_status tgf_ctx_flow(tgf_ctx* ctx, double eps, const double* t_end, int measure_every, tgf_obs* out, size_t cap,
                        int* n_written, void* stream) {
    Range range_("tgf_ctx_flow");
    tgf_status s;
    if ((s = check_ctx(ctx, -1, "tgf_ctx_flow"))) return s;
    if (!out || !t_end || !n_written) return fail(TGF_EINVAL, "tgf_ctx_flow: out, t_end and n_written must not be NULL");
    if (cap < 1) return fail(TGF_EINVAL, "tgf_ctx_flow: cap = %zu must be >= 1", cap);
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    for (int c = 0; c < ctx->ncfg; ++c) {
        int nr = 0;
        if ((s = tgf_flow_records(eps, t_end[c], measure_every, &nr))) return s;
        if ((size_t)nr > cap) return fail(TGF_EINVAL, "tgf_ctx_flow: configuration %d needs %d records, cap = %zu", c, nr, cap);
    }
    if ((s = ctx_obs(ctx, (size_t)ctx->ncfg * cap))) return s;
    if ((s = tgf_flow(ctx->prec, ctx->lat.data(), ctx->ncfg, ctx->links, ctx->links_tmp, ctx->accum,
                      static_cast<double*>(ctx->scratch), ctx->scratch_bytes, eps, t_end, measure_every,
                      ctx->reunit_every, ctx->flags | TGF_SYNC, ctx->obs, cap, n_written, stream)))
        return s;
    TGF_CUDA(cudaMemcpyAsync(out, ctx->obs, (size_t)ctx->ncfg * cap * sizeof(tgf_obs), cudaMemcpyDeviceToHost,
                             (cudaStream_t)stream));
    TGF_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return TGF_OK;
}

tgf_status tgf_ctx_save(tgf_ctx* ctx, const char* path, double t, long long step, unsigned long long seed) {
    tgf_status s;
    if ((s = check_ctx(ctx, -1, "tgf_ctx_save"))) return s;
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    return tgf_save(path, ctx->prec, ctx->lat.data(), ctx->ncfg, ctx->links, ctx->staging, ctx->staging_bytes, t, step,
                    seed, nullptr);
}

tgf_status tgf_ctx_load(tgf_ctx* ctx, const char* path, double* t, long long* step, unsigned long long* seed) {
    tgf_status s;
    if ((s = check_ctx(ctx, -1, "tgf_ctx_load"))) return s;
    DeviceGuard g(ctx->device);
    if ((s = check_guard(g, ctx->device))) return s;
    return tgf_load(path, ctx->prec, ctx->lat.data(), ctx->ncfg, ctx->links, ctx->staging, ctx->staging_bytes, t, step,
                    seed, nullptr);
}

}  // extern "C"
