// measure_static.cu -- tgf_measure_noalloc: the measurement of tgf_measure with its scratch in a
// fixed device array owned by the library, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where it may not call cudaMalloc -- a plug-in inside a host
// application whose own allocator owns all device memory and hands out only the input and
// output buffers, or a latency-critical loop that must not pay cudaMalloc's implicit device
// synchronisation.  Such a caller passes the links and the observable array only.
//
// The scratch (per-block partial sums and the clover halves, the same contents tgf_measure
// keeps in its caller-provided scratch) lives in g_static_scratch below: kStaticScratchBytes
// (36 MiB) of device memory that every GPU which loads the library holds until the process
// exits.  Every call writes all of the scratch it reads before reading it, so nothing has to be
// cleared between calls; calls whose kernels overlap on the GPU (different streams, no
// ordering) share the array and race.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tgf.h"
#include "lattice.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(36) << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch, looked up once per device.  In host code the symbol
// names a host-side stand-in, never the device memory, so it must not be passed to a kernel.
std::mutex g_mu;
void* g_addr[64] = {};

}  // namespace

extern "C" tgf_status tgf_measure_noalloc(int prec, const tgf_lattice* lat, int ncfg, const void* links,
                                          tgf_obs* obs_dev, size_t obs_stride, int rec, double t, unsigned flags,
                                          void* stream) {
    size_t need = 0;
    tgf_status s = tgf_scratch_bytes(prec, lat, ncfg, &need);
    if (s != TGF_OK) return s;
    if (need > kStaticScratchBytes)
        return (tgf_status)tgf::set_error(TGF_EINVAL,
                              "tgf_measure_noalloc: this batch needs %zu bytes of scratch, more than the library's "
                              "fixed %zu-byte device array; use tgf_measure with caller-provided scratch",
                              need, kStaticScratchBytes);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return (tgf_status)tgf::set_error(TGF_ECUDA, "tgf_measure_noalloc: cudaGetDevice failed");
    if (dev < 0 || dev >= 64) return (tgf_status)tgf::set_error(TGF_EINVAL, "tgf_measure_noalloc: device %d out of range", dev);
    void* ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess || !p)
                return (tgf_status)tgf::set_error(TGF_ECUDA, "tgf_measure_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            g_addr[dev] = p;
        }
        ptr = g_addr[dev];
    }
    return tgf_measure(prec, lat, ncfg, links, static_cast<double*>(ptr), kStaticScratchBytes, obs_dev, obs_stride,
                       rec, t, flags, stream);
}
