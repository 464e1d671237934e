// rlf_sky_model_static: the sky model for callers that cannot allocate device
// memory.
//
// rlf_sky_model needs a caller-supplied workspace for its per-source table.  Some
// callers cannot provide one: code that runs where cudaMalloc is not allowed or
// not wanted, such as inside another framework's memory pool with no spare
// allocation hook, a real-time loop that must never allocate after start-up, or
// a plugin that only receives input and output buffers.  This variant keeps that
// table in a fixed array in the library's own device memory instead.
//
// The array below is a file-scope static __device__ array: every GPU that loads
// the library holds it (about 460 KB) until the process exits.  In host code its
// name is only a host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress, once per device, with that device current, on the first
// call made on the device.  That first call should therefore come before any
// stream capture.  The address is kept per device ordinal for the life of the
// process, so the entry point must not be used across a cudaDeviceReset (which
// reloads the module and moves the array).  Every call on a device shares the
// array: calls that overlap on the GPU (different streams, or different host
// threads without ordering) race on it.  Each call clears the status word it uses
// before its kernels run; the per-source table is fully rewritten by every call.
// Arguments are checked exactly as rlf_sky_model checks them.
#include <mutex>

#include "rlf_internal.cuh"

namespace {

constexpr int kStaticMaxDevices = 64;
constexpr size_t kStatusBytes = 256;
constexpr size_t kStaticBytes = kStatusBytes + (size_t)RLF_STATIC_MAX_SRC * sizeof(rlf::SrcRow);

// status word (first 256 bytes) followed by the per-source table
static __device__ __align__(256) unsigned char g_sky_scratch[kStaticBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kStaticMaxDevices] = {};

// Device address of g_sky_scratch on the current device (looked up once per device).
rlf_status scratch_address(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return RLF_ECUDA;
    if (dev < 0 || dev >= kStaticMaxDevices) return RLF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sky_scratch) != cudaSuccess || !p) return RLF_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RLF_OK;
}

}  // namespace

extern "C" rlf_status rlf_sky_model_static(const rlf_uvw *uvw, const rlf_sources *src,
                                           const rlf_params *p, float *vis_sky, void *stream)
{
    // the same argument checks as rlf_sky_model
    rlf_status s = rlf::check_uvw(uvw);
    if (s != RLF_OK) return s;
    if (!src) return RLF_EINVAL;
    if ((s = rlf::check_src(src, 0, src->n_src)) != RLF_OK) return s;
    if (!p || !rlf::params_ok(*p) || !vis_sky) return RLF_EINVAL;
    if (src->n_src > RLF_STATIC_MAX_SRC) return RLF_ENOSPACE;   // the fixed table holds RLF_STATIC_MAX_SRC
    void *base = nullptr;
    if ((s = scratch_address(&base)) != RLF_OK) return s;
    int32_t *status = static_cast<int32_t *>(base);
    rlf::SrcRow *table = reinterpret_cast<rlf::SrcRow *>(static_cast<unsigned char *>(base) + kStatusBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const rlf::ChanTable ch = rlf::make_chan_table(*uvw, *p);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = rlf::launch_prepare(*src, 0, src->n_src, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                                nullptr, *p, table, status, st);
    // the caller's launch shape; no split-baseline records (there is no workspace to hold
    // them): in split mode each row's float-pair phase is formed on the fly
    if (e == cudaSuccess)
        e = rlf::launch_sky(*uvw, ch, table, src->n_src, false, p->precision, vis_sky, st, p->tune_sky_blocks, 1.0f,
                            rlf::SplitRows());
    return e == cudaSuccess ? RLF_OK : RLF_ECUDA;
}
