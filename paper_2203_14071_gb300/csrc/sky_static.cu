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
// stream capture.  Every call on a device shares the array: calls that overlap on
// the GPU (different streams, or different host threads without ordering) race
// on it.  Each call clears the status word it uses before its kernels run; the
// per-source table is fully rewritten by every call.
#include <cmath>
#include <cstring>
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

bool params_valid(const rlf_params &p)
{
    return p.facet_n >= 2 && p.facet_n <= RLF_MAX_FACET_N && p.facet_n % 2 == 0 && p.n_e >= 2 &&
           p.n_e <= rlf::kMaxNe && p.n_alpha >= 1 && p.n_alpha <= 64 && p.sigma_jy > 0 && p.psf_nat > 0 &&
           std::isfinite(p.psf_nat) && p.r_min_arcsec > 0 && p.r_max_arcsec >= p.r_min_arcsec && p.r_std > 0 &&
           p.thresh_frac > 0 && p.thresh_frac <= 1 && p.e_max > 0 && p.e_max <= 1 && p.nu_ref_hz > 0 &&
           std::isfinite(p.nu_ref_hz) && std::isfinite(p.beta) && std::isfinite(p.add) && std::isfinite(p.esp) &&
           (p.precision == RLF_PREC_FP64 || p.precision == RLF_PREC_MIXED || p.precision == RLF_PREC_MIXED_SPLIT) &&
           (p.flux_prior == 0 || p.flux_prior == 1) && (p.update_mode == 0 || p.update_mode == 1);
}

rlf::ChanTable channel_table(const rlf_uvw &uvw, const rlf_params &p)
{
    rlf::ChanTable ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.n = uvw.n_chan;
    double mean = 0.0;
    for (int k = 0; k < ch.n; ++k) {
        ch.s[k] = uvw.freq_hz[k] / rlf::kC;
        ch.spec[k] = std::pow(uvw.freq_hz[k] / p.nu_ref_hz, p.beta);
        ch.s_hi[k] = (float)ch.s[k];
        ch.s_lo[k] = (float)(ch.s[k] - (double)ch.s_hi[k]);
        mean += ch.spec[k];
    }
    ch.spec_off = mean / ch.n;
    ch.s0 = ch.s[0];
    ch.ds = ch.n > 1 ? (ch.s[ch.n - 1] - ch.s[0]) / (ch.n - 1) : 0.0;
    ch.ds_hi = (float)ch.ds;
    ch.ds_lo = (float)(ch.ds - (double)ch.ds_hi);
    ch.profile = p.profile;
    ch.pad = 0;
    ch.uniform = 1;
    for (int k = 0; k < ch.n; ++k)
        if (std::fabs(ch.s[k] - (ch.s0 + k * ch.ds)) > 1e-12 * ch.s0) ch.uniform = 0;
    return ch;
}

}  // namespace

extern "C" rlf_status rlf_sky_model_static(const rlf_uvw *uvw, const rlf_sources *src,
                                           const rlf_params *p, float *vis_sky, void *stream)
{
    if (!uvw || !uvw->u || !uvw->v || !uvw->w || !uvw->freq_hz || uvw->n_rows <= 0 || uvw->n_chan <= 0 ||
        uvw->n_baselines < 0)
        return RLF_EINVAL;
    if (uvw->n_chan > RLF_MAX_CHAN) return RLF_EUNSUPPORTED;
    for (int k = 0; k < uvw->n_chan; ++k)
        if (!(uvw->freq_hz[k] > 0 && std::isfinite(uvw->freq_hz[k])) ||
            (k > 0 && !(uvw->freq_hz[k] > uvw->freq_hz[k - 1])))
            return RLF_EINVAL;
    if (!src || !src->l || !src->m || !src->flux_jy || !src->e1 || !src->e2 || src->n_src <= 0) return RLF_EINVAL;
    if (!p || !params_valid(*p) || !vis_sky) return RLF_EINVAL;
    if (src->n_src > RLF_STATIC_MAX_SRC) return RLF_ENOSPACE;   // the fixed table holds RLF_STATIC_MAX_SRC
    void *base = nullptr;
    rlf_status s = scratch_address(&base);
    if (s != RLF_OK) return s;
    int32_t *status = static_cast<int32_t *>(base);
    rlf::SrcRow *table = reinterpret_cast<rlf::SrcRow *>(static_cast<unsigned char *>(base) + kStatusBytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const rlf::ChanTable ch = channel_table(*uvw, *p);
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = rlf::launch_prepare(*src, 0, src->n_src, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                                nullptr, *p, table, status, st);
    if (e == cudaSuccess) e = rlf::launch_sky(*uvw, ch, table, src->n_src, false, p->precision, vis_sky, st);
    return e == cudaSuccess ? RLF_OK : RLF_ECUDA;
}
