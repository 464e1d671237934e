// C ABI entry points (include/rlf.h): argument checks, the channel table,
// workspace carve-up and the whole-chain driver.  Host code only; the work is
// in sky.cu, extract.cu and fit.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

bool params_ok(const rlf_params &p)
{
    if (!(p.facet_n >= 2 && p.facet_n <= RLF_MAX_FACET_N && p.facet_n % 2 == 0)) return false;
    if (!(p.n_e >= 2 && p.n_e <= kMaxNe)) return false;
    if (!(p.n_alpha >= 1 && p.n_alpha <= 64)) return false;
    if (!(p.sigma_jy > 0 && std::isfinite(p.sigma_jy))) return false;
    if (!(p.psf_nat > 0 && std::isfinite(p.psf_nat))) return false;
    if (!(p.r_min_arcsec > 0 && p.r_max_arcsec >= p.r_min_arcsec && std::isfinite(p.r_max_arcsec))) return false;
    if (!(p.r_std > 0 && std::isfinite(p.r_std))) return false;
    if (!(p.thresh_frac > 0 && p.thresh_frac <= 1)) return false;
    if (!(p.e_max > 0 && p.e_max <= 1)) return false;
    if (!(p.nu_ref_hz > 0 && std::isfinite(p.nu_ref_hz))) return false;
    if (!std::isfinite(p.beta) || !std::isfinite(p.add) || !std::isfinite(p.esp)) return false;
    if (p.precision != RLF_PREC_FP64 && p.precision != RLF_PREC_MIXED && p.precision != RLF_PREC_MIXED_SPLIT)
        return false;
    if (p.flux_prior != 0 && p.flux_prior != 1) return false;
    if (p.update_mode != 0 && p.update_mode != 1) return false;
    if (p.profile != RLF_PROFILE_EXPONENTIAL && p.profile != RLF_PROFILE_GAUSSIAN) return false;
    if (p.estimator != RLF_ESTIMATOR_GRID && p.estimator != RLF_ESTIMATOR_ADAPTIVE) return false;
    if (p.estimator == RLF_ESTIMATOR_ADAPTIVE && !(p.np_max >= 1 && p.e_res > 0 && std::isfinite(p.e_res)))
        return false;
    if (p.refit_bad != 0 && p.refit_bad != 1) return false;
    if (!(p.n_pos >= 0 && p.n_pos <= RLF_MAX_POS && (p.n_pos <= 1 || p.n_pos % 2 == 1))) return false;
    if (p.n_pos > 1 && !(p.pos_step_arcsec > 0 && std::isfinite(p.pos_step_arcsec))) return false;
    if (p.tune_fit_ag != 0 && p.tune_fit_ag != 2 && p.tune_fit_ag != 4 && p.tune_fit_ag != 8) return false;
    if (p.tune_fit_blocks < 0 || p.tune_extract_waves < 0 || p.tune_sky_blocks < 0) return false;
    return true;
}

rlf_status check_uvw(const rlf_uvw *uvw)
{
    if (!uvw || !uvw->u || !uvw->v || !uvw->w || !uvw->freq_hz) return RLF_EINVAL;
    if (uvw->n_rows <= 0 || uvw->n_chan <= 0 || uvw->n_baselines < 0) return RLF_EINVAL;
    if (uvw->n_chan > RLF_MAX_CHAN || uvw->n_rows > RLF_MAX_ROWS) return RLF_EUNSUPPORTED;
    for (int k = 0; k < uvw->n_chan; ++k) {
        if (!(uvw->freq_hz[k] > 0 && std::isfinite(uvw->freq_hz[k]))) return RLF_EINVAL;
        if (k > 0 && !(uvw->freq_hz[k] > uvw->freq_hz[k - 1])) return RLF_EINVAL;
    }
    return RLF_OK;
}

rlf_status check_src(const rlf_sources *src, int32_t first, int32_t count)
{
    if (!src || !src->l || !src->m || !src->flux_jy || !src->e1 || !src->e2) return RLF_EINVAL;
    if (src->n_src <= 0 || first < 0 || count <= 0 || (int64_t)first + count > src->n_src) return RLF_EINVAL;
    return RLF_OK;
}

ChanTable make_chan_table(const rlf_uvw &uvw, const rlf_params &p)
{
    ChanTable ch;
    std::memset(&ch, 0, sizeof(ch));
    ch.n = uvw.n_chan;
    for (int k = 0; k < ch.n; ++k) {
        ch.s[k] = uvw.freq_hz[k] / kC;
        ch.spec[k] = std::pow(uvw.freq_hz[k] / p.nu_ref_hz, p.beta);
    }
    for (int k = 0; k < ch.n; ++k) {
        ch.s_hi[k] = (float)ch.s[k];
        ch.s_lo[k] = (float)(ch.s[k] - (double)ch.s_hi[k]);
    }
    double mean = 0.0;
    for (int k = 0; k < ch.n; ++k) mean += ch.spec[k];
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

namespace {

rlf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RLF_OK : RLF_ECUDA; }

int32_t fit_capacity(int32_t n_src, const rlf_params &p, int32_t which)
{
    if (which == RLF_WS_RUN) return (p.chunk > 0 && p.chunk < n_src) ? p.chunk : n_src;
    return n_src;
}

}  // namespace

size_t workspace_layout(int64_t n_rows, int32_t n_chan, int32_t n_src, const rlf_params &p,
                        int32_t which, void *base, Workspace *ws)
{
    const size_t NN = (size_t)p.facet_n * p.facet_n;
    const size_t ng = (size_t)p.n_e * p.n_e * p.n_alpha;
    const size_t cap = (size_t)fit_capacity(n_src, p, which);
    const bool fit = which == RLF_WS_FIT || which == RLF_WS_RUN;
    const bool run = which == RLF_WS_RUN;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t o_status = take(64 * sizeof(int32_t));
    const size_t o_table = take((size_t)n_src * sizeof(SrcRow));
    const size_t o_upd = take((which == RLF_WS_SKY || run) ? (size_t)n_src * sizeof(SrcRow) : 0);
    const size_t o_cells = take(fit ? (4 + (size_t)b_stride(n_offsets(p))) * cap * NN * sizeof(double) : 0);
    const size_t o_ncell = take(fit ? cap * sizeof(int32_t) : 0);
    const size_t o_order = take(fit ? cap * sizeof(int32_t) : 0);
    const size_t o_count = take(fit ? (cap + 1) * sizeof(int32_t) : 0);
    const size_t o_cc = take(fit ? cap * sizeof(double) : 0);
    const size_t o_box = take(fit ? cap * 3 * sizeof(int32_t) : 0);
    const size_t o_wide = take(fit ? cap * sizeof(int32_t) : 0);
    const size_t o_map = take(fit ? cap * sizeof(int32_t) : 0);
    const size_t o_refit = take(fit ? (cap + 1) * sizeof(int32_t) : 0);
    const bool mlp = fit && p.facet_n * p.facet_n * 2 == kMlpIn;
    const size_t o_mx = take(mlp ? cap * kMlpIn * sizeof(__half) : 0);
    const size_t o_ms = take(mlp ? mlp_scratch(nullptr, (int32_t)cap).bytes : 0);
    // a few facets at a time split their cells further (the serial order fits one facet per chunk)
    const size_t fit_parts = cap <= 16 ? 16 : kMaxFitParts;
    const size_t o_ga = take(fit ? fit_parts * cap * ng * sizeof(double) : 0);
    const size_t o_gb = take(fit ? fit_parts * cap * ng * sizeof(double) : 0);
    const size_t o_gl = take(fit ? cap * ng * sizeof(double) : 0);
    const bool adapt = fit && p.estimator == RLF_ESTIMATOR_ADAPTIVE;
    const size_t o_ad = take(adapt ? cap * adapt_doubles_per_facet(p.n_alpha) * sizeof(double) : 0);
    const size_t o_ecur = take(run ? 2 * (size_t)n_src * sizeof(double) : 0);
    const size_t o_bad = take(run ? ((size_t)n_src + 1) * sizeof(int32_t) : 0);
    const size_t o_ftmp = take(run ? 8 * cap * sizeof(double) : 0);
    const size_t o_gtmp = take(run ? cap * sizeof(int32_t) : 0);
    const size_t o_fac = take(run ? cap * 4 * NN * sizeof(double) : 0);
    const bool ext = which == RLF_WS_EXTRACT || run;
    const size_t rows = (size_t)(n_rows > 0 ? n_rows : 0), chans = (size_t)(n_chan > 0 ? n_chan : 0);
    // split baselines: the extraction's (in baseline order) and the sky calls' (row order)
    const size_t o_split = take((ext || which == RLF_WS_SKY) ? 8 * rows * sizeof(float) : 0);
    const size_t o_resid = take(ext ? rows * chans * 2 * sizeof(float) : 0);
    const size_t n_partials = std::min((size_t)kMaxPartials, (size_t)kPartialsPerSource * (size_t)(n_src > 0 ? n_src : 1));
    const size_t o_part = take(ext ? n_partials * 4 * NN * sizeof(float) : 0);
    const size_t o_ext = take(ext ? rows * sizeof(float) : 0);
    const size_t o_perm = take(ext ? rows * sizeof(int32_t) : 0);
    const size_t o_live = take(ext ? (size_t)n_src * sizeof(int32_t) : 0);
    const size_t o_ocnt = take(ext ? (size_t)kOrderBuckets * kOrderThreads * sizeof(int32_t) : 0);
    const size_t total = off + 256;   // slack for aligning an arbitrary base pointer
    if (ws && base) {
        char *b = reinterpret_cast<char *>(align_up(reinterpret_cast<size_t>(base), 256));
        ws->status = reinterpret_cast<int32_t *>(b + o_status);
        ws->table = reinterpret_cast<SrcRow *>(b + o_table);
        ws->upd = reinterpret_cast<SrcRow *>(b + o_upd);
        ws->cells = b + o_cells;
        ws->ncell = reinterpret_cast<int32_t *>(b + o_ncell);
        ws->order = reinterpret_cast<int32_t *>(b + o_order);
        ws->box = reinterpret_cast<int32_t *>(b + o_box);
        ws->wide = reinterpret_cast<int32_t *>(b + o_wide);
        ws->map_index = reinterpret_cast<int32_t *>(b + o_map);
        ws->refit = reinterpret_cast<int32_t *>(b + o_refit);
        ws->mlp_x = b + o_mx;
        ws->mlp_scratch = b + o_ms;
        ws->counters = reinterpret_cast<int32_t *>(b + o_count);
        ws->cc = reinterpret_cast<double *>(b + o_cc);
        ws->ga = reinterpret_cast<double *>(b + o_ga);
        ws->gb = reinterpret_cast<double *>(b + o_gb);
        ws->part_stride = cap * ng;
        ws->fit_parts = (int32_t)fit_parts;
        ws->gl = reinterpret_cast<double *>(b + o_gl);
        ws->adapt = reinterpret_cast<double *>(b + o_ad);
        ws->e_cur = reinterpret_cast<double *>(b + o_ecur);
        ws->bad_list = reinterpret_cast<int32_t *>(b + o_bad);
        ws->fit_tmp = reinterpret_cast<double *>(b + o_ftmp);
        ws->flag_tmp = reinterpret_cast<int32_t *>(b + o_gtmp);
        ws->facets = reinterpret_cast<double *>(b + o_fac);
        ws->uvw_split = reinterpret_cast<float *>(b + o_split);
        ws->resid = reinterpret_cast<float *>(b + o_resid);
        ws->partial = reinterpret_cast<float *>(b + o_part);
        ws->n_partials = (int32_t)n_partials;
        ws->extent = reinterpret_cast<float *>(b + o_ext);
        ws->perm = reinterpret_cast<int32_t *>(b + o_perm);
        ws->n_live = reinterpret_cast<int32_t *>(b + o_live);
        ws->order_counts = reinterpret_cast<int32_t *>(b + o_ocnt);
        ws->bytes = total;
    }
    return total;
}

}  // namespace rlf

using namespace rlf;

extern "C" {

void rlf_params_default(rlf_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->add = -0.93;
    p->esp = 0.33;
    p->psf_nat = 38.0;
    p->beta = -0.7;
    p->nu_ref_hz = 1.4e9;
    p->sigma_jy = 1e-6;
    p->e_max = 0.8;
    p->r_min_arcsec = 0.3;
    p->r_max_arcsec = 3.5;
    p->r_std = 0.3136;
    p->thresh_frac = 0.05;
    p->var_sigma_min = 5e-3;
    p->var_det_min = 5e-5;
    p->facet_n = 64;
    p->n_e = 21;
    p->n_alpha = 20;
    p->flux_prior = 0;
    p->chunk = 0;
    p->update_mode = 0;
    p->precision = RLF_PREC_MIXED;
    p->e_res = 0.003;
    p->np_max = 30;
    p->estimator = RLF_ESTIMATOR_GRID;
    p->n_pos = 1;
    p->pos_step_arcsec = 0.1;
}

size_t rlf_workspace_size(int64_t n_rows, int32_t n_chan, int32_t n_src, const rlf_params *p,
                          int32_t which)
{
    if (!p || !params_ok(*p) || n_src <= 0 || which < RLF_WS_SKY || which > RLF_WS_RUN) return 0;
    return workspace_layout(n_rows, n_chan, n_src, *p, which, nullptr, nullptr);
}

size_t rlf_facets_size(int32_t count, const rlf_params *p)
{
    if (!p || count <= 0 || !params_ok(*p)) return 0;
    return (size_t)count * 4 * p->facet_n * p->facet_n * sizeof(double);
}

const char *rlf_strerror(rlf_status s)
{
    switch (s) {
    case RLF_OK: return "ok";
    case RLF_EINVAL: return "invalid argument";
    case RLF_ECUDA: return "CUDA error";
    case RLF_ENOSPACE: return "workspace or buffer too small";
    case RLF_ETIMEOUT: return "bounded device wait timed out";
    case RLF_ENUMERIC: return "non-finite likelihood";
    case RLF_EUNSUPPORTED: return "request outside the implemented limits";
    }
    return "unknown status";
}

rlf_status rlf_sky_model(const rlf_uvw *uvw, const rlf_sources *src, const rlf_params *p,
                         float *vis_sky, void *workspace, size_t ws_bytes, void *stream)
{
    rlf_status s = check_uvw(uvw);
    if (s != RLF_OK) return s;
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    if ((s = check_src(src, 0, src ? src->n_src : 0)) != RLF_OK) return s;
    if (!vis_sky || !workspace) return RLF_EINVAL;
    Workspace ws;
    if (workspace_layout(uvw->n_rows, uvw->n_chan, src->n_src, *p, RLF_WS_SKY, workspace, &ws) > ws_bytes)
        return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ChanTable ch = make_chan_table(*uvw, *p);
    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_prepare(*src, 0, src->n_src, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                           nullptr, *p, ws.table, ws.status, st);
    SplitRows sr;
    if (e == cudaSuccess && p->precision == RLF_PREC_MIXED_SPLIT) {
        e = launch_split_uvw(*uvw, ws.uvw_split, st);
        sr.rec = ws.uvw_split;
    }
    if (e == cudaSuccess)
        e = launch_sky(*uvw, ch, ws.table, src->n_src, false, p->precision, vis_sky, st, p->tune_sky_blocks, 1.0f, sr);
    return cuda_status(e);
}

rlf_status rlf_sky_update(const rlf_uvw *uvw, const rlf_sources *src, int32_t first,
                          int32_t count, const double *e1_new, const double *e2_new,
                          const int32_t *flag, const rlf_params *p, float *vis_sky,
                          void *workspace, size_t ws_bytes, void *stream)
{
    rlf_status s = check_uvw(uvw);
    if (s != RLF_OK) return s;
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    if ((s = check_src(src, first, count)) != RLF_OK) return s;
    if (!vis_sky || !workspace || !e1_new || !e2_new) return RLF_EINVAL;
    Workspace ws;
    if (workspace_layout(uvw->n_rows, uvw->n_chan, src->n_src, *p, RLF_WS_SKY, workspace, &ws) > ws_bytes)
        return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ChanTable ch = make_chan_table(*uvw, *p);
    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_prepare(*src, first, count, src->e1, src->e2, e1_new, e2_new, flag,
                           flag ? p->update_mode : 1, nullptr, nullptr, *p, ws.upd, ws.status, st);
    SplitRows sr;
    if (e == cudaSuccess && p->precision == RLF_PREC_MIXED_SPLIT) {
        e = launch_split_uvw(*uvw, ws.uvw_split, st);
        sr.rec = ws.uvw_split;
    }
    if (e == cudaSuccess)
        e = launch_sky(*uvw, ch, ws.upd, count, true, p->precision, vis_sky, st, p->tune_sky_blocks, 1.0f, sr);
    return cuda_status(e);
}

rlf_status rlf_extract_facets(const rlf_uvw *uvw, const float *vis_data, const float *vis_sky,
                              const rlf_sources *src, int32_t first, int32_t count,
                              const rlf_params *p, double *facets, size_t facets_bytes,
                              void *workspace, size_t ws_bytes, void *stream)
{
    rlf_status s = check_uvw(uvw);
    if (s != RLF_OK) return s;
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    if ((s = check_src(src, first, count)) != RLF_OK) return s;
    if (!vis_data || !vis_sky || !facets || !workspace) return RLF_EINVAL;
    if (facets_bytes < rlf_facets_size(count, p)) return RLF_ENOSPACE;
    Workspace ws;
    if (workspace_layout(uvw->n_rows, uvw->n_chan, src->n_src, *p, RLF_WS_EXTRACT, workspace, &ws) > ws_bytes)
        return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ChanTable ch = make_chan_table(*uvw, *p);
    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_prepare(*src, first, count, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                           nullptr, *p, ws.table, ws.status, st);
    if (e == cudaSuccess) e = launch_extract_prepare(*uvw, *p, ws, st);
    if (e == cudaSuccess) e = launch_extract(*uvw, ch, vis_data, vis_sky, ws.table, count, *p, ws, facets, st);
    return cuda_status(e);
}

rlf_status rlf_fit_sources(const double *facets, const rlf_sources *src, int32_t first,
                           int32_t count, const rlf_params *p, const rlf_fit_out *out,
                           void *workspace, size_t ws_bytes, void *stream)
{
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    rlf_status s = check_src(src, first, count);
    if (s != RLF_OK) return s;
    if (!facets || !workspace || !out || !out->e1 || !out->e2 || !out->sig1 || !out->sig2 ||
        !out->alpha_arcsec || !out->flux_jy || !out->e1_smooth || !out->e2_smooth || !out->flag)
        return RLF_EINVAL;
    Workspace ws;
    if (workspace_layout(0, 1, src->n_src, *p, RLF_WS_FIT, workspace, &ws) > ws_bytes) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_prepare(*src, first, count, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                           nullptr, *p, ws.table, ws.status, st);
    if (e == cudaSuccess) e = launch_fit(facets, ws.table, count, *p, ws, *out, 0, st);
    return cuda_status(e);
}

}  // extern "C"

namespace {

// Argument checks shared by rlf_run, rlf_graph_create and rlf_autotune.
rlf_status check_run(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src, const rlf_params *p,
                     const rlf_fit_out *out, const float *vis_sky, void *workspace, size_t ws_bytes, Workspace *ws)
{
    rlf_status s = check_uvw(uvw);
    if (s != RLF_OK) return s;
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    if ((s = check_src(src, 0, src ? src->n_src : 0)) != RLF_OK) return s;
    if (!vis_data || !vis_sky || !workspace || !out || !out->e1 || !out->e2 || !out->sig1 ||
        !out->sig2 || !out->alpha_arcsec || !out->flux_jy || !out->e1_smooth || !out->e2_smooth ||
        !out->flag)
        return RLF_EINVAL;
    if (workspace_layout(uvw->n_rows, uvw->n_chan, src->n_src, *p, RLF_WS_RUN, workspace, ws) > ws_bytes)
        return RLF_ENOSPACE;
    return RLF_OK;
}

// The whole chain on stream st (arguments already checked).
cudaError_t run_chain(const rlf_uvw &uvw, const float *vis_data, const rlf_sources &src, const rlf_params &p,
                      const rlf_fit_out &out, float *vis_sky, const Workspace &ws, cudaStream_t st)
{
    const int32_t n = src.n_src;
    const ChanTable ch = make_chan_table(uvw, p);
    const int32_t chunk = fit_capacity(n, p, RLF_WS_RUN);
    double *e1c = ws.e_cur, *e2c = ws.e_cur + n;

    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(e1c, src.e1, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(e2c, src.e2, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    // the sky model of the catalogue's current shapes (circular for a fresh catalogue)
    if (e == cudaSuccess)
        e = launch_prepare(src, 0, n, e1c, e2c, nullptr, nullptr, nullptr, 0, nullptr, nullptr, p, ws.table,
                           ws.status, st);
    // baseline extents and order, and (split mode) the split baselines, which the sky
    // kernels of this call read too
    if (e == cudaSuccess) e = launch_extract_prepare(uvw, p, ws, st);
    const SplitRows sr = split_rows(uvw, p, ws);
    if (e == cudaSuccess)
        e = launch_sky(uvw, ch, ws.table, n, false, p.precision, vis_sky, st, p.tune_sky_blocks, 1.0f, sr);
    // several chunks (mixed modes): keep the residual R = D - V resident instead of V, so
    // that each chunk's extraction reads one array; the updates subtract their terms
    // from R and the sky model is restored at the end as V = D - R
    const int64_t n_vis = uvw.n_rows * uvw.n_chan;
    const bool track_resid = chunk < n && p.precision != RLF_PREC_FP64 && ws.resid && n_vis % 2 == 0;
    if (e == cudaSuccess && track_resid) e = launch_difference(vis_data, vis_sky, n_vis, ws.resid, st);
    for (int32_t first = 0; first < n && e == cudaSuccess; first += chunk) {
        const int32_t cnt = first + chunk <= n ? chunk : n - first;
        e = track_resid ? launch_extract(uvw, ch, ws.resid, nullptr, ws.table + first, cnt, p, ws, ws.facets, st)
                        : launch_extract(uvw, ch, vis_data, vis_sky, ws.table + first, cnt, p, ws, ws.facets, st);
        if (e != cudaSuccess) break;
        e = launch_fit(ws.facets, ws.table + first, cnt, p, ws, out, first, st);
        if (e != cudaSuccess) break;
        // replace the chunk's shapes in the sky model (good fits, or all with update_mode 1)
        e = launch_prepare(src, first, cnt, e1c, e2c, out.e1 + first, out.e2 + first, out.flag + first,
                           p.update_mode, e1c, e2c, p, ws.upd, ws.status, st);
        if (e != cudaSuccess) break;
        if (cnt == n) {
            // one chunk holds every source and the sky model was made from scratch at the
            // start of this call: the updated model, sum of old terms plus every (new - old),
            // is the model of the committed shapes, formed directly with one term per source
            e = launch_prepare(src, 0, n, e1c, e2c, nullptr, nullptr, nullptr, 0, nullptr, nullptr, p, ws.table,
                               ws.status, st);
            if (e == cudaSuccess)
                e = launch_sky(uvw, ch, ws.table, n, false, p.precision, vis_sky, st, p.tune_sky_blocks, 1.0f, sr);
        } else if (track_resid) {
            e = launch_sky(uvw, ch, ws.upd, cnt, true, p.precision, ws.resid, st, p.tune_sky_blocks, -1.0f, sr);
        } else {
            e = launch_sky(uvw, ch, ws.upd, cnt, true, p.precision, vis_sky, st, p.tune_sky_blocks, 1.0f, sr);
        }
    }
    // the bad fits once more, against the sky model of every other measured shape (Sec. 2.4),
    // in source order and chunks of the same size; their number sizes the launches, so the
    // stream is synchronised once here (not capturable)
    if (e == cudaSuccess && p.refit_bad) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess) return e;
        if (cs != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
        e = launch_bad_list(out.flag, n, ws.bad_list, st);
        int32_t nb = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, ws.bad_list, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        const size_t cap = (size_t)chunk;
        const rlf_fit_out tmp{ws.fit_tmp, ws.fit_tmp + cap, ws.fit_tmp + 2 * cap, ws.fit_tmp + 3 * cap,
                              ws.fit_tmp + 4 * cap, ws.fit_tmp + 5 * cap, ws.fit_tmp + 6 * cap, ws.fit_tmp + 7 * cap,
                              ws.flag_tmp};
        for (int32_t first = 0; first < nb && e == cudaSuccess; first += chunk) {
            const int32_t cnt = first + chunk <= nb ? chunk : nb - first;
            const int32_t *list = ws.bad_list + 1 + first;
            e = launch_prepare(src, 0, cnt, e1c, e2c, nullptr, nullptr, nullptr, 0, nullptr, nullptr, p, ws.table,
                               ws.status, st, list);
            if (e != cudaSuccess) break;
            e = track_resid ? launch_extract(uvw, ch, ws.resid, nullptr, ws.table, cnt, p, ws, ws.facets, st)
                            : launch_extract(uvw, ch, vis_data, vis_sky, ws.table, cnt, p, ws, ws.facets, st);
            if (e != cudaSuccess) break;
            e = launch_fit(ws.facets, ws.table, cnt, p, ws, tmp, 0, st);
            if (e != cudaSuccess) break;
            e = launch_scatter(ws.fit_tmp, ws.flag_tmp, cap, list, cnt, out, st);
            if (e != cudaSuccess) break;
            e = launch_prepare(src, 0, cnt, e1c, e2c, tmp.e1, tmp.e2, tmp.flag, p.update_mode, e1c, e2c, p, ws.upd,
                               ws.status, st, list);
            if (e != cudaSuccess) break;
            e = track_resid
                    ? launch_sky(uvw, ch, ws.upd, cnt, true, p.precision, ws.resid, st, p.tune_sky_blocks, -1.0f, sr)
                    : launch_sky(uvw, ch, ws.upd, cnt, true, p.precision, vis_sky, st, p.tune_sky_blocks, 1.0f, sr);
        }
    }
    if (e == cudaSuccess && track_resid) e = launch_difference(vis_data, ws.resid, n_vis, vis_sky, st);
    return e;
}

// Median of `reps` timings of fn on st (CUDA events), in ms; negative on error.
template <typename F>
float time_median(F fn, cudaStream_t st, int reps)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.0f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.0f;
    }
    float t[8];
    reps = reps < 1 ? 1 : (reps > 8 ? 8 : reps);
    bool ok = fn() == cudaSuccess;   // warm-up
    for (int i = 0; i < reps && ok; ++i) {
        ok = cudaEventRecord(a, st) == cudaSuccess && fn() == cudaSuccess && cudaEventRecord(b, st) == cudaSuccess &&
             cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&t[i], a, b) == cudaSuccess;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (!ok) return -1.0f;
    for (int i = 1; i < reps; ++i)
        for (int j = i; j > 0 && t[j] < t[j - 1]; --j) {
            const float x = t[j];
            t[j] = t[j - 1];
            t[j - 1] = x;
        }
    return t[reps / 2];
}

}  // namespace

struct rlf_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

extern "C" {

rlf_status rlf_run(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src,
                   const rlf_params *p, const rlf_fit_out *out, float *vis_sky,
                   void *workspace, size_t ws_bytes, void *stream)
{
    Workspace ws;
    const rlf_status s = check_run(uvw, vis_data, src, p, out, vis_sky, workspace, ws_bytes, &ws);
    if (s != RLF_OK) return s;
    return cuda_status(run_chain(*uvw, vis_data, *src, *p, *out, vis_sky, ws, static_cast<cudaStream_t>(stream)));
}

rlf_status rlf_graph_create(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src,
                            const rlf_params *p, const rlf_fit_out *out, float *vis_sky, void *workspace,
                            size_t ws_bytes, void *stream, rlf_graph **graph_out)
{
    if (!graph_out || !stream) return RLF_EINVAL;
    *graph_out = nullptr;
    Workspace ws;
    const rlf_status s = check_run(uvw, vis_data, src, p, out, vis_sky, workspace, ws_bytes, &ws);
    if (s != RLF_OK) return s;
    // the refit pass sizes its launches from the number of bad fits, read on the host
    if (p->refit_bad) return RLF_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RLF_ECUDA;
    const cudaError_t e = run_chain(*uvw, vis_data, *src, *p, *out, vis_sky, ws, st);
    const cudaError_t e2 = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess || e2 != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return RLF_ECUDA;
    }
    cudaGraphExec_t exec = nullptr;
    if (cudaGraphInstantiate(&exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return RLF_ECUDA;
    }
    rlf_graph *h = new (std::nothrow) rlf_graph{g, exec};
    if (!h) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(g);
        return RLF_ECUDA;
    }
    *graph_out = h;
    return RLF_OK;
}

rlf_status rlf_graph_launch(rlf_graph *graph, void *stream)
{
    if (!graph) return RLF_EINVAL;
    return cuda_status(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
}

void rlf_graph_destroy(rlf_graph *graph)
{
    if (!graph) return;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
}

rlf_status rlf_autotune(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src, rlf_params *p,
                        const rlf_fit_out *out, float *vis_sky, void *workspace, size_t ws_bytes, void *stream,
                        float *phase_ms)
{
    Workspace ws;
    rlf_status s = check_run(uvw, vis_data, src, p, out, vis_sky, workspace, ws_bytes, &ws);
    if (s != RLF_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t n = src->n_src;
    const int32_t chunk = fit_capacity(n, *p, RLF_WS_RUN);
    const ChanTable ch = make_chan_table(*uvw, *p);
    const int reps = 3;
    rlf_params q = *p;
    // the sky model of the catalogue and the split baselines, inputs of the timed steps
    cudaError_t e = launch_prepare(*src, 0, n, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr, nullptr, q,
                                   ws.table, ws.status, st);
    if (e == cudaSuccess) e = launch_extract_prepare(*uvw, q, ws, st);
    if (e != cudaSuccess) return RLF_ECUDA;
    const SplitRows sr = split_rows(*uvw, q, ws);
    float best[3] = {0, 0, 0};
    // 1. sky-model CTAs per SM
    {
        const int cand[] = {8, 16, 32, 64};
        float bt = 0;
        int bc = 8;
        for (int c : cand) {
            const float t = time_median([&] { return launch_sky(*uvw, ch, ws.table, n, false, q.precision, vis_sky, st, c,
                                                                1.0f, sr); },
                                        st, reps);
            if (t < 0) return RLF_ECUDA;
            if (bt == 0 || t < bt) {
                bt = t;
                bc = c;
            }
        }
        q.tune_sky_blocks = bc;
        best[0] = bt;
        if ((e = launch_sky(*uvw, ch, ws.table, n, false, q.precision, vis_sky, st, bc, 1.0f, sr)) != cudaSuccess)
            return RLF_ECUDA;
    }
    // 2. extraction waves (first chunk of sources)
    {
        const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16};
        float bt = 0;
        int bc = 2;
        for (int c : cand) {
            q.tune_extract_waves = c;
            const float t = time_median([&] {
                return launch_extract(*uvw, ch, vis_data, vis_sky, ws.table, chunk, q, ws, ws.facets, st);
            }, st, reps);
            if (t < 0) return RLF_ECUDA;
            if (bt == 0 || t < bt) {
                bt = t;
                bc = c;
            }
        }
        q.tune_extract_waves = bc;
        best[1] = bt;
        if (launch_extract(*uvw, ch, vis_data, vis_sky, ws.table, chunk, q, ws, ws.facets, st) != cudaSuccess)
            return RLF_ECUDA;
    }
    // 3. likelihood: scalelength nodes per thread x CTAs per SM
    {
        const int ags[] = {2, 4, 8};
        const int blocks[] = {1, 2, 3};
        float bt = 0;
        int ba = 4, bb = 0;
        for (int a : ags)
            for (int b : blocks) {
                q.tune_fit_ag = a;
                q.tune_fit_blocks = b;
                const float t = time_median([&] { return launch_fit(ws.facets, ws.table, chunk, q, ws, *out, 0, st); },
                                            st, reps);
                if (t < 0) return RLF_ECUDA;
                if (bt == 0 || t < bt) {
                    bt = t;
                    ba = a;
                    bb = b;
                }
            }
        q.tune_fit_ag = ba;
        q.tune_fit_blocks = bb;
        best[2] = bt;
    }
    p->tune_sky_blocks = q.tune_sky_blocks;
    p->tune_extract_waves = q.tune_extract_waves;
    p->tune_fit_ag = q.tune_fit_ag;
    p->tune_fit_blocks = q.tune_fit_blocks;
    if (phase_ms) {
        phase_ms[0] = best[0];
        phase_ms[1] = best[1];
        phase_ms[2] = best[2];
    }
    return RLF_OK;
}

size_t rlf_mlp_weights_size(void) { return mlp_weights_bytes(); }

int64_t rlf_mlp_n_params(void) { return mlp_offsets().P; }

size_t rlf_mlp_workspace_size(int32_t max_batch)
{
    if (max_batch <= 0) return 0;
    return mlp_scratch(nullptr, max_batch).bytes + 256;
}

static bool aligned16(const void *p) { return (reinterpret_cast<size_t>(p) & 15u) == 0; }

static void *align256(void *p) { return reinterpret_cast<void *>((reinterpret_cast<size_t>(p) + 255) / 256 * 256); }

rlf_status rlf_mlp_init(void *weights, const float *normals, void *stream)
{
    if (!weights || !normals) return RLF_EINVAL;
    return cuda_status(mlp_init(mlp_weights(weights), normals, static_cast<cudaStream_t>(stream)));
}

rlf_status rlf_mlp_simulate(const double *templates, const double *template_flux, int32_t n_templates,
                            const int32_t *tidx, const double *e1, const double *e2, const double *alpha_arcsec,
                            const float *normals, int32_t batch, const rlf_params *p, void *x_f16, float *y,
                            void *stream)
{
    if (!templates || !template_flux || !tidx || !e1 || !e2 || !alpha_arcsec || !normals || !x_f16 || !y || !p)
        return RLF_EINVAL;
    if (n_templates <= 0 || batch <= 0 || !params_ok(*p)) return RLF_EINVAL;
    if (p->facet_n * p->facet_n * 2 != kMlpIn) return RLF_EUNSUPPORTED;
    return cuda_status(mlp_simulate(templates, n_templates, *p, template_flux, tidx, e1, e2, alpha_arcsec, normals, batch,
                                    p->facet_n, p->sigma_jy, static_cast<__half *>(x_f16), y,
                                    static_cast<cudaStream_t>(stream)));
}

rlf_status rlf_mlp_train_step(void *weights, const void *x_f16, const float *y, int32_t batch, float lr,
                              int32_t step, float *loss, void *workspace, size_t ws_bytes, void *stream)
{
    if (!weights || !x_f16 || !y || !workspace || batch <= 0 || !aligned16(x_f16) || !aligned16(weights))
        return RLF_EINVAL;
    if (ws_bytes < rlf_mlp_workspace_size(batch)) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    const MlpScratch sc = mlp_scratch(align256(workspace), batch);
    if (loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = mlp_train_step(mlp_weights(weights), static_cast<const __half *>(x_f16), y, batch, lr, step, loss, sc, st);
    return cuda_status(e);
}

rlf_status rlf_mlp_forward(const void *weights, const void *x_f16, int32_t batch, float *out, void *workspace,
                           size_t ws_bytes, void *stream)
{
    if (!weights || !x_f16 || !out || !workspace || batch <= 0 || !aligned16(x_f16)) return RLF_EINVAL;
    if (ws_bytes < rlf_mlp_workspace_size(batch)) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const MlpScratch sc = mlp_scratch(align256(workspace), batch);
    cudaError_t e = cudaMemsetAsync(sc.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = mlp_forward(mlp_weights(const_cast<void *>(weights)), static_cast<const __half *>(x_f16), batch, sc, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, sc.o, (size_t)batch * kMlpOutPad * sizeof(float), cudaMemcpyDeviceToDevice, st);
    return cuda_status(e);
}

rlf_status rlf_mlp_encode(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                          const rlf_params *p, void *x_f16, void *workspace, size_t ws_bytes, void *stream)
{
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    rlf_status s = check_src(src, first, count);
    if (s != RLF_OK) return s;
    if (!facets || !x_f16 || !workspace) return RLF_EINVAL;
    if (p->facet_n * p->facet_n * 2 != kMlpIn) return RLF_EUNSUPPORTED;
    Workspace ws;
    if (workspace_layout(0, 1, src->n_src, *p, RLF_WS_FIT, workspace, &ws) > ws_bytes) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = launch_prepare(*src, first, count, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                                   nullptr, *p, ws.table, ws.status, st);
    if (e == cudaSuccess) e = mlp_encode(facets, ws.table, count, p->facet_n, static_cast<__half *>(x_f16), st);
    return cuda_status(e);
}

rlf_status rlf_mlp_propose(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                           const rlf_params *p, const void *weights, int32_t *origin, int32_t *wide, void *workspace,
                           size_t ws_bytes, void *stream)
{
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    rlf_status s = check_src(src, first, count);
    if (s != RLF_OK) return s;
    if (!facets || !workspace || !weights || !origin) return RLF_EINVAL;
    if (p->facet_n * p->facet_n * 2 != kMlpIn || p->n_e < kBoxE || p->n_alpha < kBoxA) return RLF_EUNSUPPORTED;
    Workspace ws;
    if (workspace_layout(0, 1, src->n_src, *p, RLF_WS_FIT, workspace, &ws) > ws_bytes) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MlpScratch sc = mlp_scratch(ws.mlp_scratch, count);
    sc.status = ws.status;
    __half *x = static_cast<__half *>(ws.mlp_x);
    cudaError_t e = launch_prepare(*src, first, count, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr,
                                   nullptr, *p, ws.table, ws.status, st);
    if (e == cudaSuccess) e = mlp_encode(facets, ws.table, count, p->facet_n, x, st);
    if (e == cudaSuccess) e = mlp_forward(mlp_weights(const_cast<void *>(weights)), x, count, sc, st);
    if (e == cudaSuccess) e = mlp_propose(sc.o, count, grid_const(*p), origin, wide ? wide : ws.wide, st);
    return cuda_status(e);
}

rlf_status rlf_fit_sources_mlp(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                               const rlf_params *p, const void *weights, const rlf_fit_out *out,
                               int32_t *n_fallback, void *workspace, size_t ws_bytes, void *stream)
{
    if (!p || !params_ok(*p)) return RLF_EINVAL;
    rlf_status s = check_src(src, first, count);
    if (s != RLF_OK) return s;
    if (!facets || !workspace || !weights || !out || !out->e1 || !out->e2 || !out->sig1 || !out->sig2 ||
        !out->alpha_arcsec || !out->flux_jy || !out->e1_smooth || !out->e2_smooth || !out->flag)
        return RLF_EINVAL;
    if (p->facet_n * p->facet_n * 2 != kMlpIn || p->precision == RLF_PREC_FP64 || p->n_e < kBoxE ||
        p->n_alpha < kBoxA || n_offsets(*p) > 1)
        return RLF_EUNSUPPORTED;
    Workspace ws;
    if (workspace_layout(0, 1, src->n_src, *p, RLF_WS_FIT, workspace, &ws) > ws_bytes) return RLF_ENOSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess)
        e = launch_prepare(*src, first, count, src->e1, src->e2, nullptr, nullptr, nullptr, 0, nullptr, nullptr, *p,
                           ws.table, ws.status, st);
    if (e == cudaSuccess) e = launch_fit_mlp(facets, ws.table, count, *p, ws, weights, *out, n_fallback, st);
    return cuda_status(e);
}

rlf_status rlf_read_status(void *workspace, int32_t *status_out, void *stream)
{
    if (!workspace || !status_out) return RLF_EINVAL;
    Workspace ws;
    rlf_params p;
    rlf_params_default(&p);
    workspace_layout(0, 1, 1, p, RLF_WS_SKY, workspace, &ws);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ws.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return RLF_ECUDA;
    *status_out = v;
    if (v & RLF_DEV_TIMEOUT) return RLF_ETIMEOUT;
    if (v & RLF_DEV_NONFINITE) return RLF_ENUMERIC;
    return RLF_OK;
}

}  // extern "C"
