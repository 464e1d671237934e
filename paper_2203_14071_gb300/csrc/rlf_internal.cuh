// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/rlf.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/rlf.h"

namespace rlf {

constexpr double kC = 299792458.0;                      // speed of light, m/s
constexpr double kPi = 3.14159265358979323846;
constexpr double kArcsec = kPi / 648000.0;               // arcsec -> rad
constexpr int kThreads = 256;                            // threads per CTA of every kernel
constexpr int kSkyTile = 128;                            // sources staged per shared-memory tile
constexpr int kCellTile = 128;                           // facet cells staged per tile in the fit
constexpr int kAlphaPerThread = 4;                       // scalelength nodes per fit thread
constexpr int kMaxNe = 32;                               // grid nodes per e component (estimator smem)

// Per-source constants derived on the device from the catalogue (Sec. 2.2, 2.3).
struct SrcRow {
    double l, m, n1;        // direction cosines and n - 1
    double flux;            // S (0 when the source is not used)
    double alpha_rad;       // scalelength of the sky model and of the facet size
    double du;              // facet cell side in wavelengths, 1 / (K alpha)
    double mu;              // ln(alpha_med / arcsec) from Eq. 4, prior mean
    double q[3];            // 4 pi^2 alpha^2 |A^{-T} k|^2 = q0 u^2 + q1 u v + q2 v^2 (k = (u, v) nu / c)
    double qn[3];           // the same for the updated shape (sky update only)
    int32_t invalid;        // input values out of range
    int32_t pad;
};

// Channel constants, passed by value (fits the 4 KB kernel-parameter space).
struct ChanTable {
    int32_t n;              // channels
    int32_t uniform;        // s[k] = s0 + k ds to 1e-12 relative
    double s0, ds;          // nu / c of channel 0 and its step, 1/m
    double s[RLF_MAX_CHAN];     // nu_k / c (host division, the value the cell index uses)
    double spec[RLF_MAX_CHAN];  // (nu_k / nu_ref)^beta
};

// Grid constants of the likelihood (Sec. 2.4).
struct GridConst {
    int32_t n_e, n_alpha, n_ag, flux_prior;
    double e_max;
    double r_min, r_max;    // arcsec
    double r_std;
    double inv_sigma2;      // 1 / sigma^2
    double thresh_frac, var_sigma_min, var_det_min;
};

// Carve-up of the caller's workspace.
struct Workspace {
    int32_t *status;        // [64] device status words
    SrcRow *table;          // [n_src]
    SrcRow *upd;            // [n_src] update table
    void *cells;            // [5][cap][N*N] T
    int32_t *ncell;         // [cap]
    double *cc;             // [cap]
    double *ga, *gb, *gl;   // [cap][n_e^2][n_alpha]
    double *e_cur;          // [2][n_src]
    double *facets;         // [chunk][4][N*N]
    size_t bytes;
};

size_t workspace_layout(int64_t n_rows, int32_t n_chan, int32_t n_src, const rlf_params &p,
                        int32_t which, void *base, Workspace *ws);

// launchers (return cudaGetLastError())
cudaError_t launch_prepare(const rlf_sources &src, int32_t first, int32_t count,
                           const double *e1, const double *e2, const double *e1n,
                           const double *e2n, const int32_t *flag, int32_t update_mode,
                           double *e1_commit, double *e2_commit,
                           const rlf_params &p, SrcRow *out, int32_t *status, cudaStream_t st);
cudaError_t launch_sky(const rlf_uvw &uvw, const ChanTable &ch, const SrcRow *table, int32_t n_src,
                       bool update, int32_t precision, float *vis, cudaStream_t st);
cudaError_t launch_extract(const rlf_uvw &uvw, const ChanTable &ch, const float *data,
                           const float *sky, const SrcRow *table, int32_t count,
                           const rlf_params &p, double *facets, cudaStream_t st);
cudaError_t launch_fit(const double *facets, const SrcRow *table, int32_t count,
                       const rlf_params &p, const Workspace &ws, const rlf_fit_out &out,
                       int32_t out_offset, cudaStream_t st);

}  // namespace rlf
