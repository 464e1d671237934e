/*
 * rlf.h - C ABI of the GB300 (sm_103a) RadioLensfit hot path.
 *
 * The library implements the data-parallel core of RadioLensfit
 * (Rivi & Miller, arXiv 2203.14071):
 *   - the analytic sky model: the sum over the catalogue of the exponential-disk
 *     visibility of Eq. 1 with the shear matrix of Eq. 2 (Sec. 2.2);
 *   - per-source isolation of the residual visibilities, phase shift to the
 *     source and averaging into a facet of cell size 1/(K alpha) (Sec. 2.3);
 *   - the chi^2 likelihood of each facet on an (e1, e2, alpha) grid with the
 *     flux marginalised analytically and alpha numerically, reduced to the
 *     ellipticity estimate and its spread (Sec. 2.4), and the sky-model update
 *     with the measured shapes (Sec. 2.2, Sec. 3.1).
 *
 * Conventions shared by every entry point
 *   - Pointers documented as "device" point to GPU global memory owned by the
 *     caller; the library never frees them and never allocates device memory.
 *     Scratch space is the caller-provided workspace (see rlf_workspace_size).
 *   - Pointers documented as "host" point to ordinary CPU memory and are read
 *     before the call returns.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream).  Work is
 *     enqueued on it and the call returns without waiting for the GPU, except
 *     where noted.
 *   - Visibilities are complex64, stored as interleaved float pairs (re, im),
 *     row-major [n_rows][n_chan] (channel fastest), in Jy.
 *   - Argument errors found on the host return RLF_EINVAL / RLF_EUNSUPPORTED /
 *     RLF_ENOSPACE before anything is enqueued.  Per-source value errors
 *     (flux <= 0 or not finite, |e| >= 1, l^2 + m^2 >= 1) are found on the GPU:
 *     the source contributes nothing, its fit flag gets RLF_FLAG_INVALID and the
 *     workspace status word gets RLF_DEV_INVALID_SOURCE (read it with
 *     rlf_read_status).  A CUDA launch failure returns RLF_ECUDA.
 */
#ifndef RLF_H
#define RLF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RLF_OK = 0,
    RLF_EINVAL = 1,        /* null pointer, non-positive size, bad parameter */
    RLF_ECUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    RLF_ENOSPACE = 3,      /* workspace or facet buffer smaller than required */
    RLF_ETIMEOUT = 4,      /* a bounded device wait gave up (status word); reserved: no entry
                              point of this version waits on the device */
    RLF_ENUMERIC = 5,      /* a non-finite likelihood was produced (status word) */
    RLF_EUNSUPPORTED = 6   /* valid request outside the implemented limits */
} rlf_status;

/* arithmetic of the path */
enum {
    RLF_PREC_FP64 = 0,     /* every step in double precision */
    RLF_PREC_MIXED = 1,    /* FP32 model and FP32 sums of products over tiles of at most 128
                              cells (likelihood) or one run of visibilities (facets); FP64 phase
                              argument and its range reduction, cell-index decisions, the
                              accumulation of the likelihood's tile sums a and b, the
                              log-likelihood (logarithms, error functions) and the alpha
                              marginal and its normalisation */
    RLF_PREC_MIXED_SPLIT = 2 /* FP32 model and tile sums as in RLF_PREC_MIXED, but the phase
                              argument and its range reduction, and the accumulation of the
                              tile sums a and b, are carried as pairs of floats with error-free
                              FP32 products and sums (about 48 significant bits), and the
                              estimate takes its logarithms, error functions and exponentials
                              (values of order one) in FP32 while the terms that cancel at high
                              SNR, -C/2 + b^2/(2a), stay FP64; GB300 runs this at its FP32 rate
                              instead of its much lower FP64 rate.  Measured against the FP64
                              oracle on the 37M-visibility, 200-source workload: |de| <= 1e-6 at
                              SNR 10 */
};

/* estimator of the ellipticity from the likelihood (Sec. 2.4) */
enum {
    RLF_ESTIMATOR_GRID = 0,      /* threshold moments over the fixed (e1, e2) grid */
    RLF_ESTIMATOR_ADAPTIVE = 1   /* then, while fewer than np_max samples are kept, halved lattices
                                    around the kept samples down to a step of e_res; the
                                    estimate is the last lattice's.  The number of halvings is
                                    returned in bits 8-11 of the fit flag. */
};
#define RLF_FLAG_LEVELS_SHIFT 8

/* source brightness profile (Sec. 2.2 and its footnote); alpha keeps its meaning (grid,
   Eq. 4 prior, facet cell size) under both */
enum {
    RLF_PROFILE_EXPONENTIAL = 0, /* I(r) ~ exp(-r / alpha): (1 + 4 pi^2 alpha^2 |A^-T k|^2)^{-3/2} */
    RLF_PROFILE_GAUSSIAN = 1     /* I(r) ~ exp(-r^2 / (2 sigma^2)) of the same FWHM, sigma = alpha
                                    sqrt(ln 2 / 2): exp(-2 pi^2 sigma^2 |A^-T k|^2) */
};

/* bits of the per-source fit flag */
enum {
    RLF_FLAG_BAD = 1,      /* Sec. 4.1 cut: sigma(e_i) or sqrt(det cov) not above its minimum */
    RLF_FLAG_INVALID = 2,  /* the source's input values are out of range */
    RLF_FLAG_EMPTY = 4,    /* the facet holds no visibility */
    RLF_FLAG_REFIT = 8     /* rlf_run with refit_bad: fitted again after the whole catalogue */
};

/* bits of the device status word */
enum {
    RLF_DEV_INVALID_SOURCE = 1,
    RLF_DEV_NONFINITE = 2,
    RLF_DEV_TIMEOUT = 4    /* a bounded wait ran out: the proposal network's tensor-core GEMM
                              (rlf_mlp_propose, rlf_fit_sources_mlp; the results of the call
                              are then invalid; rlf_mlp_forward and rlf_mlp_train_step keep
                              the flag in their own scratch and do not report it) */
};

/* workspace users for rlf_workspace_size */
enum { RLF_WS_SKY = 0, RLF_WS_EXTRACT = 1, RLF_WS_FIT = 2, RLF_WS_RUN = 3 };

/* Largest channel count, row count and facet side handled by one call. */
#define RLF_MAX_CHAN 128
#define RLF_MAX_ROWS 2147483647
#define RLF_MAX_FACET_N 64
/* Largest position-offset grid side (rlf_params.n_pos). */
#define RLF_MAX_POS 5

/* Observation: baselines in metres (Sec. 2.2: (u, v, w) with w towards the phase centre). */
typedef struct {
    int64_t n_rows;          /* number of (baseline, time) rows, 1 .. RLF_MAX_ROWS */
    int32_t n_chan;          /* channels, 1 .. RLF_MAX_CHAN */
    int32_t n_baselines;     /* rows are time-major with this many baselines per time step
                                (the Measurement Set order); 0 if unknown.  Only speed
                                depends on it: extraction walks each baseline's time series */
    const double *u;         /* device [n_rows], metres */
    const double *v;         /* device [n_rows], metres */
    const double *w;         /* device [n_rows], metres */
    const double *freq_hz;   /* host [n_chan], channel centres, strictly increasing */
} rlf_uvw;

/* Catalogue (Sec. 2.1): ordered by decreasing flux or SNR by the caller. */
typedef struct {
    int32_t n_src;           /* > 0 */
    int32_t reserved;
    const double *l;         /* device [n_src], direction cosine */
    const double *m;         /* device [n_src], direction cosine */
    const double *flux_jy;   /* device [n_src], integrated flux at nu_ref, > 0 */
    const double *alpha_arcsec; /* device [n_src] catalogue scalelength, <= 0 entries (or a
                                   NULL pointer) use the Eq. 4 median for the flux */
    const double *e1;        /* device [n_src], shape currently in the sky model */
    const double *e2;        /* device [n_src] */
} rlf_sources;

/* Algorithm parameters; rlf_params_default gives the paper's values. */
typedef struct {
    double add, esp;         /* Eq. 4 intercept and slope (ADD = -0.93, ESP = 0.33) */
    double psf_nat;          /* facet field-of-view factor K (Sec. 2.3, K = 38 in Sec. 4.1) */
    double beta;             /* spectral index (-0.7, Sec. 2.2) */
    double nu_ref_hz;        /* reference frequency of the fluxes */
    double sigma_jy;         /* noise standard deviation per visibility component */
    double e_max;            /* grid e1, e2 in [-e_max, e_max] */
    double r_min_arcsec, r_max_arcsec; /* scalelength range [RMIN, RMAX] (Sec. 4.2) */
    double r_std;            /* log-normal prior width R_STD (Sec. 2.4) */
    double thresh_frac;      /* fraction of the maximum kept by the estimator (0.05) */
    double var_sigma_min;    /* bad fit if sigma(e_i) <= this (5e-3, Sec. 4.1) */
    double var_det_min;      /* bad fit if sqrt(det cov) <= this (5e-5, Sec. 4.1) */
    int32_t facet_n;         /* facet side in cells, even, 2 .. RLF_MAX_FACET_N */
    int32_t n_e;             /* grid nodes per ellipticity component, 2 .. 64 */
    int32_t n_alpha;         /* scalelength nodes, 1 .. 64 */
    int32_t flux_prior;      /* 0: uniform on S >= 0; 1: uniform on the real line */
    int32_t chunk;           /* sources per extract/fit/update step of rlf_run; <= 0: all */
    int32_t update_mode;     /* 0: update the sky model with good fits only; 1: with all */
    int32_t precision;       /* RLF_PREC_FP64, RLF_PREC_MIXED or RLF_PREC_MIXED_SPLIT */
    /* launch shapes (0: library default); rlf_autotune fills them by timing */
    int32_t tune_fit_ag;        /* scalelength nodes per likelihood thread: 2, 4 or 8 (default 4) */
    int32_t tune_fit_blocks;    /* CTAs per SM of the persistent fit (default: all that fit) */
    int32_t tune_extract_waves; /* CTA waves per extraction batch (default 2) */
    int32_t tune_sky_blocks;    /* CTAs per SM of the sky-model kernels (default 8) */
    int32_t profile;         /* source brightness profile: RLF_PROFILE_EXPONENTIAL (Eq. 1, the
                                default) or RLF_PROFILE_GAUSSIAN (footnote to Sec. 2.2) */
    double e_res;            /* adaptive sampling: finest step in e, E_RES (0.003, Sec. 2.4) */
    int32_t np_max;          /* adaptive sampling: kept samples that end it, NP_MAX (30, Sec. 2.4) */
    int32_t estimator;       /* RLF_ESTIMATOR_GRID (default) or RLF_ESTIMATOR_ADAPTIVE */
    int32_t refit_bad;       /* rlf_run: 1 = fit the bad fits again after every other source,
                                against the final sky model (Sec. 2.4) */
    int32_t n_pos;           /* position marginal (Sec. 2.4): offsets per axis, 1 (0 reads as 1:
                                the catalogue position is exact, the default), 3 or RLF_MAX_POS;
                                uniform prior over the n_pos x n_pos grid of offsets centred on the
                                catalogue position.  Not with rlf_fit_mlp (RLF_EUNSUPPORTED). */
    double pos_step_arcsec;  /* position marginal: offset step, > 0 (default 0.1") */
} rlf_params;

/* Per-source results, each a device array of `count` entries. */
typedef struct {
    double *e1, *e2;         /* likelihood-weighted mean over the kept grid points */
    double *sig1, *sig2;     /* their standard deviations */
    double *alpha_arcsec;    /* posterior mean scalelength over the kept points */
    double *flux_jy;         /* b/a at the maximum a posteriori grid point */
    double *e1_smooth, *e2_smooth; /* mean over every grid point (no threshold) */
    int32_t *flag;           /* RLF_FLAG_* bits */
} rlf_fit_out;

/* Fill *p with the paper's defaults: ADD, ESP, K = 38, beta = -0.7, RMIN 0.3",
 * RMAX 3.5", R_STD 0.3136, 5% threshold, 5e-3 / 5e-5 cuts, 21 x 21 e nodes on
 * [-0.8, 0.8], 20 alpha nodes, 64 x 64 facets, RLF_PREC_MIXED, chunk = all, the
 * exponential profile, the grid estimator, no refit, position exact (n_pos = 1,
 * pos_step_arcsec = 0.1). */
void rlf_params_default(rlf_params *p);

/* Bytes of workspace needed by entry point `which` (RLF_WS_*) for these sizes;
 * RLF_WS_RUN covers every entry point.  0 for invalid arguments. */
size_t rlf_workspace_size(int64_t n_rows, int32_t n_chan, int32_t n_src, const rlf_params *p,
                          int32_t which);

/* Bytes of a facet buffer holding `count` facets: count * 4 * facet_n^2 doubles. */
size_t rlf_facets_size(int32_t count, const rlf_params *p);

/*
 * Sky model, Sec. 2.2 (Eq. 1 summed over the catalogue, Eq. 2 shear):
 *   vis_sky[r, c] = sum_j (nu_c/nu_ref)^beta S_j (1 + 4 pi^2 alpha_j^2 |A_j^{-T} k|^2)^{-3/2}
 *                   * exp(2 pi i (u l_j + v m_j + w (n_j - 1)) nu_c / c)
 * with k = (u, v) nu_c / c, alpha_j the catalogue scalelength or the Eq. 4 median
 * and A_j built from the sources' current (e1, e2).  vis_sky (device
 * [n_rows][n_chan][2] float) is overwritten.
 */
rlf_status rlf_sky_model(const rlf_uvw *uvw, const rlf_sources *src, const rlf_params *p,
                         float *vis_sky, void *workspace, size_t ws_bytes, void *stream);

/*
 * Sky-model update, Sec. 2.2 and Sec. 3.1: for each source i in
 * [first, first + count) selected by update_mode (all, or flag[i - first] has no
 * RLF_FLAG_BAD / RLF_FLAG_INVALID / RLF_FLAG_EMPTY bit),
 *   vis_sky += model_i(e_new) - model_i(e_old)
 * where e_old is src->e1/e2 and e_new is e1_new/e2_new (device [count]).
 * flag (device [count]) may be NULL, which updates every source in the range.
 */
rlf_status rlf_sky_update(const rlf_uvw *uvw, const rlf_sources *src, int32_t first,
                          int32_t count, const double *e1_new, const double *e2_new,
                          const int32_t *flag, const rlf_params *p, float *vis_sky,
                          void *workspace, size_t ws_bytes, void *stream);

/*
 * Facet extraction, Sec. 2.3, for sources [first, first + count):
 *   x = (D - V_sky + model_i) exp(-2 pi i (u l_i + v m_i + w (n_i - 1)) nu / c)
 * averaged in cells of side du_i = 1 / (K alpha_i) wavelengths on a facet_n x
 * facet_n window centred on the origin; cell (iu, iv) = floor(k / du_i) + facet_n/2,
 * visibilities outside the window are dropped.  model_i uses the source's
 * current (e1, e2).  facets (device) receives, per source, 4 planes of
 * facet_n^2 doubles: sum Re x, sum Im x, count, sum (nu/nu_ref)^beta; cell
 * index iv * facet_n + iu.  facets_bytes must be >= rlf_facets_size(count, p).
 */
rlf_status rlf_extract_facets(const rlf_uvw *uvw, const float *vis_data, const float *vis_sky,
                              const rlf_sources *src, int32_t first, int32_t count,
                              const rlf_params *p, double *facets, size_t facets_bytes,
                              void *workspace, size_t ws_bytes, void *stream);

/*
 * Source fitting, Sec. 2.4, for the `count` facets in `facets` (sources
 * [first, first + count)).  With D_c = mean x, s_c = mean spectral factor and
 * w_c = n_c / sigma^2 per non-empty cell and M_c the Eq. 1 brightness factor at
 * the cell centre (w = 0):
 *   a = sum w_c s_c^2 M_c^2,  b = sum w_c s_c M_c Re D_c,  C = sum w_c |D_c|^2
 *   logL = -C/2 + b^2/(2a) + ln sqrt(pi/(2a)) + ln erfc(-b / sqrt(2a))
 * on e1, e2 nodes -e_max + k 2 e_max/(n_e - 1) with |e| < 1 and alpha nodes
 * RMIN + (RMAX - RMIN)(k/(n_alpha - 1))^2.  alpha is marginalised with
 * trapezoid weights and a log-normal prior (mean ln alpha from Eq. 4, width
 * R_STD); the e points at or above thresh_frac of the maximum give the mean and
 * spread; the Sec. 4.1 cut sets RLF_FLAG_BAD.  Results go to *out.
 * With p->n_pos > 1 the position is marginalised too (Sec. 2.4), with a uniform
 * prior over the offsets x_j = (i - h, k - h) pos_step_arcsec, h = (n_pos - 1)/2:
 * a source offset by x_j carries exp(2 pi i k.x_j) in its facet model, so a and C
 * are unchanged, b_j = sum w_c s_c M_c Re(D_c exp(-2 pi i k_c.x_j)), and logL is
 * the log of the mean over j of exp(logL(b_j)); flux_jy is b/a at the best offset
 * of the MAP point.
 */
rlf_status rlf_fit_sources(const double *facets, const rlf_sources *src, int32_t first,
                           int32_t count, const rlf_params *p, const rlf_fit_out *out,
                           void *workspace, size_t ws_bytes, void *stream);

/*
 * The whole chain, Sec. 2: circular sky model from the catalogue shapes in src
 * (normally zero), then for each chunk of p->chunk sources in catalogue order:
 * extract their facets from the current sky model, fit them, and replace their
 * shapes in the sky model (update_mode).  chunk = 1 is the serial order;
 * chunk = n_src extracts every facet from the initial model (Sec. 3.1).
 * vis_sky (device, [n_rows][n_chan][2]) ends holding the final sky model; out
 * holds n_src results.  The workspace must be rlf_workspace_size(..., RLF_WS_RUN).
 * With p->refit_bad = 1 the fits flagged bad are then fitted once more, in source
 * order and chunks of the same size, against the sky model that holds every other
 * measured shape (Sec. 2.4); their results replace the first ones and carry
 * RLF_FLAG_REFIT.  Their number sizes those launches, so rlf_run then synchronises
 * `stream` once.
 */
rlf_status rlf_run(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src,
                   const rlf_params *p, const rlf_fit_out *out, float *vis_sky,
                   void *workspace, size_t ws_bytes, void *stream);

/*
 * Learned proposal of the likelihood sub-grid.  An addition to the method: the
 * paper has no counterpart (its fit searches the likelihood with Nelder-Mead, Sec. 2.4).
 * A perceptron reads a facet (facet_n must be 64: x = [Re D_c / S, Im D_c / S],
 * 8192 values, empty cells 0, f16) and predicts (mu, logvar) of (e1, e2,
 * ln(alpha/arcsec)): h1 = relu(x W1 + b1) [256], h2 = relu(h1 W2 + b2) [256],
 * o = h2 W3 + b3 [8], o[0:3] = mu, o[3:6] = logvar, o[6:8] = 0.  Trained with the
 * Gaussian NLL (logvar clamped to [-8, 8]) and Adam (beta 0.9, 0.999, eps 1e-8).
 *
 * Weights blob (device, rlf_mlp_weights_size() bytes, caller-owned), with
 * P = rlf_mlp_n_params() and the parameter order W1 [8192][256], b1 [256],
 * W2 [256][256], b2 [256], W3 [256][8], b3 [8] (row-major, columns 6 and 7 of W3
 * zero): f32 params [P] | f32 Adam m [P] | f32 Adam v [P] | f32 gradients [P] |
 * f16 copies of W1, W2, W3 (used by the tensor-core GEMMs; the first layer's GEMM
 * transposes W1 into its scratch on every call).
 */
#define RLF_MLP_IN 8192
#define RLF_MLP_OUT 8
size_t rlf_mlp_weights_size(void);
int64_t rlf_mlp_n_params(void);
/* Scratch bytes for rlf_mlp_train_step / rlf_mlp_forward with up to max_batch facets. */
size_t rlf_mlp_workspace_size(int32_t max_batch);
/* He initialisation from P standard normals (device, e.g. from a seeded RNG); zero biases and moments. */
rlf_status rlf_mlp_init(void *weights, const float *normals, void *stream);
/*
 * Training facets from the likelihood's own facet model (Sec. 2.4): for sample b,
 * template t = tidx[b] (a facet [4][64*64] as from rlf_extract_facets, of flux
 * template_flux[t], cell size 1/(K alpha_med(flux)) by Eq. 4), every non-empty cell
 *   x_c = s_c M(k_c; e1[b], e2[b], alpha_arcsec[b]) + (sigma_jy / flux) z / sqrt(n_c)
 * with z = normals[b][0 or 1][c] (device [batch][2][4096] standard normals) for the
 * real and imaginary parts; y[b] = (e1, e2, ln alpha) (device [batch][3] f32).
 * x_f16: device [batch][8192] f16.
 */
rlf_status rlf_mlp_simulate(const double *templates, const double *template_flux, int32_t n_templates,
                            const int32_t *tidx, const double *e1, const double *e2, const double *alpha_arcsec,
                            const float *normals, int32_t batch, const rlf_params *p, void *x_f16, float *y,
                            void *stream);
/* One Adam step on a batch (x_f16 [batch][8192] and the weights blob 16-byte aligned, else
 * RLF_EINVAL; y [batch][3]); the first layer's forward GEMM and its weight gradient run
 * on tcgen05; step >= 1 is the Adam time
 * step (bias correction); step = 0 computes the gradients into the blob and leaves the
 * parameters unchanged.  loss (device f32, may be NULL) receives the batch NLL. */
rlf_status rlf_mlp_train_step(void *weights, const void *x_f16, const float *y, int32_t batch, float lr,
                              int32_t step, float *loss, void *workspace, size_t ws_bytes, void *stream);
/* out (device [batch][8] f32): the network's outputs for x_f16 (16-byte aligned, else
 * RLF_EINVAL).  The first layer runs on tcgen05 (TMA-staged f16 operands, f32
 * accumulators in TMEM), the others on mma.sync. */
rlf_status rlf_mlp_forward(const void *weights, const void *x_f16, int32_t batch, float *out, void *workspace,
                           size_t ws_bytes, void *stream);
/* Network inputs (device [count][8192] f16) of facets [count][4][64*64] of sources
 * [first, first + count).  Workspace: rlf_workspace_size(..., RLF_WS_FIT). */
rlf_status rlf_mlp_encode(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                          const rlf_params *p, void *x_f16, void *workspace, size_t ws_bytes, void *stream);
/*
 * The network's proposal alone: for the `count` facets [count][4][64*64] of sources
 * [first, first + count), origin (device [count][3] int32) receives the (e1 node, e2
 * node, alpha node) origin of the 7 x 7 x 5 box of grid nodes centred on the node
 * nearest the predicted mean (clamped inside the grid), and wide (device [count]
 * int32, may be NULL) 1 where the predicted spread of e1 or e2 exceeds three node
 * spacings (the full grid is then needed), else 0.  Requires facet_n = 64, n_e >= 7
 * and n_alpha >= 5.  Workspace: rlf_workspace_size(..., RLF_WS_FIT).  The paper has no
 * counterpart (its fit searches the likelihood with Nelder-Mead, Sec. 2.4).
 */
rlf_status rlf_mlp_propose(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                           const rlf_params *p, const void *weights, int32_t *origin, int32_t *wide, void *workspace,
                           size_t ws_bytes, void *stream);

/*
 * rlf_fit_sources on a narrowed grid: the network proposes each facet's 7 x 7 x 5
 * box of grid nodes centred on the node nearest mu (clamped inside the grid); the
 * likelihood and the estimate are computed on the box only (alpha quadrature on the
 * box's nodes, points outside the box excluded).  A facet is refitted on the full
 * grid when the predicted spread of e1 or e2 exceeds three node spacings, when its
 * box MAP point lies on a face of the box that is not a face of the grid (an inner
 * face), or when a box point whose alpha marginal L(e) reaches half the estimate's
 * threshold (thresh_frac max L / 2) lies on an inner e face or has, at an inner alpha
 * face, an alpha-profile term above 1e-6 L(e).  The refitted facets' results are the
 * full grid's; the others' thresholded estimate (e1, e2, sig1, sig2, alpha, flux, flag)
 * is the full grid's up to the alpha tail so bounded, while e1_smooth/e2_smooth cover
 * the box's points only.
 * n_fallback (device int32, may be NULL) receives the number of refitted facets.
 * Requires facet_n = 64, a mixed precision mode, n_e >= 7 and n_alpha >= 5.
 */
rlf_status rlf_fit_sources_mlp(const double *facets, const rlf_sources *src, int32_t first, int32_t count,
                               const rlf_params *p, const void *weights, const rlf_fit_out *out,
                               int32_t *n_fallback, void *workspace, size_t ws_bytes, void *stream);

/*
 * The whole chain as a captured CUDA graph (the batched form: one graph holds the
 * sky model, every extraction, the persistent fit and the update; with chunk =
 * n_src that is one launch per step).  rlf_graph_create records rlf_run's work on
 * `stream` (a non-default cudaStream_t, required) into a graph and instantiates it;
 * every pointer, size, parameter and host channel value is baked in, so later
 * launches recompute the chain on the current contents of the same buffers.
 * rlf_graph_launch enqueues one replay on `stream`.  The graph object is host
 * memory owned by the library; free it with rlf_graph_destroy.  Sec. 2 and Sec. 3.1
 * define the chain; the graph is an execution form, not a change of the method.
 * p->refit_bad = 1 is not capturable (RLF_EUNSUPPORTED).
 */
typedef struct rlf_graph_s rlf_graph;
rlf_status rlf_graph_create(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src,
                            const rlf_params *p, const rlf_fit_out *out, float *vis_sky, void *workspace,
                            size_t ws_bytes, void *stream, rlf_graph **graph_out);
rlf_status rlf_graph_launch(rlf_graph *graph, void *stream);
void rlf_graph_destroy(rlf_graph *graph);

/*
 * Autotuner of the launch shapes (the tune_* fields of rlf_params) for this
 * workload: times the sky model over CTAs per SM {8, 16, 32, 64}, the extraction
 * of the first chunk over {1, 2, 3, 4, 6, 8, 12, 16} CTA waves, and the persistent fit over
 * scalelength nodes per thread {2, 4, 8} x CTAs per SM {1, 2, 3} (median of 3
 * runs each, CUDA events on `stream`), and writes the fastest choices into *p.
 * Arguments as for rlf_run; vis_sky, out and the workspace are overwritten.
 * phase_ms (host [3], may be NULL) receives the best sky, extraction and fit
 * times.  Waits for `stream`.  The results depend on these fields only through the
 * rounding of the extraction's partial sums (their grouping follows the wave count).
 */
rlf_status rlf_autotune(const rlf_uvw *uvw, const float *vis_data, const rlf_sources *src, rlf_params *p,
                        const rlf_fit_out *out, float *vis_sky, void *workspace, size_t ws_bytes, void *stream,
                        float *phase_ms);

/*
 * Sky model without any caller-provided device memory.  There is no counterpart
 * in the paper: it is the same computation as rlf_sky_model for callers that
 * cannot allocate device memory (code running where cudaMalloc is not allowed or
 * not wanted, e.g. inside another framework's memory pool, a real-time loop that
 * must not allocate after start-up, or a plugin handed only its input and output
 * buffers).  The per-source table that rlf_sky_model keeps in the workspace lives
 * here in a fixed device array inside the library (about 460 KB on every GPU that
 * loads the library, held until the process exits).
 *   - At most RLF_STATIC_MAX_SRC sources; more returns RLF_ENOSPACE and enqueues
 *     nothing.  Other arguments as for rlf_sky_model, checked the same way.
 *   - The first call on a device looks up the array's device address (once per
 *     device, with that device current); make that first call before any stream
 *     capture.  The address is kept for the life of the process: do not use this
 *     entry point across a cudaDeviceReset.
 *   - The launch shape follows p->tune_sky_blocks as in rlf_sky_model.  In
 *     RLF_PREC_MIXED_SPLIT each row's float-pair phase is formed on the fly (there is
 *     no workspace for the split-baseline records rlf_sky_model writes first); the
 *     result is the same to FP32 rounding.
 *   - Calls share the array: calls that overlap on the GPU (other streams, or
 *     other host threads without ordering) race on it.  Each call rewrites what it
 *     reads, so earlier contents do not matter.
 *   - Per-source value errors are not reported (there is no workspace status to
 *     read): such sources contribute nothing, as in rlf_sky_model.
 * Never calls cudaMalloc, cudaFree or any allocating routine.
 */
#define RLF_STATIC_MAX_SRC 4096
rlf_status rlf_sky_model_static(const rlf_uvw *uvw, const rlf_sources *src, const rlf_params *p,
                                float *vis_sky, void *stream);

/* Copy the workspace's device status word (RLF_DEV_* bits) to *status_out and clear it.
 * Waits for `stream`.  Returns RLF_ETIMEOUT / RLF_ENUMERIC when those bits are set. */
rlf_status rlf_read_status(void *workspace, int32_t *status_out, void *stream);

/* Static text for a status code. */
const char *rlf_strerror(rlf_status s);

#ifdef __cplusplus
}
#endif

#endif /* RLF_H */
