// Internal declarations shared by the CUDA translation units of the library.
// Nothing here is part of the C ABI (include/rlf.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/rlf.h"

namespace rlf {

constexpr double kC = 299792458.0;                      // speed of light, m/s
constexpr double kPi = 3.14159265358979323846;
constexpr double kArcsec = kPi / 648000.0;               // arcsec -> rad
constexpr int kThreads = 256;                            // threads per CTA of every kernel
constexpr int kMaxFitParts = 4;                          // cell parts per facet in a persistent fit
constexpr int kOrderBuckets = 512;                       // extent buckets of the baseline ordering
constexpr int kOrderThreads = 256;
constexpr int kSkyTile = 128;                            // sources staged per shared-memory tile
constexpr int kCellTile = 128;                           // facet cells staged per tile in the fit
constexpr int kMaxNe = 32;                               // grid nodes per e component (estimator smem)
constexpr int kAdaptSide = 17, kAdaptMax = kAdaptSide * kAdaptSide;  // adaptive lattice: per component, samples
constexpr int kAdaptRanks = 4;                           // partial sums per sample in the clustered adaptive sampler
// adaptive-sampling scratch per facet (doubles): ln L, a, b per (sample, alpha) of two
// levels; the cluster ranks' partial a, b; the lattice; the samples to evaluate (int);
// control words
__host__ __device__ inline size_t adapt_doubles_per_facet(int n_alpha)
{
    return (size_t)kAdaptMax * n_alpha * (6 + 2 * kAdaptRanks) + 2 * kAdaptMax + (kAdaptMax + 1) / 2 + 8;
}
constexpr int kMaxPartials = 8192;                       // (source, part) partial facets per extraction batch
constexpr int kPartialsPerSource = 64;                  // workspace partials per source below kMaxPartials

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
    int32_t profile;        // RLF_PROFILE_EXPONENTIAL or RLF_PROFILE_GAUSSIAN
    int32_t pad;
    double s0, ds;          // nu / c of channel 0 and its step, 1/m
    double spec_off;        // mean spectral factor: FP32 sums accumulate spec - spec_off
    double s[RLF_MAX_CHAN];     // nu_k / c (host division, the value the cell index uses)
    double spec[RLF_MAX_CHAN];  // (nu_k / nu_ref)^beta
    float s_hi[RLF_MAX_CHAN], s_lo[RLF_MAX_CHAN];  // s as a float pair, s_hi + s_lo
    float ds_hi, ds_lo;                             // ds as a float pair
};

// ---- error-free FP32 transformations (float-float arithmetic) -------------------------
// A value carried as hi + lo with |lo| <= ulp(hi)/2 has about 48 significant bits.
// two_prod: a * b = p + e exactly (FMA residual).  two_sum: a + b = s + e exactly
// (Knuth).  The __f*_rn intrinsics are never contracted or reassociated.

__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// phase argument u l + v m + w (n - 1) in metres as P + E, from float-pair inputs.
// Products are exact (two_prod); the cross terms hi*lo carry about 2^-24 of the
// product and are summed in FP32; lo*lo terms (2^-48 of the product) are dropped.
__device__ __forceinline__ void phase_metres(float uh, float ul, float vh, float vl, float wh, float wl,
                                             float lh, float ll, float mh, float ml, float nh, float nl,
                                             float &P, float &E)
{
    float p1, e1, p2, e2, p3, e3;
    two_prod(uh, lh, p1, e1);
    two_prod(vh, mh, p2, e2);
    two_prod(wh, nh, p3, e3);
    const float cross = fmaf(uh, ll, ul * lh) + fmaf(vh, ml, vl * mh) + fmaf(wh, nl, wl * nh);
    float s12, t12, t;
    two_sum(p1, p2, s12, t12);
    two_sum(s12, p3, P, t);
    E = ((e1 + e2) + e3) + (t12 + t) + cross;
}

// fractional part in [-1/2, 1/2] of (P + E) * (sh + sl) cycles
__device__ __forceinline__ float frac_cycles(float P, float E, float sh, float sl)
{
    float q, eq;
    two_prod(P, sh, q, eq);
    const float r = __fsub_rn(q, rintf(q));          // exact
    const float f = r + (eq + fmaf(P, sl, E * sh));
    return f - rintf(f);
}

// ---- the source profile's brightness factor (Eq. 1) -------------------------------------
// From qs = 4 pi^2 alpha^2 |A^{-T} k|^2 (the source's quadratic form times s^2):
//   exponential disc (1 + qs)^{-3/2};
//   Gaussian exp(-2 pi^2 sigma^2 |A^{-T} k|^2) with sigma^2 = alpha^2 ln 2 / 2 (the FWHM of
//   the exponential of scalelength alpha), i.e. 2^{-qs/4}.
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// q = the quadratic form in metres^2, f2 = s^2 (one FMA or two multiplies, one MUFU)
template <bool kGauss>
__device__ __forceinline__ float brightness(float q, float f2)
{
    if (kGauss) return ex2_approx(-0.25f * q * f2);
    const float r = rsqrtf(fmaf(q, f2, 1.0f));
    return r * r * r;
}

__device__ __forceinline__ double brightness64(double qs, int profile)
{
    if (profile == RLF_PROFILE_GAUSSIAN) return exp2(-0.25 * qs);
    const double x = 1.0 + qs;
    return 1.0 / (x * sqrt(x));
}

// ---- paired FP32 arithmetic (Blackwell f32x2 instructions) ----------------------------
// Two floats in one 64-bit register pair; one instruction issues both lanes.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float a, float b)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ void up2(f32x2 v, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// brightness() of two channels: q broadcast, f2 per channel
template <bool kGauss>
__device__ __forceinline__ f32x2 brightness2(f32x2 q2, f32x2 f2)
{
    float x0, x1;
    if (kGauss) {
        up2(mul2(mul2(pk2(-0.25f, -0.25f), q2), f2), x0, x1);
        return pk2(ex2_approx(x0), ex2_approx(x1));
    }
    up2(fma2(q2, f2, pk2(1.0f, 1.0f)), x0, x1);
    const f32x2 r = pk2(rsqrtf(x0), rsqrtf(x1));
    return mul2(mul2(r, r), r);
}

__device__ __forceinline__ void split_double(double x, float &hi, float &lo)
{
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

constexpr int kBoxE = 7, kBoxA = 5;                     // learned-proposal sub-box (e1, e2, alpha nodes)
constexpr int kMlpIn = 8192, kMlpHidden = 256, kMlpOut = 6, kMlpOutPad = 8;

// Position offsets of the likelihood's position marginal (Sec. 2.4): n_pos^2, 1 when
// the position is exact.
inline int n_offsets(const rlf_params &p)
{
    return p.n_pos > 1 ? p.n_pos * p.n_pos : 1;
}

// Values per cell of the compacted B block: one plane when the position is exact, else
// the offsets' B of each cell side by side, padded to whole 16-byte FP32 vectors.
__host__ __device__ inline int b_stride(int n_offsets)
{
    return n_offsets > 1 ? (n_offsets + 3) / 4 * 4 : 1;
}

// Grid constants of the likelihood (Sec. 2.4).
struct GridConst {
    const int32_t *box;     // per-facet sub-box origins [count][3] (e1, e2, alpha node), or null: full grid
    int32_t n_e, n_alpha, n_ag, flux_prior;
    int32_t profile, n_pos; // n_pos: position offsets per axis (1: position exact)
    double pos_step;        // position offset step, radians
    int32_t estimator, np_max;
    double e_res;
    double e_max;
    double r_min, r_max;    // arcsec
    double r_std;
    double inv_sigma2;      // 1 / sigma^2
    double thresh_frac, var_sigma_min, var_det_min;
    int32_t split;          // RLF_PREC_MIXED_SPLIT: FP32 tile sums added to float pairs, FP32 logarithms,
                            // error functions and exponentials in the estimate; otherwise (FP32 kernels of
                            // RLF_PREC_MIXED) tile sums added in FP64 and the estimate in FP64
    int32_t pad_;
    int32_t *box_fail;      // sub-box fits: set to 1 for a facet whose box cannot stand for the full grid
};

// FP64 accumulation in the registers of a float pair: the pair holds the two 32-bit halves
// of a double (no extra registers beside the float-pair form of the same kernels).
__device__ __forceinline__ double pair_as_double(float hi, float lo)
{
    return __hiloint2double(__float_as_int(hi), __float_as_int(lo));
}

__device__ __forceinline__ void double_to_pair(double d, float &hi, float &lo)
{
    hi = __int_as_float(__double2hiint(d));
    lo = __int_as_float(__double2loint(d));
}

// Add x to an accumulator held in (hi, lo): a float pair (hi + lo, error-free two-sum,
// about 48 significant bits) when `split`, else a double stored in the two registers.
__device__ __forceinline__ void acc_add(bool split, float &hi, float &lo, float x)
{
    if (split) {
        float sum, err;
        two_sum(hi, x, sum, err);
        hi = sum;
        lo = __fadd_rn(lo, err);
    } else {
        double_to_pair(pair_as_double(hi, lo) + (double)x, hi, lo);
    }
}

__device__ __forceinline__ double acc_value(bool split, float hi, float lo)
{
    return split ? (double)hi + (double)lo : pair_as_double(hi, lo);
}

// Carve-up of the caller's workspace.
struct Workspace {
    int32_t *status;        // [64] device status words
    SrcRow *table;          // [n_src]
    SrcRow *upd;            // [n_src] update table
    void *cells;            // T: planes uu, uv, vv, A [4][cap][N*N], then B [cap][N*N][b_stride]
    int32_t *ncell;         // [cap]
    int32_t *order;         // [cap] facets in largest-first order
    int32_t *counters;      // [cap + 1] work-item counter, per-facet finished tiles
    int32_t *box;           // [cap][3] learned-proposal sub-box origins
    int32_t *wide;          // [cap] proposal too wide: full grid
    int32_t *map_index;     // [cap] flat grid index of each facet's MAP point
    int32_t *refit;         // [cap + 1] facets to refit on the full grid, count first
    void *mlp_x;            // [cap][8192] f16 network inputs
    void *mlp_scratch;      // network activations for cap facets
    double *cc;             // [cap]
    double *ga, *gb;        // [fit_parts][cap][n_e^2][n_alpha] per-part likelihood sums
    size_t part_stride;     // cap * n_e^2 * n_alpha
    int32_t fit_parts;      // cell parts per facet the grids hold (kMaxFitParts; 16 when cap <= 16)
    double *gl;             // [cap][n_e^2][n_alpha]
    double *adapt;          // adaptive sampling: [cap][289][n_alpha][3] log-likelihood, a, b
    int32_t *bad_list;      // refit pass: [n_src + 1] count, then the bad fits in source order
    double *fit_tmp;        // refit pass: [8][cap] results of a refit chunk (FP64 fields)
    int32_t *flag_tmp;      // refit pass: [cap] flags of a refit chunk
    double *e_cur;          // [2][n_src]
    double *facets;         // [chunk][4][N*N]
    float *uvw_split;       // [n_rows][8]: uh, ul, vh, vl, wh, wl, 0, 0 (u, v, w as float pairs; split mode)
    float *resid;           // [n_rows][n_chan][2]: D - V_sky for batched extraction
    float *partial;         // [n_partials][4][N*N]: per-CTA partial facets of the extraction
    int32_t n_partials;     // min(kMaxPartials, 64 n_src)
    float *extent;          // [n_rows] per baseline: min over time of max(|u|, |v|), rounded down
    int32_t *perm;          // [n_rows] baselines in increasing order of extent (first n_baselines used)
    int32_t *n_live;        // [n_src] per source of an extraction batch: baselines to walk
    int32_t *order_counts;  // [kOrderBuckets][kOrderThreads] scratch of the ordering
    size_t bytes;
};

size_t workspace_layout(int64_t n_rows, int32_t n_chan, int32_t n_src, const rlf_params &p,
                        int32_t which, void *base, Workspace *ws);

// Host-side argument checks shared by every entry point (api.cu): the parameters, the
// observation and a source range; and the channel table of a call.
bool params_ok(const rlf_params &p);
rlf_status check_uvw(const rlf_uvw *uvw);
rlf_status check_src(const rlf_sources *src, int32_t first, int32_t count);
ChanTable make_chan_table(const rlf_uvw &uvw, const rlf_params &p);

// launchers (return cudaGetLastError())
cudaError_t launch_prepare(const rlf_sources &src, int32_t first, int32_t count,
                           const double *e1, const double *e2, const double *e1n,
                           const double *e2n, const int32_t *flag, int32_t update_mode,
                           double *e1_commit, double *e2_commit,
                           const rlf_params &p, SrcRow *out, int32_t *status, cudaStream_t st,
                           const int32_t *list = nullptr);
// Split-baseline records of a call (split mode): record i = {uh, ul, vh, vl, wh, wl, 0, 0}
// of row (i / stride) * stride + perm[i % stride] (perm set), else of row i.  rec null:
// the sky kernels split u, v, w on the fly.
struct SplitRows {
    const float *rec = nullptr;
    const int32_t *perm = nullptr;
    int32_t stride = 1;
};
SplitRows split_rows(const rlf_uvw &uvw, const rlf_params &p, const Workspace &ws);
// split records of every row in row order (no baseline order), for the standalone sky calls
cudaError_t launch_split_uvw(const rlf_uvw &uvw, float *out, cudaStream_t st);
cudaError_t launch_sky(const rlf_uvw &uvw, const ChanTable &ch, const SrcRow *table, int32_t n_src,
                       bool update, int32_t precision, float *vis, cudaStream_t st,
                       int32_t blocks_per_sm = 0, float sign = 1.0f, const SplitRows &sr = SplitRows());
// out = a - b over n4 float4 (the residual D - V, or the sky model D - R)
cudaError_t launch_difference(const float *a, const float *b, int64_t n_complex, float *out, cudaStream_t st);
// Per call, before the extraction batches: each baseline's smallest uv extent over
// time, the baselines ordered by it, and (split-phase mode) the split baselines in
// that order.
cudaError_t launch_extract_prepare(const rlf_uvw &uvw, const rlf_params &p, const Workspace &ws, cudaStream_t st);
cudaError_t launch_extract(const rlf_uvw &uvw, const ChanTable &ch, const float *data,
                           const float *sky, const SrcRow *table, int32_t count,
                           const rlf_params &p, const Workspace &ws, double *facets, cudaStream_t st);
// refit pass: the bad fits in source order (list[0] = count), results scattered back
cudaError_t launch_bad_list(const int32_t *flag, int32_t n, int32_t *list, cudaStream_t st);
cudaError_t launch_scatter(const double *tmp, const int32_t *ftmp, size_t cap, const int32_t *list, int32_t cnt,
                           const rlf_fit_out &out, cudaStream_t st);
cudaError_t launch_fit(const double *facets, const SrcRow *table, int32_t count,
                       const rlf_params &p, const Workspace &ws, const rlf_fit_out &out,
                       int32_t out_offset, cudaStream_t st);
GridConst grid_const(const rlf_params &p);
// learned-proposal fit: compaction, network, sub-box fit, refit of the facets that need the full grid
cudaError_t launch_fit_mlp(const double *facets, const SrcRow *table, int32_t count, const rlf_params &p,
                           const Workspace &ws, const void *weights, const rlf_fit_out &out, int32_t *n_fallback,
                           cudaStream_t st);

// ---- learned proposal (mlp.cu) ---------------------------------------------------------
struct MlpOffsets {
    int64_t W1, b1, W2, b2, W3, b3, P;   // f32 parameter offsets (W3 padded to 8 columns)
    int64_t W1h_n, W2h_n, W3h_n;         // f16 copies of the weight matrices, in that order
};
struct MlpWeights {
    float *w, *m, *v, *g;                // parameters, Adam moments, gradients [P]
    __half *h;                           // f16 W1 | W2 | W3
};
struct MlpScratch {
    __half *h1, *h2, *g16, *dz2, *dz1;
    float *o, *g32;
    float *part;            // split-K partial sums of the first layer
    __half *w1t;            // W1 transposed, [256][8192] (the tensor-core GEMM's K-major B)
    __half *xT, *dzT;       // x and dz1 transposed, [8192][Bp] and [256][Bp] (the weight gradient's operands)
    int32_t *status;        // RLF_DEV_TIMEOUT from the tensor-core GEMM's bounded waits
    size_t bytes;
};
MlpOffsets mlp_offsets();
MlpWeights mlp_weights(void *blob);
size_t mlp_weights_bytes();
MlpScratch mlp_scratch(void *base, int32_t max_batch);
cudaError_t mlp_forward(const MlpWeights &W, const __half *x, int32_t B, const MlpScratch &s, cudaStream_t st);
// first layer on tcgen05 (mlp_umma.cu): part[z][m][n] over n_slices K slices; x and W1t
// 16-byte aligned; cudaErrorNotSupported, launching nothing, when the driver cannot
// encode their tensor maps
cudaError_t mlp_layer1_umma(const __half *x, int32_t M, const __half *W1h, __half *W1t, float *part, int32_t n_slices,
                            int32_t *status, cudaStream_t st);
// the batch padded for the weight-gradient GEMM's K (a multiple of 64)
inline int32_t mlp_batch_pad(int32_t B) { return (B + 63) / 64 * 64; }
// dW1 = x^T dz1 on tcgen05 (mlp_umma.cu), through transposed, zero-padded copies xT, dzT
cudaError_t mlp_dw1_umma(const __half *x, int32_t B, const __half *dz1, __half *xT, __half *dzT, float *dW1,
                         int32_t *status, cudaStream_t st);
cudaError_t mlp_train_step(const MlpWeights &W, const __half *x, const float *y, int32_t B, float lr, int32_t step,
                           float *loss, const MlpScratch &s, cudaStream_t st);
cudaError_t mlp_init(const MlpWeights &W, const float *z, cudaStream_t st);
cudaError_t mlp_encode(const double *facets, const SrcRow *table, int32_t count, int32_t N, __half *x,
                       cudaStream_t st);
cudaError_t mlp_simulate(const double *tmpl, int32_t n_tmpl, const rlf_params &p, const double *tflux,
                         const int32_t *tidx, const double *e1, const double *e2, const double *alpha_as,
                         const float *z, int32_t B, int32_t N, double sigma, __half *x, float *y, cudaStream_t st);
cudaError_t mlp_propose(const float *o, int32_t count, const GridConst &gc, int32_t *origin, int32_t *wide,
                        cudaStream_t st);

}  // namespace rlf
