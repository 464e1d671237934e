// Source fitting (Sec. 2.4): facet compaction, the likelihood grid over
// (e1, e2, alpha) with the flux marginalised analytically, the numerical alpha
// marginal and the thresholded estimate with the bad-fit cut of Sec. 4.1.
//
//   compact_kernel    one CTA per facet: the non-empty cells in increasing cell
//                     order, as (uu, uv, vv) in units of du^2 (exact for the
//                     half-integer cell centres), A = w s^2, B = w s Re D (with the
//                     position marginal one B per offset, side by side), and
//                     C = sum w |D|^2 in FP64.
//   fit_persistent_kernel  one launch for every facet: CTAs take work items
//                     (facet in largest-first order, tile of grid pairs) from an
//                     atomic counter; the CTA finishing a facet's last tile runs its
//                     estimate (fused tail).
//   grid_tile         work item = (facet, tile of (e point, alpha group)); cells are
//                     staged through shared memory; each thread evaluates its
//                     alpha nodes for every cell: one quadratic form per cell,
//                     then per alpha one FMA, one rsqrt and the a, b products.
//                     Mixed precision sums the products in FP32 over a tile of
//                     cells and adds the tile sums to FP64 accumulators
//                     (RLF_PREC_MIXED) or float pairs (RLF_PREC_MIXED_SPLIT); two
//                     scalelength nodes share each paired (f32x2) instruction.
//   estimate_source   one CTA per facet: logL, alpha marginal, threshold,
//                     moments, MAP point, flags; FP64 throughout except the
//                     logarithms, error functions and exponentials of split mode.
//   fit_persistent_pos_kernel / grid_tile_pos, grid_tile_posn   the grid with the
//                     position marginal (Sec. 2.4): one (e, alpha) point per thread
//                     (FP64, n_pos 5) or three alpha nodes of one e point (FP32, n_pos
//                     3), every offset's b, the marginal over offsets in the epilogue.
//   adaptive_cluster_kernel / adaptive_kernel   adaptive sampling around the maximum
//                     (Sec. 2.4) after the grid fit: halved lattices, a cluster of four
//                     CTAs per facet (FP32, one position) or one CTA per facet.
#include <cooperative_groups.h>

#include <cfloat>
#include <cmath>
#include <type_traits>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

template <typename T>
__global__ void __launch_bounds__(kThreads)
compact_kernel(const double *__restrict__ facets, const SrcRow *__restrict__ table, int32_t N,
               double inv_sigma2, int32_t n_pos, double pos_step, size_t plane, T *__restrict__ cells,
               int32_t *__restrict__ ncell, double *__restrict__ cc_out)
{
    __shared__ int32_t warp_tot[kThreads / 32];
    __shared__ double warp_cc[kThreads / 32];
    const int s = blockIdx.x;
    const int NN = N * N;
    const double *f = facets + (size_t)s * 4 * NN;
    const int per = (NN + kThreads - 1) / kThreads;
    const int c0 = threadIdx.x * per;
    int mine = 0;
    double cc = 0.0;
    for (int i = 0; i < per; ++i) {
        const int c = c0 + i;
        if (c < NN && f[2 * NN + c] > 0.0) {
            ++mine;
            const double n = f[2 * NN + c], in = 1.0 / n;
            const double dr = f[c] * in, di = f[NN + c] * in;
            cc += n * inv_sigma2 * (dr * dr + di * di);
        }
    }
    // exclusive scan of the per-thread counts (warp shuffles, then the warp totals)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    double ccw = cc;
    for (int o = 16; o > 0; o >>= 1) ccw += __shfl_down_sync(0xffffffffu, ccw, o);
    if (lane == 31) warp_tot[wid] = incl;
    if (lane == 0) warp_cc[wid] = ccw;
    __syncthreads();
    int base = 0;
    for (int i = 0; i < wid; ++i) base += warp_tot[i];
    int pos = base + incl - mine;
    const double du = table[s].du;
    const int nj = n_pos > 1 ? n_pos * n_pos : 1;
    const int h = (n_pos - 1) / 2;
    T *uu = cells + (size_t)s * NN;
    T *uv = uu + plane;
    T *vv = uv + plane;
    T *A = vv + plane;
    T *B = A + plane;
    for (int i = 0; i < per; ++i) {
        const int c = c0 + i;
        if (c < NN && f[2 * NN + c] > 0.0) {
            const double n = f[2 * NN + c], in = 1.0 / n;
            const double dr = f[c] * in;
            const double sbar = f[3 * NN + c] * in;
            const double wc = n * inv_sigma2;
            const int iu = c % N, iv = c / N;
            const double cu = iu - N / 2 + 0.5, cv = iv - N / 2 + 0.5;
            uu[pos] = (T)(cu * cu);
            uv[pos] = (T)(cu * cv);
            vv[pos] = (T)(cv * cv);
            A[pos] = (T)(wc * sbar * sbar);
            if (nj == 1) {
                B[pos] = (T)(wc * sbar * dr);
            } else {
                // B of offset x_j = (dl, dm): w s Re(D exp(-2 pi i k.x_j)), k = du (cu, cv); the
                // cell's values side by side (zero padding)
                const double di = f[NN + c] * in;
                const int nb = b_stride(nj);
                T *row = cells + 4 * plane + ((size_t)s * NN + pos) * nb;
                for (int j = nj; j < nb; ++j) row[j] = T(0);
                for (int j = 0; j < nj; ++j) {
                    const double dl = (j / n_pos - h) * pos_step, dm = (j % n_pos - h) * pos_step;
                    const double th = 2.0 * du * (cu * dl + cv * dm);   // phase / pi
                    double sn, cs;
                    if constexpr (std::is_same<T, float>::value) {
                        float sf, cf;
                        sincospif((float)th, &sf, &cf);
                        sn = sf;
                        cs = cf;
                    } else {
                        sincospi(th, &sn, &cs);
                    }
                    row[j] = (T)(wc * sbar * (dr * cs + di * sn));
                }
            }
            ++pos;
        }
    }
    if (threadIdx.x == 0) {
        int tot = 0;
        double ct = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) {
            tot += warp_tot[i];
            ct += warp_cc[i];
        }
        ncell[s] = tot;
        cc_out[s] = ct;
    }
}

__device__ __forceinline__ double grid_e(const GridConst &g, int k)
{
    return -g.e_max + k * (2.0 * g.e_max / (g.n_e - 1));
}

__device__ __forceinline__ double grid_alpha(const GridConst &g, int k)
{
    const double t = g.n_alpha > 1 ? (double)k / (g.n_alpha - 1) : 0.0;
    return g.r_min + (g.r_max - g.r_min) * t * t;
}

// One work item of the likelihood grid: facet s, threads over (e point, alpha group)
// pairs tile * kThreads .. tile * kThreads + kThreads - 1, over part `part` of
// `n_parts` equal ranges of the facet's cells.  Writes the part's a, b sums in FP64
// to ga, gb (the caller offsets them to the part's slice).
template <typename T, int AG, bool kGauss>
__device__ void grid_tile(int s, int tile, int part, int n_parts, const T *__restrict__ cells,
                          const int32_t *__restrict__ ncell, const SrcRow *__restrict__ table, size_t plane,
                          int32_t NN, const GridConst &gc, double *__restrict__ ga, double *__restrict__ gb)
{
    __shared__ T sm[5][kCellTile];
    const int pair = tile * kThreads + threadIdx.x;
    const int ne2 = gc.n_e * gc.n_e;
    int e_idx, ag, i1, i2, k_lo = 0, k_hi = gc.n_alpha;
    bool on;
    if (gc.box) {
        // sub-box mode: pairs run over the box's e points and alpha groups only
        const int el = pair / gc.n_ag;
        ag = pair % gc.n_ag;
        on = el < kBoxE * kBoxE;
        i1 = gc.box[s * 3 + 0] + el / kBoxE;
        i2 = gc.box[s * 3 + 1] + el % kBoxE;
        k_lo = gc.box[s * 3 + 2];
        k_hi = k_lo + kBoxA;
        e_idx = on ? i1 * gc.n_e + i2 : ne2;
    } else {
        e_idx = pair / gc.n_ag;
        ag = pair % gc.n_ag;
        i1 = e_idx / gc.n_e;
        i2 = e_idx % gc.n_e;
        on = e_idx < ne2;
    }
    double e1 = 0.0, e2 = 0.0;
    if (on) {
        e1 = grid_e(gc, i1);
        e2 = grid_e(gc, i2);
        on = e1 * e1 + e2 * e2 < 1.0;
    }
    const double du = table[s].du;
    T p11 = 0, p12 = 0, p22 = 0;
    T calpha[AG];
    int nk = 0;
    if (on) {
        const double det = 1.0 - e1 * e1 - e2 * e2;
        const double id2 = 1.0 / (det * det);
        p11 = (T)(((1.0 + e1) * (1.0 + e1) + e2 * e2) * id2);
        p12 = (T)(4.0 * e2 * id2);
        p22 = (T)(((1.0 - e1) * (1.0 - e1) + e2 * e2) * id2);
    }
#pragma unroll
    for (int j = 0; j < AG; ++j) {
        const int k = k_lo + ag * AG + j;
        if (k < k_hi) {
            const double al = grid_alpha(gc, k) * kArcsec * du;
            calpha[j] = (T)(4.0 * kPi * kPi * al * al);
            nk = j + 1;
        } else {
            calpha[j] = T(0);
        }
    }
    // FP64 path: FP64 accumulators; FP32 path: the 128-cell tile sums are added to
    // float pairs (hi + lo, exact two-sum, about 48 significant bits, at FP32 speed) in
    // split mode, and in FP64 (a double held in the same two registers) otherwise
    double da[AG], db[AG];
    float ah[AG], al[AG], bh[AG], bl[AG];
#pragma unroll
    for (int j = 0; j < AG; ++j) {
        da[j] = db[j] = 0.0;
        ah[j] = al[j] = bh[j] = bl[j] = 0.0f;
    }
    const bool split = gc.split != 0;
    auto ff_add = [split](float &hi, float &lo, float x) { acc_add(split, hi, lo, x); };

    // the parts split the facet's 128-cell tiles, not its cells: every tile is summed the
    // same way however many parts the launch uses (a fit split over CTAs and one that is
    // not then differ only in how the float-pair tile sums are added, ~1e-14 relative)
    const int nc_all = ncell[s];
    const int n_tiles = (nc_all + kCellTile - 1) / kCellTile;
    const int c_begin = (int)((int64_t)n_tiles * part / n_parts) * kCellTile;
    const int nc = min(nc_all, (int)((int64_t)n_tiles * (part + 1) / n_parts) * kCellTile);
    const T *cu = cells + (size_t)s * NN;
    for (int c0 = c_begin; c0 < nc; c0 += kCellTile) {
        const int nt = min(kCellTile, nc - c0);
        __syncthreads();
        for (int j = threadIdx.x; j < nt; j += kThreads) {
#pragma unroll
            for (int q = 0; q < 5; ++q) sm[q][j] = cu[q * plane + c0 + j];
        }
        __syncthreads();
        if (!on) continue;
        if constexpr (std::is_same<T, float>::value && AG % 2 == 0) {
            // two scalelength nodes per paired FP32 instruction
            // Gaussian profile: c2 carries -alpha-coefficient / 4 and M = 2^(c2 Q)
            f32x2 c2[AG / 2], pa2[AG / 2], pb2[AG / 2];
            const f32x2 one2 = pk2(1.0f, 1.0f), zero2 = pk2(0.0f, 0.0f);
            const float cs = kGauss ? -0.25f : 1.0f;
#pragma unroll
            for (int j = 0; j < AG / 2; ++j) {
                c2[j] = pk2(cs * calpha[2 * j], cs * calpha[2 * j + 1]);
                pa2[j] = pb2[j] = zero2;
            }
            for (int c = 0; c < nt; ++c) {
                const float Q = p11 * sm[0][c] + p12 * sm[1][c] + p22 * sm[2][c];
                const f32x2 Q2 = pk2(Q, Q), A2 = pk2(sm[3][c], sm[3][c]), B2 = pk2(sm[4][c], sm[4][c]);
#pragma unroll
                for (int j = 0; j < AG / 2; ++j) {
                    float x0, x1;
                    f32x2 M2;
                    if (kGauss) {
                        up2(mul2(c2[j], Q2), x0, x1);
                        M2 = pk2(ex2_approx(x0), ex2_approx(x1));
                    } else {
                        up2(fma2(c2[j], Q2, one2), x0, x1);
                        const f32x2 r2 = pk2(rsqrtf(x0), rsqrtf(x1));
                        M2 = mul2(mul2(r2, r2), r2);
                    }
                    pa2[j] = fma2(mul2(A2, M2), M2, pa2[j]);
                    pb2[j] = fma2(B2, M2, pb2[j]);
                }
            }
#pragma unroll
            for (int j = 0; j < AG / 2; ++j) {
                float a0, a1, b0, b1;
                up2(pa2[j], a0, a1);
                up2(pb2[j], b0, b1);
                ff_add(ah[2 * j], al[2 * j], a0);
                ff_add(ah[2 * j + 1], al[2 * j + 1], a1);
                ff_add(bh[2 * j], bl[2 * j], b0);
                ff_add(bh[2 * j + 1], bl[2 * j + 1], b1);
            }
        } else {
            T pa[AG], pb[AG];
#pragma unroll
            for (int j = 0; j < AG; ++j) pa[j] = pb[j] = T(0);
            for (int c = 0; c < nt; ++c) {
                const T Q = p11 * sm[0][c] + p12 * sm[1][c] + p22 * sm[2][c];
                const T A = sm[3][c], B = sm[4][c];
#pragma unroll
                for (int j = 0; j < AG; ++j) {
                    T M;
                    if constexpr (std::is_same<T, float>::value) {
                        M = brightness<kGauss>(calpha[j], Q);
                    } else {
                        M = brightness64(calpha[j] * Q, kGauss ? RLF_PROFILE_GAUSSIAN : RLF_PROFILE_EXPONENTIAL);
                    }
                    const T AM = A * M;
                    pa[j] += AM * M;
                    pb[j] += B * M;
                }
            }
#pragma unroll
            for (int j = 0; j < AG; ++j) {
                if constexpr (std::is_same<T, float>::value) {
                    ff_add(ah[j], al[j], pa[j]);
                    ff_add(bh[j], bl[j], pb[j]);
                } else {
                    da[j] += (double)pa[j];
                    db[j] += (double)pb[j];
                }
            }
        }
    }
    if constexpr (std::is_same<T, float>::value) {
#pragma unroll
        for (int j = 0; j < AG; ++j) {
            da[j] = acc_value(split, ah[j], al[j]);
            db[j] = acc_value(split, bh[j], bl[j]);
        }
    }
    if (e_idx < ne2) {
        const size_t base = ((size_t)s * ne2 + e_idx) * gc.n_alpha + k_lo + (size_t)ag * AG;
        for (int j = 0; j < nk; ++j) {
            ga[base + j] = on ? da[j] : 0.0;
            gb[base + j] = on ? db[j] : 0.0;
        }
    }
}

// block reductions over NT threads (fixed tree order)
template <int NT = kThreads>
__device__ double block_sum(double x, double *scratch)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = x;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += scratch[i];
    return t;
}

template <int NT = kThreads>
__device__ double block_max(double x, double *scratch)
{
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) scratch[wid] = x;
    __syncthreads();
    double t = -INFINITY;
    for (int i = 0; i < NT / 32; ++i) t = fmax(t, scratch[i]);
    return t;
}

// argmax with ties to the lowest index
template <int NT = kThreads>
__device__ void block_argmax(double &v, long long &idx, double *sv, long long *si)
{
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, o);
        const long long oi = __shfl_down_sync(0xffffffffu, idx, o);
        if (ov > v || (ov == v && oi < idx)) {
            v = ov;
            idx = oi;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sv[wid] = v;
        si[wid] = idx;
    }
    __syncthreads();
    v = -INFINITY;
    idx = 0x7fffffffffffffffLL;
    for (int i = 0; i < NT / 32; ++i)
        if (sv[i] > v || (sv[i] == v && si[i] < idx)) {
            v = sv[i];
            idx = si[i];
        }
}

// flux-marginalised log-likelihood (Sec. 2.4); for b < 0 the erfc factor is
// written through erfcx so that b^2/(2a) cancels analytically
__device__ double flux_marginal(double a, double b, double cc, int flux_prior)
{
    if (flux_prior == 1) return -0.5 * cc + b * b / (2.0 * a) + 0.5 * log(2.0 * kPi / a);
    const double x = -b / sqrt(2.0 * a);
    if (x > 0.0) return -0.5 * cc + 0.5 * log(kPi / (2.0 * a)) + log(erfcx(x));
    return -0.5 * cc + b * b / (2.0 * a) + 0.5 * log(kPi / (2.0 * a)) + log(erfc(x));
}

// The same with the logarithms and error functions, whose values are O(1), in FP32:
// absolute error ~1e-6 in ln L (far below the FP32 model's ~1e-7 b^2/a); the terms
// that cancel at high SNR, -C/2 + b^2/(2a), stay FP64.  Used by the mixed modes,
// where the FP64 transcendentals of 8820 grid points in one CTA dominated the
// estimate's time.
__device__ double flux_marginal_mixed(double a, double b, double cc, int flux_prior)
{
    const float lg = 0.5f * logf(3.14159265358979323846f / (2.0f * (float)a));
    if (flux_prior == 1) return -0.5 * cc + b * b / (2.0 * a) + (double)(lg + 0.5f * 1.38629436111989061883f);
    const float x = (float)(-b) * rsqrtf((float)(2.0 * a));
    if (x > 0.0f) return -0.5 * cc + (double)(lg + logf(erfcxf(x)));
    return -0.5 * cc + b * b / (2.0 * a) + (double)(lg + logf(erfcf(x)));
}

// Position marginal (Sec. 2.4), FP64: ln of the mean over the NJ offsets of
// exp(logL(a, b_j)), and the b of the best offset (the first of equal ones).
template <int NJ>
__device__ double position_marginal(double a, const double *b, double cc, int flux_prior, double &b_best)
{
    double m = -INFINITY, sum = 0.0;
    b_best = b[0];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const double v = flux_marginal(a, b[j], cc, flux_prior);
        if (v > m) {
            sum = sum * (m == -INFINITY ? 0.0 : exp(m - v)) + 1.0;
            m = v;
            b_best = b[j];
        } else {
            sum += exp(v - m);
        }
    }
    return m + log(sum / NJ);
}

// The same from float-pair sums b_j = bh_j + bl_j, with no FP64 per offset.  logL
// grows with b (flux prior S >= 0; with the real-line prior, with |b|), so the best
// offset is the largest b, and logL_j - logL_best = F(b_j) - F(b_best) with
// F(b) = b^2/(2a) + ln erfc(-b/sqrt(2a)) (= ln erfcx(-b/sqrt(2a)) for b < 0): the b^2
// part is (b_j - b_m)(b_j + b_m)/(2a), both factors formed from the pairs in FP32, so
// it keeps FP32 relative accuracy however large b^2/(2a) is.  One FP64 logL, at the
// best offset.
template <int NJ>
__device__ double position_marginal_ff(double a, const float *bh, const float *bl, double cc, int flux_prior,
                                       double &b_best)
{
    float mh = bh[0], ml = bl[0];
#pragma unroll
    for (int j = 1; j < NJ; ++j) {
        const float d = (bh[j] - mh) + (bl[j] - ml);
        const float s = (bh[j] + mh) + (bl[j] + ml);
        if (flux_prior == 1 ? d * s > 0.0f : d > 0.0f) {
            mh = bh[j];
            ml = bl[j];
        }
    }
    b_best = (double)mh + (double)ml;
    const float ia = 0.5f / (float)a, r2a = rsqrtf((float)(2.0 * a));
    const float bm = mh + ml;
    float lm = 0.0f;
    if (flux_prior != 1) {
        const float xm = -bm * r2a;
        lm = xm > 0.0f ? logf(erfcxf(xm)) : logf(erfcf(xm));
    }
    float sum = 0.0f;
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const float d = (bh[j] - mh) + (bl[j] - ml);
        const float s = (bh[j] + mh) + (bl[j] + ml);
        float G;
        if (flux_prior == 1) {
            G = d * s * ia;
        } else {
            const float bj = bh[j] + bl[j], xj = -bj * r2a;
            const float q = bj >= 0.0f ? d * s * ia : (bm >= 0.0f ? -bm * bm * ia : 0.0f);
            G = q + (xj > 0.0f ? logf(erfcxf(xj)) : logf(erfcf(xj))) - lm;
        }
        sum += expf(G);
    }
    return flux_marginal_mixed(a, b_best, cc, flux_prior) + (double)logf(sum / NJ);
}

// One work item of the likelihood grid with the position marginal: facet s, one
// (e point, alpha node) per thread for pairs tile * kThreads .. + kThreads - 1, every
// cell, every offset.  Per cell: the brightness M once, a += A M^2 and, for the NJ
// offsets, b_j += B_j M, two offsets per paired FP32 instruction (FP32 tile sums added
// to float pairs, as in grid_tile).  The thread then writes a, the best offset's b and
// the marginal logL of its point (ga, gb, gl).
template <typename T, int NJ, bool kGauss>
__device__ void grid_tile_pos(int s, int tile, const T *__restrict__ cells, const int32_t *__restrict__ ncell,
                              const SrcRow *__restrict__ table, size_t plane, int32_t NN, const GridConst &gc,
                              const double *__restrict__ ccv, double *__restrict__ ga, double *__restrict__ gb,
                              double *__restrict__ gl)
{
    constexpr bool f32 = std::is_same<T, float>::value;
    constexpr int NB = (NJ + 3) / 4 * 4;            // B values per cell (b_stride)
    constexpr int NP = (NJ + 1) / 2;                // offset pairs
    constexpr int kT = f32 ? kCellTile : kCellTile / 2;
    __shared__ __align__(16) T sg[kT][4];           // uu, uv, vv, A of each staged cell
    __shared__ __align__(16) T sb[kT][NB];          // B_j of each staged cell
    const int pair = tile * kThreads + threadIdx.x;
    const int ne2 = gc.n_e * gc.n_e, na = gc.n_alpha;
    const int e_idx = pair / na, k = pair % na;
    const int i1 = e_idx / gc.n_e, i2 = e_idx % gc.n_e;
    bool on = e_idx < ne2;
    double e1 = 0.0, e2 = 0.0;
    if (on) {
        e1 = grid_e(gc, i1);
        e2 = grid_e(gc, i2);
        on = e1 * e1 + e2 * e2 < 1.0;
    }
    const double du = table[s].du;
    T p11 = 0, p12 = 0, p22 = 0, ca = 0;
    if (on) {
        const double det = 1.0 - e1 * e1 - e2 * e2;
        const double id2 = 1.0 / (det * det);
        p11 = (T)(((1.0 + e1) * (1.0 + e1) + e2 * e2) * id2);
        p12 = (T)(4.0 * e2 * id2);
        p22 = (T)(((1.0 - e1) * (1.0 - e1) + e2 * e2) * id2);
        const double al = grid_alpha(gc, k) * kArcsec * du;
        ca = (T)(4.0 * kPi * kPi * al * al);
    }
    double da = 0.0, db[NJ];
    float ah = 0.0f, al = 0.0f, bh[NJ], bl[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        db[j] = 0.0;
        bh[j] = bl[j] = 0.0f;
    }
    const bool split = gc.split != 0;
    auto ff_add = [split](float &hi, float &lo, float x) { acc_add(split, hi, lo, x); };
    const int nc = ncell[s];
    const T *cu = cells + (size_t)s * NN;
    for (int c0 = 0; c0 < nc; c0 += kT) {
        const int nt = min(kT, nc - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * nt; i += kThreads) sg[i % nt][i / nt] = cu[(i / nt) * plane + c0 + i % nt];
        // the cells' B rows: one contiguous run (16-byte vectors in FP32)
        const T *brow = cells + 4 * plane + ((size_t)s * NN + c0) * NB;
        if constexpr (f32) {
            const float4 *src = reinterpret_cast<const float4 *>(brow);
            float4 *dst = reinterpret_cast<float4 *>(&sb[0][0]);
            for (int i = threadIdx.x; i < nt * NB / 4; i += kThreads) dst[i] = src[i];
        } else {
            for (int i = threadIdx.x; i < nt * NB; i += kThreads) (&sb[0][0])[i] = brow[i];
        }
        __syncthreads();
        if (!on) continue;
        if constexpr (f32) {
            float pa = 0.0f;
            f32x2 pb2[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) pb2[q] = pk2(0.0f, 0.0f);
#pragma unroll 2
            for (int c = 0; c < nt; ++c) {
                const float4 g4 = *reinterpret_cast<const float4 *>(&sg[c][0]);
                const float Q = p11 * g4.x + p12 * g4.y + p22 * g4.z;
                const float M = brightness<kGauss>(ca, Q);
                pa = fmaf(g4.w * M, M, pa);
                const f32x2 M2 = pk2(M, M);
                const ulonglong2 *row = reinterpret_cast<const ulonglong2 *>(&sb[c][0]);
#pragma unroll
                for (int q = 0; q < NB / 4; ++q) {
                    const ulonglong2 v = row[q];
                    pb2[2 * q] = fma2(v.x, M2, pb2[2 * q]);
                    if (2 * q + 1 < NP) pb2[2 * q + 1] = fma2(v.y, M2, pb2[2 * q + 1]);
                }
            }
            ff_add(ah, al, pa);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float b0, b1;
                up2(pb2[q], b0, b1);
                ff_add(bh[2 * q], bl[2 * q], b0);
                if (2 * q + 1 < NJ) ff_add(bh[2 * q + 1], bl[2 * q + 1], b1);
            }
        } else {
            T pa = T(0), pb[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) pb[j] = T(0);
            for (int c = 0; c < nt; ++c) {
                const T Q = p11 * sg[c][0] + p12 * sg[c][1] + p22 * sg[c][2];
                const T M = brightness64(ca * Q, kGauss ? RLF_PROFILE_GAUSSIAN : RLF_PROFILE_EXPONENTIAL);
                const T AM = sg[c][3] * M;
                pa += AM * M;
#pragma unroll
                for (int j = 0; j < NJ; ++j) pb[j] += sb[c][j] * M;
            }
            da += (double)pa;
#pragma unroll
            for (int j = 0; j < NJ; ++j) db[j] += (double)pb[j];
        }
    }
    if (e_idx >= ne2) return;
    const size_t g = ((size_t)s * ne2 + e_idx) * na + k;
    if (on && nc > 0) {
        double bb;
        if constexpr (f32) {
            da = acc_value(split, ah, al);
            if (split) {
                gl[g] = position_marginal_ff<NJ>(da, bh, bl, ccv[s], gc.flux_prior, bb);
            } else {
#pragma unroll
                for (int j = 0; j < NJ; ++j) db[j] = pair_as_double(bh[j], bl[j]);
                gl[g] = position_marginal<NJ>(da, db, ccv[s], gc.flux_prior, bb);
            }
        } else {
            gl[g] = position_marginal<NJ>(da, db, ccv[s], gc.flux_prior, bb);
        }
        ga[g] = da;
        gb[g] = bb;
    } else {
        gl[g] = -INFINITY;
        ga[g] = 0.0;
        gb[g] = 0.0;
    }
}

// grid_tile_pos in FP32 with NODES scalelength nodes per thread (n_pos <= 3): item
// tile * kThreads + threadIdx.x is (e point, alpha nodes NODES g .. NODES g + NODES - 1).
// Each staged cell's quadratic form, A and B_j row are read from shared memory once for
// all the nodes, which divides the shared-memory reads per evaluation by NODES (the
// broadcasts of the B rows bound the one-node form); the brightness values and every
// b_j update are paired FP32 instructions.  The arithmetic of each node is the one-node
// form's, operation for operation, so the results are the same bit for bit.
template <int NJ, int NODES, bool kGauss>
__device__ void grid_tile_posn(int s, int tile, const float *__restrict__ cells, const int32_t *__restrict__ ncell,
                               const SrcRow *__restrict__ table, size_t plane, int32_t NN, const GridConst &gc,
                               const double *__restrict__ ccv, double *__restrict__ ga, double *__restrict__ gb,
                               double *__restrict__ gl)
{
    constexpr int NB = (NJ + 3) / 4 * 4;            // B values per cell (b_stride)
    constexpr int NP = (NJ + 1) / 2;                // offset pairs
    constexpr int NM = (NODES + 1) / 2;             // node pairs (the last one half used when NODES is odd)
    __shared__ __align__(16) float sg[kCellTile][4];
    __shared__ __align__(16) float sb[kCellTile][NB];
    const int item = tile * kThreads + threadIdx.x;
    const int ne2 = gc.n_e * gc.n_e, na = gc.n_alpha, nag = (na + NODES - 1) / NODES;
    const int e_idx = item / nag, k0 = NODES * (item % nag);
    const int nk = min(NODES, na - k0);
    const int i1 = e_idx / gc.n_e, i2 = e_idx % gc.n_e;
    bool on = e_idx < ne2;
    double e1 = 0.0, e2 = 0.0;
    if (on) {
        e1 = grid_e(gc, i1);
        e2 = grid_e(gc, i2);
        on = e1 * e1 + e2 * e2 < 1.0;
    }
    const double du = table[s].du;
    float p11 = 0.0f, p12 = 0.0f, p22 = 0.0f, ca[2 * NM];
#pragma unroll
    for (int j = 0; j < 2 * NM; ++j) ca[j] = 0.0f;
    if (on) {
        const double det = 1.0 - e1 * e1 - e2 * e2;
        const double id2 = 1.0 / (det * det);
        p11 = (float)(((1.0 + e1) * (1.0 + e1) + e2 * e2) * id2);
        p12 = (float)(4.0 * e2 * id2);
        p22 = (float)(((1.0 - e1) * (1.0 - e1) + e2 * e2) * id2);
#pragma unroll
        for (int j = 0; j < 2 * NM; ++j) {
            const double al = grid_alpha(gc, j < nk ? k0 + j : k0) * kArcsec * du;
            ca[j] = (float)(4.0 * kPi * kPi * al * al);
        }
    }
    // Gaussian profile: c2 carries -alpha-coefficient / 4 and M = 2^(c2 Q)
    const float cs = kGauss ? -0.25f : 1.0f;
    f32x2 c2[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) c2[m] = pk2(cs * ca[2 * m], cs * ca[2 * m + 1]);
    const f32x2 one2 = pk2(1.0f, 1.0f), zero2 = pk2(0.0f, 0.0f);
    float ah[NODES], al[NODES], bh[NODES][NJ], bl[NODES][NJ];
#pragma unroll
    for (int n = 0; n < NODES; ++n) {
        ah[n] = al[n] = 0.0f;
#pragma unroll
        for (int j = 0; j < NJ; ++j) bh[n][j] = bl[n][j] = 0.0f;
    }
    const bool split = gc.split != 0;
    const int nc = ncell[s];
    const float *cu = cells + (size_t)s * NN;
    for (int c0 = 0; c0 < nc; c0 += kCellTile) {
        const int nt = min(kCellTile, nc - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < 4 * nt; i += kThreads) sg[i % nt][i / nt] = cu[(i / nt) * plane + c0 + i % nt];
        {
            const float4 *src = reinterpret_cast<const float4 *>(cells + 4 * plane + ((size_t)s * NN + c0) * NB);
            float4 *dst = reinterpret_cast<float4 *>(&sb[0][0]);
            for (int i = threadIdx.x; i < nt * NB / 4; i += kThreads) dst[i] = src[i];
        }
        __syncthreads();
        if (!on) continue;
        f32x2 pa2[NM], pb[NODES][NP];
#pragma unroll
        for (int m = 0; m < NM; ++m) pa2[m] = zero2;
#pragma unroll
        for (int n = 0; n < NODES; ++n)
#pragma unroll
            for (int q = 0; q < NP; ++q) pb[n][q] = zero2;
#pragma unroll 2
        for (int c = 0; c < nt; ++c) {
            const float4 g4 = *reinterpret_cast<const float4 *>(&sg[c][0]);
            const float Q = p11 * g4.x + p12 * g4.y + p22 * g4.z;
            const f32x2 Q2 = pk2(Q, Q), A2 = pk2(g4.w, g4.w);
            f32x2 Mn[NODES];
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                float x0, x1;
                f32x2 M2;
                if (kGauss) {
                    up2(mul2(c2[m], Q2), x0, x1);
                    M2 = pk2(ex2_approx(x0), 2 * m + 1 < NODES ? ex2_approx(x1) : 0.0f);
                } else {
                    up2(fma2(c2[m], Q2, one2), x0, x1);
                    const f32x2 r2 = pk2(rsqrtf(x0), 2 * m + 1 < NODES ? rsqrtf(x1) : 0.0f);
                    M2 = mul2(mul2(r2, r2), r2);
                }
                pa2[m] = fma2(mul2(A2, M2), M2, pa2[m]);
                float m0, m1;
                up2(M2, m0, m1);
                Mn[2 * m] = pk2(m0, m0);
                if (2 * m + 1 < NODES) Mn[2 * m + 1] = pk2(m1, m1);
            }
            const ulonglong2 *row = reinterpret_cast<const ulonglong2 *>(&sb[c][0]);
#pragma unroll
            for (int q = 0; q < NB / 4; ++q) {
                const ulonglong2 v = row[q];
#pragma unroll
                for (int n = 0; n < NODES; ++n) {
                    pb[n][2 * q] = fma2(v.x, Mn[n], pb[n][2 * q]);
                    if (2 * q + 1 < NP) pb[n][2 * q + 1] = fma2(v.y, Mn[n], pb[n][2 * q + 1]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < NM; ++m) {
            float a0, a1;
            up2(pa2[m], a0, a1);
            acc_add(split, ah[2 * m], al[2 * m], a0);
            if (2 * m + 1 < NODES) acc_add(split, ah[2 * m + 1], al[2 * m + 1], a1);
        }
#pragma unroll
        for (int n = 0; n < NODES; ++n)
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float b0, b1;
                up2(pb[n][q], b0, b1);
                acc_add(split, bh[n][2 * q], bl[n][2 * q], b0);
                if (2 * q + 1 < NJ) acc_add(split, bh[n][2 * q + 1], bl[n][2 * q + 1], b1);
            }
    }
    if (e_idx >= ne2) return;
#pragma unroll
    for (int j = 0; j < NODES; ++j) {
        if (j >= nk) break;
        const size_t g = ((size_t)s * ne2 + e_idx) * na + k0 + j;
        if (on && nc > 0) {
            const double da = acc_value(split, ah[j], al[j]);
            double bb;
            if (split) {
                gl[g] = position_marginal_ff<NJ>(da, bh[j], bl[j], ccv[s], gc.flux_prior, bb);
            } else {
                double db[NJ];
#pragma unroll
                for (int i = 0; i < NJ; ++i) db[i] = pair_as_double(bh[j][i], bl[j][i]);
                gl[g] = position_marginal<NJ>(da, db, ccv[s], gc.flux_prior, bb);
            }
            ga[g] = da;
            gb[g] = bb;
        } else {
            gl[g] = -INFINITY;
            ga[g] = 0.0;
            gb[g] = 0.0;
        }
    }
}

// Estimate of facet s from its complete a, b grid (block-wide, FP64; with `mixed`
// the logarithms, error functions and exponentials in FP32).  logl_ready: gl already
// holds logL of every valid point (the position marginal's grid writes it).
__device__ void estimate_source(bool mixed, bool logl_ready, int s, const double *__restrict__ ga,
                                const double *__restrict__ gb,
                                double *__restrict__ gl, const int32_t *__restrict__ ncell,
                                const double *__restrict__ ccv, const SrcRow *__restrict__ table,
                                const GridConst &gc, const rlf_fit_out &out, int32_t out_offset,
                                int32_t *__restrict__ status, int32_t *__restrict__ map_out)
{
    __shared__ double red[kThreads / 32];
    __shared__ long long redi[kThreads / 32];
    __shared__ double qp[64], alph[64], lnp[64];
    __shared__ double Le[kMaxNe * kMaxNe], Ae[kMaxNe * kMaxNe];
    const int ne = gc.n_e, na = gc.n_alpha, ne2 = ne * ne;
    const long long ng = (long long)ne2 * na;
    const SrcRow S = table[s];
    const int nc = ncell[s];
    const double cc = ccv[s];
    const double *a = ga + (size_t)s * ng;
    const double *b = gb + (size_t)s * ng;
    double *lg = gl + (size_t)s * ng;

    if (threadIdx.x < na) {
        const int k = threadIdx.x;
        const double ak = grid_alpha(gc, k);
        double q;
        if (na == 1) q = 1.0;
        else if (k == 0) q = 0.5 * (grid_alpha(gc, 1) - ak);
        else if (k == na - 1) q = 0.5 * (ak - grid_alpha(gc, na - 2));
        else q = 0.5 * (grid_alpha(gc, k + 1) - grid_alpha(gc, k - 1));
        const double z = (log(ak) - S.mu) / gc.r_std;
        qp[k] = q * exp(-0.5 * z * z) / (ak * gc.r_std * sqrt(2.0 * kPi));
        alph[k] = ak;
        lnp[k] = -0.5 * z * z - log(ak);
    }
    // logL on every valid point
    double lmax = -INFINITY;
    bool bad_num = false;
    for (long long g = threadIdx.x; g < ng; g += kThreads) {
        const int e_idx = (int)(g / na);
        const double e1 = grid_e(gc, e_idx / ne), e2 = grid_e(gc, e_idx % ne);
        double v = -INFINITY;
        bool in_box = true;
        if (gc.box) {
            const int d1 = e_idx / ne - gc.box[s * 3 + 0], d2 = e_idx % ne - gc.box[s * 3 + 1];
            const int dk = (int)(g % na) - gc.box[s * 3 + 2];
            in_box = d1 >= 0 && d1 < kBoxE && d2 >= 0 && d2 < kBoxE && dk >= 0 && dk < kBoxA;
        }
        if (in_box && nc > 0 && e1 * e1 + e2 * e2 < 1.0) {
            if (logl_ready) v = lg[g];
            else v = mixed ? flux_marginal_mixed(a[g], b[g], cc, gc.flux_prior) : flux_marginal(a[g], b[g], cc, gc.flux_prior);
            if (!isfinite(v)) bad_num = true;
        }
        lg[g] = v;
        lmax = fmax(lmax, v);
    }
    if (bad_num) atomicOr(status, RLF_DEV_NONFINITE);
    lmax = block_max(lmax, red);
    __syncthreads();
    // alpha marginal per e point
    double Lm = 0.0;
    for (int e = threadIdx.x; e < ne2; e += kThreads) {
        double sL = 0.0, sA = 0.0;
        for (int k = 0; k < na; ++k) {
            const double v = lg[(size_t)e * na + k];
            if (v == -INFINITY) continue;
            const double t = qp[k] * (mixed ? (double)expf((float)(v - lmax)) : exp(v - lmax));
            sL += t;
            sA += t * alph[k];
        }
        Le[e] = sL;
        Ae[e] = sA;
        Lm = fmax(Lm, sL);
    }
    const double Lmax = block_max(Lm, red);
    __syncthreads();
    // Sub-box fit: the box stands for the full grid only when nothing near the threshold
    // touches a face of the box that is not a face of the grid.  Every e point with
    // L(e) >= thresh_frac Lmax / 2 must lie off the inner e faces, and its alpha profile at
    // an inner alpha face must be below 1e-6 L(e) (the alpha marginal over the box's nodes
    // then misses at most ~1e-5 of the full grid's).  Otherwise the facet is fitted again
    // on the full grid.
    if (gc.box && gc.box_fail) {
        const int o1 = gc.box[s * 3 + 0], o2 = gc.box[s * 3 + 1], ok = gc.box[s * 3 + 2];
        const double cut = 0.5 * gc.thresh_frac * Lmax;
        bool fail = false;
        for (int e = threadIdx.x; e < ne2; e += kThreads) {
            const double L = Le[e];
            if (!(L > 0.0) || L < cut) continue;
            const int i1 = e / ne, i2 = e % ne;
            if ((i1 == o1 && o1 > 0) || (i1 == o1 + kBoxE - 1 && o1 + kBoxE < ne) || (i2 == o2 && o2 > 0) ||
                (i2 == o2 + kBoxE - 1 && o2 + kBoxE < ne))
                fail = true;
            const int kf[2] = {ok > 0 ? ok : -1, ok + kBoxA < na ? ok + kBoxA - 1 : -1};
            for (int f = 0; f < 2; ++f) {
                if (kf[f] < 0) continue;
                const double v = lg[(size_t)e * na + kf[f]];
                if (v == -INFINITY) continue;
                const double t = qp[kf[f]] * (mixed ? (double)expf((float)(v - lmax)) : exp(v - lmax));
                if (t > 1.0e-6 * L) fail = true;
            }
        }
        if (fail) gc.box_fail[s] = 1;
    }
    // moments above the threshold and over every point
    double W = 0, m1 = 0, m2 = 0, WA = 0, Ws = 0, s1 = 0, s2 = 0;
    for (int e = threadIdx.x; e < ne2; e += kThreads) {
        const double L = Le[e];
        if (!(L > 0.0)) continue;
        const double e1 = grid_e(gc, e / ne), e2 = grid_e(gc, e % ne);
        Ws += L;
        s1 += L * e1;
        s2 += L * e2;
        if (L >= gc.thresh_frac * Lmax) {
            W += L;
            m1 += L * e1;
            m2 += L * e2;
            WA += Ae[e];
        }
    }
    W = block_sum(W, red);
    m1 = block_sum(m1, red);
    m2 = block_sum(m2, red);
    WA = block_sum(WA, red);
    Ws = block_sum(Ws, red);
    s1 = block_sum(s1, red);
    s2 = block_sum(s2, red);
    const double e1m = W > 0 ? m1 / W : 0.0, e2m = W > 0 ? m2 / W : 0.0;
    double c11 = 0, c22 = 0, c12 = 0;
    for (int e = threadIdx.x; e < ne2; e += kThreads) {
        const double L = Le[e];
        if (!(L > 0.0) || L < gc.thresh_frac * Lmax) continue;
        const double d1 = grid_e(gc, e / ne) - e1m, d2 = grid_e(gc, e % ne) - e2m;
        c11 += L * d1 * d1;
        c22 += L * d2 * d2;
        c12 += L * d1 * d2;
    }
    c11 = block_sum(c11, red);
    c22 = block_sum(c22, red);
    c12 = block_sum(c12, red);
    // MAP grid point: logL + ln p(alpha), ties to the lowest flat index
    double best = -INFINITY;
    long long gbest = 0x7fffffffffffffffLL;
    for (long long g = threadIdx.x; g < ng; g += kThreads) {
        const double v = lg[g];
        if (v == -INFINITY) continue;
        const double lp = v + lnp[g % na];
        if (lp > best || (lp == best && g < gbest)) {
            best = lp;
            gbest = g;
        }
    }
    block_argmax(best, gbest, red, redi);
    if (threadIdx.x == 0) {
        if (W > 0) {
            c11 /= W;
            c22 /= W;
            c12 /= W;
        }
        const double sd1 = sqrt(c11), sd2 = sqrt(c22);
        const double det = c11 * c22 - c12 * c12;
        const double sdet = det > 0 ? sqrt(det) : 0.0;
        int flag = 0;
        if (!(W > 0) || sd1 <= gc.var_sigma_min || sd2 <= gc.var_sigma_min || sdet <= gc.var_det_min)
            flag |= RLF_FLAG_BAD;
        if (S.invalid) flag |= RLF_FLAG_INVALID;
        if (nc == 0) flag |= RLF_FLAG_EMPTY;
        const int o = out_offset + s;
        double fl = 0.0;
        if (best > -INFINITY && a[gbest] > 0) fl = b[gbest] / a[gbest];
        out.e1[o] = e1m;
        out.e2[o] = e2m;
        out.sig1[o] = sd1;
        out.sig2[o] = sd2;
        out.alpha_arcsec[o] = W > 0 ? WA / W : 0.0;
        out.flux_jy[o] = fl;
        out.e1_smooth[o] = Ws > 0 ? s1 / Ws : 0.0;
        out.e2_smooth[o] = Ws > 0 ? s2 / Ws : 0.0;
        out.flag[o] = flag;
        if (map_out) map_out[s] = best > -INFINITY ? (int32_t)gbest : -1;
    }
}


// Largest facets first (LPT order): rank of facet i = number of facets with more
// cells, ties by index.  order[rank] = i.
__global__ void lpt_order_kernel(const int32_t *__restrict__ ncell, int32_t count, int32_t *__restrict__ order)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int ni = ncell[i];
    int rank = 0;
    for (int j = 0; j < count; ++j) {
        const int nj = ncell[j];
        rank += (nj > ni) || (nj == ni && j < i);
    }
    order[rank] = i;
}

// Persistent likelihood fit: every CTA takes work items (facet in LPT order,
// tile of grid pairs, part of the facet's cells) from an atomic counter until none
// is left; the CTA that completes a facet's last item (per-facet atomic counter
// after a fence) adds the parts' sums in part order and runs that facet's
// estimate.  Nothing waits on another CTA.  When the launch has fewer (facet, tile)
// items than CTAs (few facets, or the 7 x 7 x 5 sub-box), each facet's cells are
// split into up to max_parts parts (kMaxFitParts, or more for a small workspace)
// so that every CTA has work; the number of
// facets may be known only on the device (refit list), so the split is chosen here.
template <typename T, int AG, bool kGauss>
__global__ void __launch_bounds__(kThreads, 3)
fit_persistent_kernel(const T *__restrict__ cells, const int32_t *__restrict__ ncell,
                      const SrcRow *__restrict__ table, size_t plane, int32_t NN, int32_t tiles_per_src,
                      int32_t count, const int32_t *__restrict__ count_dev, const int32_t *__restrict__ order,
                      int32_t *__restrict__ counters, const GridConst gc, double *__restrict__ ga,
                      double *__restrict__ gb, size_t part_stride, int32_t max_parts, double *__restrict__ gl,
                      const double *__restrict__ ccv, rlf_fit_out out, int32_t out_offset,
                      int32_t *__restrict__ status, int32_t *__restrict__ map_out)
{
    __shared__ int s_item, s_last;
    int32_t *item_counter = counters;
    int32_t *src_done = counters + 1;
    const int n_src = count_dev ? *count_dev : count;
    const int64_t pairs_items = (int64_t)n_src * tiles_per_src;
    int n_parts = pairs_items > 0 ? (int)((gridDim.x + pairs_items - 1) / pairs_items) : 1;
    n_parts = n_parts < 1 ? 1 : (n_parts > max_parts ? max_parts : n_parts);
    const int per_src = tiles_per_src * n_parts;
    const int total = n_src * per_src;
    const size_t ng = (size_t)gc.n_e * gc.n_e * gc.n_alpha;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(item_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int s = order[item / per_src];
        const int rem = item % per_src;
        const int tile = rem / n_parts, part = rem % n_parts;
        grid_tile<T, AG, kGauss>(s, tile, part, n_parts, cells, ncell, table, plane, NN, gc, ga + part * part_stride,
                         gb + part * part_stride);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&src_done[s], 1) == per_src - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (n_parts > 1) {
                // parts 1.. into part 0, in part order (entries a part did not write are
                // outside the sub-box and never read)
                double *a0 = ga + (size_t)s * ng, *b0 = gb + (size_t)s * ng;
                for (size_t g = threadIdx.x; g < ng; g += kThreads) {
                    double a = a0[g], b = b0[g];
                    for (int q = 1; q < n_parts; ++q) {
                        a += a0[q * part_stride + g];
                        b += b0[q * part_stride + g];
                    }
                    a0[g] = a;
                    b0[g] = b;
                }
                __syncthreads();
            }
            estimate_source(std::is_same<T, float>::value && gc.split, false, s, ga, gb, gl, ncell, ccv, table, gc,
                            out, out_offset, status, map_out);
        }
        __syncthreads();
    }
}

// The persistent fit with the position marginal: work item = (facet in LPT order, tile
// of (e point, alpha node) pairs, or of (e point, alpha node pair) items in the two-node
// FP32 form) over every cell; the CTA completing a facet's last tile runs its estimate
// on the marginal logL the tiles wrote.
template <typename T, int NJ>
constexpr bool kPos2 = std::is_same<T, float>::value && NJ <= 9;
constexpr int kPosNodes = 3;   // scalelength nodes per thread in that form

template <typename T, int NJ, bool kGauss>
__global__ void __launch_bounds__(kThreads, 2)
fit_persistent_pos_kernel(const T *__restrict__ cells, const int32_t *__restrict__ ncell,
                          const SrcRow *__restrict__ table, size_t plane, int32_t NN, int32_t tiles_per_src,
                          int32_t count, const int32_t *__restrict__ order, int32_t *__restrict__ counters,
                          const GridConst gc, double *__restrict__ ga, double *__restrict__ gb,
                          double *__restrict__ gl, const double *__restrict__ ccv, rlf_fit_out out,
                          int32_t out_offset, int32_t *__restrict__ status)
{
    __shared__ int s_item, s_last;
    const int total = count * tiles_per_src;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counters, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) break;
        const int s = order[item / tiles_per_src];
        if constexpr (kPos2<T, NJ>)
            grid_tile_posn<NJ, kPosNodes, kGauss>(s, item % tiles_per_src, cells, ncell, table, plane, NN, gc, ccv,
                                                  ga, gb, gl);
        else
            grid_tile_pos<T, NJ, kGauss>(s, item % tiles_per_src, cells, ncell, table, plane, NN, gc, ccv, ga, gb,
                                         gl);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(&counters[1 + s], 1) == tiles_per_src - 1;
        __syncthreads();
        if (s_last) {
            __threadfence();
            estimate_source(std::is_same<T, float>::value && gc.split, true, s, ga, gb, gl, ncell, ccv, table, gc, out,
                            out_offset, status, nullptr);
        }
        __syncthreads();
    }
}

// ---- adaptive sampling around the maximum (Sec. 2.4) ---------------------------------
// After the grid fit: one CTA per facet.  Level 0 is the grid (its log-likelihood
// grid gl and sums ga, gb); while fewer than np_max samples of the alpha marginal
// L(e) lie at or above thresh_frac of its maximum and the step exceeds e_res, the
// step is halved and every multiple of it in the box of the kept samples, widened by
// the previous step, is sampled (|e| < 1, at most 17 per component around the MAP
// sample).  The estimate is the last level's, by the rules of the grid estimate.
constexpr int kAT = 512;    // threads of an adaptive-sampling CTA (one facet each)
constexpr int kATc = 128;   // threads of a CTA of the cluster form
constexpr int kATcBlocks = 5;   // its CTAs per SM (96 registers; 4 left 40 % of the warp slots empty, 6 spilled)
constexpr int kAdaptR = 4;  // CTAs per facet in the cluster form
static_assert(kAdaptR <= kAdaptRanks && kAdaptR <= 8, "a portable cluster, within the partials' scratch");

struct AdaptResult {
    double e1m, e2m, sd1, sd2, am, flux, e1s, e2s;
    int bad, kept, map_i;
    double box[4];
};

// block-wide estimate over np samples (e of sample i: grid node i / n_e, i % n_e when
// e1s is null); lg, a, b are [np][n_alpha]
template <int NT>
__device__ void estimate_over_samples(bool mixed, int np, const double *e1s, const double *e2s,
                                      const double *__restrict__ lg, const double *__restrict__ a,
                                      const double *__restrict__ b, const GridConst &gc, const double *qp,
                                      const double *alph, const double *lnp, double *Ls, double *As,
                                      AdaptResult &res)
{
    __shared__ double red[NT / 32];
    __shared__ long long redi[NT / 32];
    const int na = gc.n_alpha, ne = gc.n_e;
    const long long npa = (long long)np * na;
    auto e1_of = [&](int i) { return e1s ? e1s[i] : grid_e(gc, i / ne); };
    auto e2_of = [&](int i) { return e2s ? e2s[i] : grid_e(gc, i % ne); };
    double lmax = -INFINITY;
    for (long long g = threadIdx.x; g < npa; g += NT) lmax = fmax(lmax, lg[g]);
    lmax = block_max<NT>(lmax, red);
    __syncthreads();
    double Lm = 0.0;
    for (int i = threadIdx.x; i < np; i += NT) {
        double sL = 0.0, sA = 0.0;
        for (int k = 0; k < na; ++k) {
            const double v = lg[(size_t)i * na + k];
            if (v == -INFINITY) continue;
            const double t = qp[k] * (mixed ? (double)expf((float)(v - lmax)) : exp(v - lmax));
            sL += t;
            sA += t * alph[k];
        }
        Ls[i] = sL;
        As[i] = sA;
        Lm = fmax(Lm, sL);
    }
    const double Lmax = block_max<NT>(Lm, red);
    __syncthreads();
    double W = 0, m1 = 0, m2 = 0, WA = 0, Ws = 0, s1 = 0, s2 = 0, kept = 0;
    double lo1 = INFINITY, hi1 = -INFINITY, lo2 = INFINITY, hi2 = -INFINITY;
    for (int i = threadIdx.x; i < np; i += NT) {
        const double L = Ls[i];
        if (!(L > 0.0)) continue;
        const double e1 = e1_of(i), e2 = e2_of(i);
        Ws += L;
        s1 += L * e1;
        s2 += L * e2;
        if (L >= gc.thresh_frac * Lmax) {
            kept += 1.0;
            W += L;
            m1 += L * e1;
            m2 += L * e2;
            WA += As[i];
            lo1 = fmin(lo1, e1);
            hi1 = fmax(hi1, e1);
            lo2 = fmin(lo2, e2);
            hi2 = fmax(hi2, e2);
        }
    }
    W = block_sum<NT>(W, red);
    m1 = block_sum<NT>(m1, red);
    m2 = block_sum<NT>(m2, red);
    WA = block_sum<NT>(WA, red);
    Ws = block_sum<NT>(Ws, red);
    s1 = block_sum<NT>(s1, red);
    s2 = block_sum<NT>(s2, red);
    kept = block_sum<NT>(kept, red);
    lo1 = -block_max<NT>(-lo1, red);
    hi1 = block_max<NT>(hi1, red);
    lo2 = -block_max<NT>(-lo2, red);
    hi2 = block_max<NT>(hi2, red);
    const double e1m = W > 0 ? m1 / W : 0.0, e2m = W > 0 ? m2 / W : 0.0;
    double c11 = 0, c22 = 0, c12 = 0;
    for (int i = threadIdx.x; i < np; i += NT) {
        const double L = Ls[i];
        if (!(L > 0.0) || L < gc.thresh_frac * Lmax) continue;
        const double d1 = e1_of(i) - e1m, d2 = e2_of(i) - e2m;
        c11 += L * d1 * d1;
        c22 += L * d2 * d2;
        c12 += L * d1 * d2;
    }
    c11 = block_sum<NT>(c11, red);
    c22 = block_sum<NT>(c22, red);
    c12 = block_sum<NT>(c12, red);
    double best = -INFINITY;
    long long gbest = 0x7fffffffffffffffLL;
    for (long long g = threadIdx.x; g < npa; g += NT) {
        const double v = lg[g];
        if (v == -INFINITY) continue;
        const double lp = v + lnp[g % na];
        if (lp > best || (lp == best && g < gbest)) {
            best = lp;
            gbest = g;
        }
    }
    block_argmax<NT>(best, gbest, red, redi);
    if (threadIdx.x == 0) {
        if (W > 0) {
            c11 /= W;
            c22 /= W;
            c12 /= W;
        }
        const double det = c11 * c22 - c12 * c12;
        res.e1m = e1m;
        res.e2m = e2m;
        res.sd1 = sqrt(c11);
        res.sd2 = sqrt(c22);
        const double sdet = det > 0 ? sqrt(det) : 0.0;
        res.bad = !(W > 0) || res.sd1 <= gc.var_sigma_min || res.sd2 <= gc.var_sigma_min || sdet <= gc.var_det_min;
        res.am = W > 0 ? WA / W : 0.0;
        res.flux = (best > -INFINITY && a[gbest] > 0) ? b[gbest] / a[gbest] : 0.0;
        res.e1s = Ws > 0 ? s1 / Ws : 0.0;
        res.e2s = Ws > 0 ? s2 / Ws : 0.0;
        res.kept = (int)kept;
        res.map_i = best > -INFINITY ? (int)(gbest / na) : -1;
        res.box[0] = lo1;
        res.box[1] = hi1;
        res.box[2] = lo2;
        res.box[3] = hi2;
    }
    __syncthreads();
}

// quadrature weights qp_k (trapezoid in alpha times the lognormal prior of Eq. 4), the
// nodes alpha_k and the log prior lnp_k of the scalelength grid (threads k < n_alpha)
__device__ void alpha_weights(const GridConst &gc, const SrcRow &S, double *qp, double *alph, double *lnp)
{
    const int na = gc.n_alpha;
    if (threadIdx.x < na) {
        const int k = threadIdx.x;
        const double ak = grid_alpha(gc, k);
        double q;
        if (na == 1) q = 1.0;
        else if (k == 0) q = 0.5 * (grid_alpha(gc, 1) - ak);
        else if (k == na - 1) q = 0.5 * (ak - grid_alpha(gc, na - 2));
        else q = 0.5 * (grid_alpha(gc, k + 1) - grid_alpha(gc, k - 1));
        const double z = (log(ak) - S.mu) / gc.r_std;
        qp[k] = q * exp(-0.5 * z * z) / (ak * gc.r_std * sqrt(2.0 * kPi));
        alph[k] = ak;
        lnp[k] = -0.5 * z * z - log(ak);
    }
}

// exclusive prefix sum over the NT threads of a block, in thread order; *total gets
// the sum (scratch: NT / 32 + 1 ints)
template <int NT>
__device__ int block_exclusive_scan(int x, int *scratch, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __syncthreads();
    if (lane == 31) scratch[wid] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < NT / 32; ++w) {
        if (w < wid) before += scratch[w];
        all += scratch[w];
    }
    *total = all;
    return before + incl - x;
}

// The next lattice (one thread): every multiple of hn = h / 2 in the box of the kept
// samples widened by h, |e| < 1, at most kAdaptSide per component around the MAP
// sample; returns the number of samples written to e1s, e2s.
__device__ int plan_lattice(const GridConst &gc, const AdaptResult &res, int level, double h, double *e1s, double *e2s,
                            short *i1s = nullptr, short *i2s = nullptr, int *lo_out = nullptr, int *hi_out = nullptr)
{
    const int ne = gc.n_e;
    const double hn = 0.5 * h;
    const double cen[2] = {level == 0 ? grid_e(gc, res.map_i / ne) : e1s[res.map_i],
                           level == 0 ? grid_e(gc, res.map_i % ne) : e2s[res.map_i]};
    int lo[2], hi[2];
    for (int d = 0; d < 2; ++d) {
        lo[d] = (int)ceil((res.box[2 * d] - h) / hn - 1e-9);
        hi[d] = (int)floor((res.box[2 * d + 1] + h) / hn + 1e-9);
        if (hi[d] - lo[d] + 1 > kAdaptSide) {
            const int c = (int)llround(cen[d] / hn);
            lo[d] = c - kAdaptSide / 2;
            hi[d] = c + kAdaptSide / 2;
        }
    }
    int np = 0;
    for (int i1 = lo[0]; i1 <= hi[0]; ++i1)
        for (int i2 = lo[1]; i2 <= hi[1]; ++i2) {
            const double a1 = i1 * hn, a2 = i2 * hn;
            if (!(a1 * a1 + a2 * a2 < 1.0)) continue;
            e1s[np] = a1;
            e2s[np] = a2;
            if (i1s) {
                i1s[np] = (short)i1;
                i2s[np] = (short)i2;
            }
            ++np;
        }
    if (lo_out) {
        lo_out[0] = lo[0];
        lo_out[1] = lo[1];
        hi_out[0] = hi[0];
        hi_out[1] = hi[1];
    }
    return np;
}

// the last level's estimate as the fit result of facet s (one thread)
__device__ void write_adapt_result(const AdaptResult &res, const SrcRow &S, int level, int s, const rlf_fit_out &out,
                                   int32_t out_offset)
{
    int flag = res.bad ? RLF_FLAG_BAD : 0;
    if (S.invalid) flag |= RLF_FLAG_INVALID;
    const int o = out_offset + s;
    out.e1[o] = res.e1m;
    out.e2[o] = res.e2m;
    out.sig1[o] = res.sd1;
    out.sig2[o] = res.sd2;
    out.alpha_arcsec[o] = res.am;
    out.flux_jy[o] = res.flux;
    out.e1_smooth[o] = res.e1s;
    out.e2_smooth[o] = res.e2s;
    out.flag[o] = flag | (level << RLF_FLAG_LEVELS_SHIFT);
}

// One CTA per facet (the position marginal and the FP64 form): each thread one
// (sample, alpha) pair over all of the facet's cells, level after level.
template <typename T, bool kGauss, int NJ>
__global__ void __launch_bounds__(kAT, 1)
adaptive_kernel(const T *__restrict__ cells, const int32_t *__restrict__ ncell, const SrcRow *__restrict__ table,
                size_t plane, int32_t NN, const GridConst gc, const double *__restrict__ ga,
                const double *__restrict__ gb, const double *__restrict__ gl, const double *__restrict__ ccv,
                double *__restrict__ scratch, rlf_fit_out out, int32_t out_offset)
{
    constexpr bool mixed = std::is_same<T, float>::value;
    const bool split = gc.split != 0;
    const bool fp32_norm = mixed && split;   // FP32 logarithms, error functions and exponentials
    // cells per staged tile: uu, uv, vv, A and NJ B planes (B per position offset)
    constexpr int kTA = (NJ > 1 && !mixed) ? kCellTile / 2 : kCellTile;
    constexpr int NB = NJ > 1 ? (NJ + 3) / 4 * 4 : 1;   // B values per cell (b_stride)
    __shared__ T sm[NJ > 1 ? 4 : 5][kTA];
    __shared__ __align__(16) T sbr[NJ > 1 ? kTA : 1][NB];
    __shared__ double qp[64], alph[64], lnp[64];
    __shared__ double Ls[kMaxNe * kMaxNe > kAdaptMax ? kMaxNe * kMaxNe : kAdaptMax];
    __shared__ double As[kMaxNe * kMaxNe > kAdaptMax ? kMaxNe * kMaxNe : kAdaptMax];
    __shared__ double e1s[kAdaptMax], e2s[kAdaptMax];
    __shared__ AdaptResult res;
    __shared__ int s_np;
    const int s = blockIdx.x;
    const int ne = gc.n_e, na = gc.n_alpha;
    const size_t ng = (size_t)ne * ne * na;
    const SrcRow S = table[s];
    const int nc = ncell[s];
    const double cc = ccv[s];
    alpha_weights(gc, S, qp, alph, lnp);
    __syncthreads();
    // level 0: the grid
    estimate_over_samples<kAT>(fp32_norm, ne * ne, nullptr, nullptr, gl + s * ng, ga + s * ng, gb + s * ng, gc, qp, alph,
                          lnp, Ls, As, res);
    double h = 2.0 * gc.e_max / (ne - 1);
    int level = 0;
    double *slg = scratch + (size_t)s * adapt_doubles_per_facet(na);
    double *sa = slg + (size_t)kAdaptMax * na, *sb = sa + (size_t)kAdaptMax * na;
    while (res.kept < gc.np_max && h > gc.e_res && res.map_i >= 0 && nc > 0) {
        // the next lattice (thread 0), then every (sample, alpha) pair over the cells
        const double hn = 0.5 * h;
        if (threadIdx.x == 0) s_np = plan_lattice(gc, res, level, h, e1s, e2s);
        __syncthreads();
        const int np = s_np;
        const T *cu = cells + (size_t)s * NN;
        for (int base = 0; base < np * na; base += kAT) {
            const int pr = base + threadIdx.x;
            const bool on = pr < np * na;
            const int i = on ? pr / na : 0, k = on ? pr % na : 0;
            const double e1 = e1s[i], e2 = e2s[i];
            const double det = 1.0 - e1 * e1 - e2 * e2;
            const double id2 = 1.0 / (det * det);
            const T p11 = (T)(((1.0 + e1) * (1.0 + e1) + e2 * e2) * id2);
            const T p12 = (T)(4.0 * e2 * id2);
            const T p22 = (T)(((1.0 - e1) * (1.0 - e1) + e2 * e2) * id2);
            const double alr = alph[k] * kArcsec * S.du;
            const T ca = (T)(4.0 * kPi * kPi * alr * alr);
            float ah = 0.0f, al = 0.0f, bh[NJ], bl[NJ];
            double da = 0.0, db[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                bh[j] = bl[j] = 0.0f;
                db[j] = 0.0;
            }
            for (int c0 = 0; c0 < nc; c0 += kTA) {
                const int nt = min(kTA, nc - c0);
                __syncthreads();
                for (int j = threadIdx.x; j < nt; j += kAT) {
#pragma unroll
                    for (int q = 0; q < (NJ > 1 ? 4 : 5); ++q) sm[q][j] = cu[q * plane + c0 + j];
                }
                if constexpr (NJ > 1) {
                    const T *brow = cells + 4 * plane + ((size_t)s * NN + c0) * NB;
                    for (int i = threadIdx.x; i < nt * NB; i += kAT) (&sbr[0][0])[i] = brow[i];
                }
                __syncthreads();
                if (!on) continue;
                T pa = T(0), pb[NJ];
#pragma unroll
                for (int j = 0; j < NJ; ++j) pb[j] = T(0);
                for (int c = 0; c < nt; ++c) {
                    const T Q = p11 * sm[0][c] + p12 * sm[1][c] + p22 * sm[2][c];
                    T M;
                    if constexpr (mixed) M = brightness<kGauss>(ca, Q);
                    else M = brightness64(ca * Q, kGauss ? RLF_PROFILE_GAUSSIAN : RLF_PROFILE_EXPONENTIAL);
                    pa += sm[3][c] * M * M;
                    if constexpr (NJ == 1) {
                        pb[0] += sm[4][c] * M;
                    } else {
#pragma unroll
                        for (int j = 0; j < NJ; ++j) pb[j] += sbr[c][j] * M;
                    }
                }
                if constexpr (mixed) {
                    acc_add(split, ah, al, pa);
#pragma unroll
                    for (int j = 0; j < NJ; ++j) acc_add(split, bh[j], bl[j], pb[j]);
                } else {
                    da += (double)pa;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) db[j] += (double)pb[j];
                }
            }
            if (on) {
                if constexpr (mixed) {
                    da = acc_value(split, ah, al);
#pragma unroll
                    for (int j = 0; j < NJ; ++j) db[j] = acc_value(split, bh[j], bl[j]);
                }
                sa[pr] = da;
                if constexpr (NJ == 1) {
                    sb[pr] = db[0];
                    slg[pr] = fp32_norm ? flux_marginal_mixed(da, db[0], cc, gc.flux_prior)
                                        : flux_marginal(da, db[0], cc, gc.flux_prior);
                } else {
                    double bb;
                    if (fp32_norm) slg[pr] = position_marginal_ff<NJ>(da, bh, bl, cc, gc.flux_prior, bb);
                    else slg[pr] = position_marginal<NJ>(da, db, cc, gc.flux_prior, bb);
                    sb[pr] = bb;
                }
            }
        }
        __threadfence_block();
        __syncthreads();
        estimate_over_samples<kAT>(fp32_norm, np, e1s, e2s, slg, sa, sb, gc, qp, alph, lnp, Ls, As, res);
        h = hn;
        ++level;
    }
    if (level > 0 && threadIdx.x == 0) write_adapt_result(res, S, level, s, out, out_offset);
}

// The FP32 form with one position (the common case) as a cluster of kAdaptR CTAs per
// facet (facets in the grid fit's order, most cells first), so that the serial levels
// of a facet with many cells spread over several SMs.  Rank r sums the lattice's new
// (sample, alpha) pairs over its share of the facet's 128-cell tiles (the tiles cut as
// in the grid's parts), four scalelength nodes per thread with the quadratic form of
// a cell once for them (two nodes per paired FP32 instruction; tile sums added to
// float pairs), and stores its partial a, b per pair (FP64) in the facet's scratch.
// The leader (rank 0) runs the estimate: it adds the ranks' partials in rank order,
// forms ln L, estimates over the samples and writes the next lattice.  A sample the
// lattice shares with the previous one (even multiples of the new step: the same e
// bit for bit, hence the same sums) is not evaluated again; the leader copies its a,
// b and ln L.  Hardware cluster barriers order the steps (no polling).  Scratch per
// facet (adapt_doubles_per_facet): ln L, a, b [2 levels][kAdaptMax][na]; partial a, b
// [kAdaptRanks >= kAdaptR][kAdaptMax][na][2]; lattice e1, e2 [kAdaptMax]; the samples
// to evaluate [kAdaptMax] (int); control words.
template <bool kGauss>
__global__ void __cluster_dims__(kAdaptR, 1, 1) __launch_bounds__(kATc, kATcBlocks)
adaptive_cluster_kernel(const float *__restrict__ cells, const int32_t *__restrict__ ncell,
                        const SrcRow *__restrict__ table, size_t plane, int32_t NN, const GridConst gc,
                        const double *__restrict__ ga, const double *__restrict__ gb, const double *__restrict__ gl,
                        const double *__restrict__ ccv, const int32_t *__restrict__ order,
                        double *__restrict__ scratch, rlf_fit_out out, int32_t out_offset)
{
    namespace cg = cooperative_groups;
    const cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const bool leader = rank == 0;
    const bool split = gc.split != 0;   // FP32 logarithms, error functions and exponentials in split mode
    __shared__ float sm[5][kCellTile];
    __shared__ double qp[64], alph[64], lnp[64];
    __shared__ double Ls[kMaxNe * kMaxNe > kAdaptMax ? kMaxNe * kMaxNe : kAdaptMax];
    __shared__ double As[kMaxNe * kMaxNe > kAdaptMax ? kMaxNe * kMaxNe : kAdaptMax];
    __shared__ double e1s[kAdaptMax], e2s[kAdaptMax];
    __shared__ int elist[kAdaptMax];                 // samples to evaluate
    __shared__ short li1[kAdaptMax], li2[kAdaptMax];   // leader: integer coordinates of the samples
    __shared__ short src[kAdaptMax];                 // leader: the previous lattice's sample, or -1
    __shared__ short pmap[kAdaptMax];                // leader: the lattice's box -> sample (-1: |e| >= 1)
    __shared__ int plo[2], pw;                       // leader: that box's origin and e2 width
    __shared__ int box_lo[2], box_hi[2], scan_tmp[kATc / 32 + 1];
    __shared__ AdaptResult res;
    const int s = order[blockIdx.x / kAdaptR];   // facets with the most cells first
    const int ne = gc.n_e, na = gc.n_alpha;
    const size_t ng = (size_t)ne * ne * na, nsa = (size_t)kAdaptMax * na;
    const SrcRow S = table[s];
    const int nc = ncell[s];
    const double cc = ccv[s];
    double *base = scratch + (size_t)s * adapt_doubles_per_facet(na);   // ln L, a, b of two levels
    double *part = base + 6 * nsa;                                      // [rank][pair][2]
    double *lat = part + (size_t)kAdaptRanks * nsa * 2;                 // e1 [kAdaptMax], e2 [kAdaptMax]
    int *glist = reinterpret_cast<int *>(lat + 2 * kAdaptMax);          // samples to evaluate [kAdaptMax]
    int *ctl = glist + kAdaptMax;                                       // samples, samples to evaluate
    // this rank's tiles of the facet's cells
    const int n_tiles = (nc + kCellTile - 1) / kCellTile;
    const int c_begin = (int)((int64_t)n_tiles * rank / kAdaptR) * kCellTile;
    const int c_end = min(nc, (int)((int64_t)n_tiles * (rank + 1) / kAdaptR) * kCellTile);
    alpha_weights(gc, S, qp, alph, lnp);
    __syncthreads();
    double h = 2.0 * gc.e_max / (ne - 1);
    int level = 0;
    // The next lattice from the estimate `res` of level `level` at step h (every thread
    // of the leader): the samples of plan_lattice in its order (e1 outer, e2 inner), which
    // of them the previous lattice holds, the list to evaluate.  Candidates of the box
    // are split over the threads in order and placed by a prefix sum.
    constexpr int kPer = (kAdaptMax + kATc - 1) / kATc;   // candidates per thread
    auto plan = [&](bool more) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int lo[2] = {0, 0}, hi[2] = {-1, -1};
            if (more) {
                // the box as plan_lattice makes it (the centre read before e1s, e2s change)
                const double hn = 0.5 * h;
                const double cen[2] = {level == 0 ? grid_e(gc, res.map_i / ne) : e1s[res.map_i],
                                       level == 0 ? grid_e(gc, res.map_i % ne) : e2s[res.map_i]};
                for (int d = 0; d < 2; ++d) {
                    lo[d] = (int)ceil((res.box[2 * d] - h) / hn - 1e-9);
                    hi[d] = (int)floor((res.box[2 * d + 1] + h) / hn + 1e-9);
                    if (hi[d] - lo[d] + 1 > kAdaptSide) {
                        const int c = (int)llround(cen[d] / hn);
                        lo[d] = c - kAdaptSide / 2;
                        hi[d] = c + kAdaptSide / 2;
                    }
                }
            }
            box_lo[0] = lo[0];
            box_lo[1] = lo[1];
            box_hi[0] = hi[0];
            box_hi[1] = hi[1];
        }
        __syncthreads();
        const double hn = 0.5 * h;
        const int w2 = box_hi[1] - box_lo[1] + 1;
        const int total = (box_hi[0] - box_lo[0] + 1) * w2;   // at most kAdaptMax
        // this thread's candidates, kept when |e| < 1
        bool keep[kPer];
        int n_keep = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int c = threadIdx.x * kPer + q;
            keep[q] = false;
            if (c < total) {
                const double a1 = (box_lo[0] + c / w2) * hn, a2 = (box_lo[1] + c % w2) * hn;
                keep[q] = a1 * a1 + a2 * a2 < 1.0;
            }
            n_keep += keep[q] ? 1 : 0;
        }
        int np;
        int pos = block_exclusive_scan<kATc>(n_keep, scan_tmp, &np);
        // place the samples; find each one in the previous lattice's map
        int n_new = 0;
        int from_q[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            from_q[q] = -1;
            if (!keep[q]) continue;
            const int c = threadIdx.x * kPer + q;
            const int i1 = box_lo[0] + c / w2, i2 = box_lo[1] + c % w2;
            e1s[pos] = i1 * hn;
            e2s[pos] = i2 * hn;
            li1[pos] = (short)i1;
            li2[pos] = (short)i2;
            if (level >= 1 && (i1 & 1) == 0 && (i2 & 1) == 0) {
                const int j1 = i1 / 2 - plo[0], j2 = i2 / 2 - plo[1];
                if (j1 >= 0 && j2 >= 0 && j2 < pw && (j1 + 1) * pw <= kAdaptMax) from_q[q] = pmap[j1 * pw + j2];
            }
            src[pos] = (short)from_q[q];
            n_new += from_q[q] < 0 ? 1 : 0;
            ++pos;
        }
        int n_eval;
        int epos = block_exclusive_scan<kATc>(n_new, scan_tmp, &n_eval);
        pos -= n_keep;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            if (!keep[q]) continue;
            if (from_q[q] < 0) {
                elist[epos] = pos;
                glist[epos] = pos;
                ++epos;
            }
            lat[pos] = e1s[pos];
            lat[kAdaptMax + pos] = e2s[pos];
            ++pos;
        }
        __syncthreads();
        // this lattice's box -> sample map, for the next level (the box is at most
        // kAdaptSide per side, so it fits)
        for (int i = threadIdx.x; i < kAdaptMax; i += kATc) pmap[i] = -1;
        __syncthreads();
        for (int i = threadIdx.x; i < np; i += kATc) pmap[(li1[i] - box_lo[0]) * w2 + (li2[i] - box_lo[1])] = (short)i;
        if (threadIdx.x == 0) {
            plo[0] = box_lo[0];
            plo[1] = box_lo[1];
            pw = w2;
            ctl[0] = np;
            ctl[1] = n_eval;
        }
    };
    if (leader) {
        // level 0: the grid
        estimate_over_samples<kATc>(split, ne * ne, nullptr, nullptr, gl + s * ng, ga + s * ng, gb + s * ng, gc, qp,
                                    alph, lnp, Ls, As, res);
        plan(res.kept < gc.np_max && h > gc.e_res && res.map_i >= 0 && nc > 0);
    }
    constexpr int kAG = 4;
    const int n_ag = (na + kAG - 1) / kAG;
    const f32x2 one2 = pk2(1.0f, 1.0f), zero2 = pk2(0.0f, 0.0f);
    const float *cu = cells + (size_t)s * NN;
    for (;;) {
        __threadfence();
        cluster.sync();
        const int np = reinterpret_cast<volatile int *>(ctl)[0];
        const int n_eval = reinterpret_cast<volatile int *>(ctl)[1];
        if (np == 0) break;
        if (!leader) {
            for (int i = threadIdx.x; i < np; i += kATc) {
                e1s[i] = lat[i];
                e2s[i] = lat[kAdaptMax + i];
            }
            for (int i = threadIdx.x; i < n_eval; i += kATc) elist[i] = glist[i];
        }
        __syncthreads();
        // this rank's partial sums of every new (sample, alpha) pair
        for (int b0 = 0; b0 < n_eval * n_ag; b0 += kATc) {
            const int it = b0 + threadIdx.x;
            const bool on = it < n_eval * n_ag;
            const int i = on ? elist[it / n_ag] : 0, g = on ? it % n_ag : 0;
            const double e1 = e1s[i], e2 = e2s[i];
            const double det = 1.0 - e1 * e1 - e2 * e2;
            const double id2 = 1.0 / (det * det);
            const float p11 = (float)(((1.0 + e1) * (1.0 + e1) + e2 * e2) * id2);
            const float p12 = (float)(4.0 * e2 * id2);
            const float p22 = (float)(((1.0 - e1) * (1.0 - e1) + e2 * e2) * id2);
            float cak[kAG];
#pragma unroll
            for (int j = 0; j < kAG; ++j) {
                const int k = g * kAG + j;
                const double alr = (k < na ? alph[k] : 0.0) * kArcsec * S.du;
                cak[j] = (float)(4.0 * kPi * kPi * alr * alr) * (kGauss ? -0.25f : 1.0f);
            }
            const f32x2 c2[2] = {pk2(cak[0], cak[1]), pk2(cak[2], cak[3])};
            float ah[kAG], al[kAG], bh[kAG], bl[kAG];
#pragma unroll
            for (int j = 0; j < kAG; ++j) ah[j] = al[j] = bh[j] = bl[j] = 0.0f;
            for (int c0 = c_begin; c0 < c_end; c0 += kCellTile) {
                const int nt = min(kCellTile, c_end - c0);
                __syncthreads();
                for (int j = threadIdx.x; j < nt; j += kATc) {
#pragma unroll
                    for (int q = 0; q < 5; ++q) sm[q][j] = cu[q * plane + c0 + j];
                }
                __syncthreads();
                if (!on) continue;
                f32x2 pa2[2] = {zero2, zero2}, pb2[2] = {zero2, zero2};
                for (int c = 0; c < nt; ++c) {
                    const float Q = p11 * sm[0][c] + p12 * sm[1][c] + p22 * sm[2][c];
                    const f32x2 Q2 = pk2(Q, Q), A2 = pk2(sm[3][c], sm[3][c]), B2 = pk2(sm[4][c], sm[4][c]);
#pragma unroll
                    for (int j2 = 0; j2 < 2; ++j2) {
                        float x0, x1;
                        f32x2 M2;
                        if (kGauss) {
                            up2(mul2(c2[j2], Q2), x0, x1);
                            M2 = pk2(ex2_approx(x0), ex2_approx(x1));
                        } else {
                            up2(fma2(c2[j2], Q2, one2), x0, x1);
                            const f32x2 r2 = pk2(rsqrtf(x0), rsqrtf(x1));
                            M2 = mul2(mul2(r2, r2), r2);
                        }
                        pa2[j2] = fma2(mul2(A2, M2), M2, pa2[j2]);
                        pb2[j2] = fma2(B2, M2, pb2[j2]);
                    }
                }
#pragma unroll
                for (int j2 = 0; j2 < 2; ++j2) {
                    float a0, a1, b0v, b1v;
                    up2(pa2[j2], a0, a1);
                    up2(pb2[j2], b0v, b1v);
                    acc_add(split, ah[2 * j2], al[2 * j2], a0);
                    acc_add(split, ah[2 * j2 + 1], al[2 * j2 + 1], a1);
                    acc_add(split, bh[2 * j2], bl[2 * j2], b0v);
                    acc_add(split, bh[2 * j2 + 1], bl[2 * j2 + 1], b1v);
                }
            }
            if (on) {
#pragma unroll
                for (int j = 0; j < kAG; ++j) {
                    const int k = g * kAG + j;
                    if (k >= na) break;
                    double *pp = part + ((size_t)rank * nsa + (size_t)i * na + k) * 2;
                    pp[0] = acc_value(split, ah[j], al[j]);
                    pp[1] = acc_value(split, bh[j], bl[j]);
                }
            }
        }
        __threadfence();
        cluster.sync();
        if (leader) {
            // the pairs' a and b (partials added in rank order, or the previous level's
            // values of a shared sample) and ln L, then the estimate
            const int cur = (level + 1) & 1;
            double *slg = base + (size_t)cur * 3 * nsa, *sa = slg + nsa, *sb = sa + nsa;
            const double *plg = base + (size_t)(cur ^ 1) * 3 * nsa, *pa = plg + nsa, *pb = pa + nsa;
            for (int pr = threadIdx.x; pr < np * na; pr += kATc) {
                const int i = pr / na, k = pr % na;
                const int from = src[i];
                if (from >= 0) {
                    const size_t q = (size_t)from * na + k;
                    slg[pr] = plg[q];
                    sa[pr] = pa[q];
                    sb[pr] = pb[q];
                    continue;
                }
                double da = 0.0, db = 0.0;
#pragma unroll
                for (int r = 0; r < kAdaptR; ++r) {
                    const double *pp = part + ((size_t)r * nsa + pr) * 2;
                    da += pp[0];
                    db += pp[1];
                }
                sa[pr] = da;
                sb[pr] = db;
                slg[pr] = split ? flux_marginal_mixed(da, db, cc, gc.flux_prior)
                                : flux_marginal(da, db, cc, gc.flux_prior);
            }
            __threadfence_block();
            __syncthreads();
            estimate_over_samples<kATc>(split, np, e1s, e2s, slg, sa, sb, gc, qp, alph, lnp, Ls, As, res);
            ++level;
            h *= 0.5;
            plan(res.kept < gc.np_max && h > gc.e_res && res.map_i >= 0);
        }
    }
    if (leader && level > 0 && threadIdx.x == 0) write_adapt_result(res, S, level, s, out, out_offset);
}

}  // namespace

namespace {

// Facets whose sub-box fit must be redone on the full grid: the proposal was too
// wide or the box's estimate found mass near the threshold on an inner face (both
// in `wide`), or the MAP point lies on a face of the box that is not a face of the grid.
__global__ void refit_list_kernel(const int32_t *__restrict__ box, const int32_t *__restrict__ wide,
                                  const int32_t *__restrict__ map_index, int32_t count, int32_t ne, int32_t na,
                                  int32_t *__restrict__ refit)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    bool again = wide[s] != 0;
    const int g = map_index[s];
    if (!again && g >= 0) {
        const int i1 = g / (ne * na), i2 = (g / na) % ne, k = g % na;
        const int o1 = box[s * 3], o2 = box[s * 3 + 1], ok = box[s * 3 + 2];
        again = (i1 == o1 && o1 > 0) || (i1 == o1 + kBoxE - 1 && o1 + kBoxE < ne) ||
                (i2 == o2 && o2 > 0) || (i2 == o2 + kBoxE - 1 && o2 + kBoxE < ne) ||
                (k == ok && ok > 0) || (k == ok + kBoxA - 1 && ok + kBoxA < na);
    }
    if (again) refit[1 + atomicAdd(&refit[0], 1)] = s;
}

template <typename T, int AG>
cudaError_t launch_persistent(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                              const int32_t *count_dev, const int32_t *order, GridConst gc, const rlf_params &p,
                              const Workspace &ws, const rlf_fit_out &out, int32_t out_offset, int32_t *map_out,
                              cudaStream_t st)
{
    gc.n_ag = gc.box ? (kBoxA + AG - 1) / AG : (gc.n_alpha + AG - 1) / AG;
    const int pairs = (gc.box ? kBoxE * kBoxE : gc.n_e * gc.n_e) * gc.n_ag;
    const int tiles = (pairs + kThreads - 1) / kThreads;
    auto kern = gc.profile == RLF_PROFILE_GAUSSIAN ? fit_persistent_kernel<T, AG, true>
                                                   : fit_persistent_kernel<T, AG, false>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (p.tune_fit_blocks > 0 && p.tune_fit_blocks < per_sm) per_sm = p.tune_fit_blocks;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // one full wave: with fewer (facet, tile) items than CTAs the kernel splits cells
    const int64_t grid = (int64_t)sms * per_sm;
    if ((e = cudaMemsetAsync(ws.counters, 0, (size_t)(count + 1) * sizeof(int32_t), st)) != cudaSuccess) return e;
    if (!order) {
        lpt_order_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, st>>>(ws.ncell, count, ws.order);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        order = ws.order;
    }
    kern<<<(int)grid, kThreads, 0, st>>>(cells, ws.ncell, table, plane, NN, tiles, count, count_dev, order,
                                         ws.counters, gc, ws.ga, ws.gb, ws.part_stride, ws.fit_parts, ws.gl, ws.cc, out,
                                         out_offset, ws.status, map_out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_persistent_ag(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                                 const int32_t *count_dev, const int32_t *order, const GridConst &gc,
                                 const rlf_params &p, const Workspace &ws, const rlf_fit_out &out,
                                 int32_t out_offset, int32_t *map_out, cudaStream_t st)
{
    switch (p.tune_fit_ag) {
    case 2:
        return launch_persistent<T, 2>(cells, table, plane, NN, count, count_dev, order, gc, p, ws, out, out_offset,
                                       map_out, st);
    case 8:
        return launch_persistent<T, 8>(cells, table, plane, NN, count, count_dev, order, gc, p, ws, out, out_offset,
                                       map_out, st);
    default:
        return launch_persistent<T, 4>(cells, table, plane, NN, count, count_dev, order, gc, p, ws, out, out_offset,
                                       map_out, st);
    }
}

template <typename T, int NJ>
cudaError_t launch_adaptive_nj(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                               const GridConst &gc, const Workspace &ws, const rlf_fit_out &out, int32_t out_offset,
                               cudaStream_t st)
{
    if constexpr (std::is_same<T, float>::value && NJ == 1) {
        auto kern = gc.profile == RLF_PROFILE_GAUSSIAN ? adaptive_cluster_kernel<true> : adaptive_cluster_kernel<false>;
        kern<<<count * kAdaptR, kATc, 0, st>>>(cells, ws.ncell, table, plane, NN, gc, ws.ga, ws.gb, ws.gl, ws.cc,
                                               ws.order, ws.adapt, out, out_offset);
    } else {
        auto kern = gc.profile == RLF_PROFILE_GAUSSIAN ? adaptive_kernel<T, true, NJ> : adaptive_kernel<T, false, NJ>;
        kern<<<count, kAT, 0, st>>>(cells, ws.ncell, table, plane, NN, gc, ws.ga, ws.gb, ws.gl, ws.cc, ws.adapt, out,
                                    out_offset);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adaptive(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                            const GridConst &gc, const Workspace &ws, const rlf_fit_out &out, int32_t out_offset,
                            cudaStream_t st)
{
    switch (gc.n_pos) {
    case 3: return launch_adaptive_nj<T, 9>(cells, table, plane, NN, count, gc, ws, out, out_offset, st);
    case 5: return launch_adaptive_nj<T, 25>(cells, table, plane, NN, count, gc, ws, out, out_offset, st);
    default: return launch_adaptive_nj<T, 1>(cells, table, plane, NN, count, gc, ws, out, out_offset, st);
    }
}

template <typename T, int NJ>
cudaError_t launch_persistent_pos(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                                  const GridConst &gc, const rlf_params &p, const Workspace &ws,
                                  const rlf_fit_out &out, int32_t out_offset, cudaStream_t st)
{
    const int pairs = gc.n_e * gc.n_e * (kPos2<T, NJ> ? (gc.n_alpha + kPosNodes - 1) / kPosNodes : gc.n_alpha);
    const int tiles = (pairs + kThreads - 1) / kThreads;
    auto kern = gc.profile == RLF_PROFILE_GAUSSIAN ? fit_persistent_pos_kernel<T, NJ, true>
                                                   : fit_persistent_pos_kernel<T, NJ, false>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (p.tune_fit_blocks > 0 && p.tune_fit_blocks < per_sm) per_sm = p.tune_fit_blocks;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)count * tiles, wave = (int64_t)sms * per_sm;
    const int grid = (int)(items < wave ? items : wave);
    if ((e = cudaMemsetAsync(ws.counters, 0, (size_t)(count + 1) * sizeof(int32_t), st)) != cudaSuccess) return e;
    lpt_order_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, st>>>(ws.ncell, count, ws.order);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    kern<<<grid, kThreads, 0, st>>>(cells, ws.ncell, table, plane, NN, tiles, count, ws.order, ws.counters, gc, ws.ga,
                                    ws.gb, ws.gl, ws.cc, out, out_offset, ws.status);
    return cudaGetLastError();
}

// the grid fit (and adaptive refinement) of `count` compacted facets
template <typename T>
cudaError_t launch_grid_fit(const T *cells, const SrcRow *table, size_t plane, int32_t NN, int32_t count,
                            const GridConst &gc, const rlf_params &p, const Workspace &ws, const rlf_fit_out &out,
                            int32_t out_offset, cudaStream_t st)
{
    cudaError_t e;
    if (gc.n_pos == 3)
        e = launch_persistent_pos<T, 9>(cells, table, plane, NN, count, gc, p, ws, out, out_offset, st);
    else if (gc.n_pos == 5)
        e = launch_persistent_pos<T, 25>(cells, table, plane, NN, count, gc, p, ws, out, out_offset, st);
    else if constexpr (std::is_same<T, float>::value)
        e = launch_persistent_ag<float>(cells, table, plane, NN, count, nullptr, nullptr, gc, p, ws, out, out_offset,
                                        nullptr, st);
    else
        e = launch_persistent<double, 4>(cells, table, plane, NN, count, nullptr, nullptr, gc, p, ws, out, out_offset,
                                         nullptr, st);
    if (e == cudaSuccess && p.estimator == RLF_ESTIMATOR_ADAPTIVE)
        e = launch_adaptive<T>(cells, table, plane, NN, count, gc, ws, out, out_offset, st);
    return e;
}

}  // namespace

namespace {

// The bad fits in source order, in one CTA: list[0] = their number, list[1..] = indices.
__global__ void bad_list_kernel(const int32_t *__restrict__ flag, int32_t n, int32_t *__restrict__ list)
{
    __shared__ int wsum[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const bool on = i < n && (flag[i] & RLF_FLAG_BAD);
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[w] = __popc(m);
        __syncthreads();
        int off = 0;
        for (int j = 0; j < w; ++j) off += wsum[j];
        if (on) list[1 + base + off + __popc(m & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base += off + __popc(m);
        __syncthreads();
    }
    if (threadIdx.x == 0) list[0] = base;
}

// Results of a refit chunk (rows t) back to their sources list[t], marked as refitted.
__global__ void scatter_kernel(const double *__restrict__ tmp, const int32_t *__restrict__ ftmp, size_t cap,
                               const int32_t *__restrict__ list, int32_t cnt, rlf_fit_out out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int i = list[t];
    out.e1[i] = tmp[t];
    out.e2[i] = tmp[cap + t];
    out.sig1[i] = tmp[2 * cap + t];
    out.sig2[i] = tmp[3 * cap + t];
    out.alpha_arcsec[i] = tmp[4 * cap + t];
    out.flux_jy[i] = tmp[5 * cap + t];
    out.e1_smooth[i] = tmp[6 * cap + t];
    out.e2_smooth[i] = tmp[7 * cap + t];
    out.flag[i] = ftmp[t] | RLF_FLAG_REFIT;
}

}  // namespace

cudaError_t launch_bad_list(const int32_t *flag, int32_t n, int32_t *list, cudaStream_t st)
{
    bad_list_kernel<<<1, 1024, 0, st>>>(flag, n, list);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const double *tmp, const int32_t *ftmp, size_t cap, const int32_t *list, int32_t cnt,
                           const rlf_fit_out &out, cudaStream_t st)
{
    scatter_kernel<<<(cnt + kThreads - 1) / kThreads, kThreads, 0, st>>>(tmp, ftmp, cap, list, cnt, out);
    return cudaGetLastError();
}

GridConst grid_const(const rlf_params &p)
{
    GridConst gc;
    gc.box = nullptr;
    gc.n_e = p.n_e;
    gc.n_alpha = p.n_alpha;
    gc.n_ag = 0;
    gc.flux_prior = p.flux_prior;
    gc.profile = p.profile;
    gc.n_pos = p.n_pos > 1 ? p.n_pos : 1;
    gc.pos_step = p.pos_step_arcsec * kArcsec;
    gc.estimator = p.estimator;
    gc.np_max = p.np_max;
    gc.e_res = p.e_res;
    gc.e_max = p.e_max;
    gc.r_min = p.r_min_arcsec;
    gc.r_max = p.r_max_arcsec;
    gc.r_std = p.r_std;
    gc.inv_sigma2 = 1.0 / (p.sigma_jy * p.sigma_jy);
    gc.thresh_frac = p.thresh_frac;
    gc.var_sigma_min = p.var_sigma_min;
    gc.var_det_min = p.var_det_min;
    gc.split = p.precision == RLF_PREC_MIXED_SPLIT ? 1 : 0;
    gc.pad_ = 0;
    gc.box_fail = nullptr;
    return gc;
}

cudaError_t launch_fit(const double *facets, const SrcRow *table, int32_t count,
                       const rlf_params &p, const Workspace &ws, const rlf_fit_out &out,
                       int32_t out_offset, cudaStream_t st)
{
    const int N = p.facet_n, NN = N * N;
    const GridConst gc = grid_const(p);
    const size_t plane = (size_t)count * NN;
    cudaError_t e;
    if (p.precision != RLF_PREC_FP64) {
        float *cells = static_cast<float *>(ws.cells);
        compact_kernel<float><<<count, kThreads, 0, st>>>(facets, table, N, gc.inv_sigma2, gc.n_pos, gc.pos_step,
                                                          plane, cells, ws.ncell, ws.cc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return launch_grid_fit<float>(cells, table, plane, NN, count, gc, p, ws, out, out_offset, st);
    }
    double *cells = static_cast<double *>(ws.cells);
    compact_kernel<double><<<count, kThreads, 0, st>>>(facets, table, N, gc.inv_sigma2, gc.n_pos, gc.pos_step, plane,
                                                       cells, ws.ncell, ws.cc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_grid_fit<double>(cells, table, plane, NN, count, gc, p, ws, out, out_offset, st);
}

cudaError_t launch_fit_mlp(const double *facets, const SrcRow *table, int32_t count, const rlf_params &p,
                           const Workspace &ws, const void *weights, const rlf_fit_out &out, int32_t *n_fallback,
                           cudaStream_t st)
{
    const int N = p.facet_n, NN = N * N;
    GridConst gc = grid_const(p);
    const size_t plane = (size_t)count * NN;
    float *cells = static_cast<float *>(ws.cells);
    compact_kernel<float><<<count, kThreads, 0, st>>>(facets, table, N, gc.inv_sigma2, 1, 0.0, plane, cells,
                                                      ws.ncell, ws.cc);
    cudaError_t e = cudaGetLastError();
    // the network's proposal of each facet's sub-box
    const MlpWeights W = mlp_weights(const_cast<void *>(weights));
    MlpScratch sc = mlp_scratch(ws.mlp_scratch, count);
    sc.status = ws.status;
    __half *x = static_cast<__half *>(ws.mlp_x);
    if (e == cudaSuccess) e = mlp_encode(facets, table, count, N, x, st);
    if (e == cudaSuccess) e = mlp_forward(W, x, count, sc, st);
    if (e == cudaSuccess) e = mlp_propose(sc.o, count, gc, ws.box, ws.wide, st);
    // the likelihood on every facet's sub-box
    // one scalelength node per thread: 7 x 7 x 5 = 245 of the CTA's 256 threads busy;
    // the estimate marks the boxes that cannot stand for the full grid in ws.wide
    gc.box = ws.box;
    gc.box_fail = ws.wide;
    if (e == cudaSuccess)
        e = launch_persistent<float, 1>(cells, table, plane, NN, count, nullptr, nullptr, gc, p, ws, out, 0,
                                        ws.map_index, st);
    // the facets that need the full grid, in one more persistent launch
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.refit, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) {
        refit_list_kernel<<<(count + kThreads - 1) / kThreads, kThreads, 0, st>>>(ws.box, ws.wide, ws.map_index,
                                                                                 count, p.n_e, p.n_alpha, ws.refit);
        e = cudaGetLastError();
    }
    gc.box = nullptr;
    gc.box_fail = nullptr;
    if (e == cudaSuccess)
        e = launch_persistent_ag<float>(cells, table, plane, NN, count, ws.refit, ws.refit + 1, gc, p, ws, out, 0,
                                        nullptr, st);
    if (e == cudaSuccess && n_fallback)
        e = cudaMemcpyAsync(n_fallback, ws.refit, sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
    return e;
}

}  // namespace rlf
