// Facet extraction (Sec. 2.3): residual isolation, phase shift to the source and
// averaging of the shifted visibilities into a facet_n x facet_n uv grid of
// cell side du = 1 / (K alpha).
//
// The residual of source i is D - V_sky + model_i; model_i carries the phase
// exp(+2 pi i phi_i), so after the shift it is the real number S s M(k) and
// x = (D - V_sky) exp(-2 pi i phi_i) + S s M(k).
//
// Mixed-precision kernel (extract_pair_kernel).  The residual D - V_sky is formed
// once per call (one streaming pass) and every source of the batch reads it.  A CTA
// owns (source, part) and keeps a private copy of the facet in shared memory; the
// part is an interleaved share of (block of baselines, channel group, time slice)
// units.  A lane walks one baseline's time series for two adjacent channels.  A
// baseline's uv track moves slowly (a few per cent of a cell per 60 s step at the
// facet sizes of the method), so consecutive visibilities of one channel usually
// fall in the same cell: the lane sums that run in registers and appends it to its
// own ring in shared memory only when the cell changes; the rings are drained into
// the facet with shared-memory atomics.  At the end the CTA stores its partial facet
// with plain coalesced stores, and facet_reduce_kernel sums the parts of each cell
// in FP64 in a fixed order (no global atomics).  Inside a CTA the drains land in
// varying order, so repeated runs agree to FP32 rounding.  blockIdx.x runs over the
// sources, so the CTAs reading the same baselines run together and share them
// through L2.
//
// Shared-memory planes: sum Re x, sum Im x (FP32), count (int32), and the sum of
// spec - spec_off (FP32, spec_off the band mean; the flush adds count * spec_off
// back in FP64, which keeps the rounding of cells with 1e5 visibilities far
// below 1e-6 relative).
//
// Cell index: both coordinates are computed in FP32 (u * (nu/c/du)); when the
// value lies within the FP32 error bound of a cell edge the index is recomputed
// in FP64 as floor((u * nu/c) / du), the definition, so the decision is the
// FP64 one.
#include <cmath>
#include <type_traits>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

__global__ void residual_kernel(const float4 *__restrict__ d, const float4 *__restrict__ s, int64_t n4,
                                float4 *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = d[i], b = s[i];
        out[i] = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
    }
}

// u, v, w as float pairs, one 32-byte record per row (two vector loads in the
// extraction); with `perm`, column j of every time step holds baseline perm[j] (rows
// are [time][stride] and n is a multiple of stride).
__global__ void split_uvw_kernel(const double *__restrict__ u, const double *__restrict__ v,
                                 const double *__restrict__ w, int64_t n, int32_t stride,
                                 const int32_t *__restrict__ perm, float *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm ? (i / stride) * stride + perm[i % stride] : i;
        float uh, ul, vh, vl, wh, wl;
        split_double(u[r], uh, ul);
        split_double(v[r], vh, vl);
        split_double(w[r], wh, wl);
        float4 *o = reinterpret_cast<float4 *>(out) + 2 * i;
        o[0] = make_float4(uh, ul, vh, vl);
        o[1] = make_float4(wh, wl, 0.0f, 0.0f);
    }
}

// Smallest Chebyshev extent max(|u|, |v|) (metres) of each baseline over time, rounded
// down to FP32: for every row r = b + t * stride, max(|u_r|, |v_r|) >= extent[b].
__global__ void track_extent_kernel(const double *__restrict__ u, const double *__restrict__ v, int64_t n_rows,
                                    int32_t stride, float *__restrict__ extent)
{
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < stride; b += gridDim.x * blockDim.x) {
        double m = 1.0e300;
        for (int64_t r = b; r < n_rows; r += stride) m = fmin(m, fmax(fabs(u[r]), fabs(v[r])));
        extent[b] = __double2float_rd(m);
    }
}

// Order bucket of an extent: 20 buckets per octave from 0.25 m (any monotone map works;
// the order only groups baselines of similar extent).
__device__ __forceinline__ int extent_bucket(float e)
{
    if (!(e > 0.25f)) return 0;
    const int b = (int)floorf((log2f(e) + 2.0f) * 20.0f);
    return b < kOrderBuckets - 1 ? b : kOrderBuckets - 1;
}

// Stable counting sort of the n baselines by extent bucket, in one CTA: thread t owns
// the contiguous index range [t * per, (t + 1) * per); counts[bucket][t] holds its
// bucket counts, then its output offsets; equal buckets keep index order, so the
// result is the same on every run.
__global__ void __launch_bounds__(kOrderThreads)
order_kernel(const float *__restrict__ extent, int32_t n, int32_t *__restrict__ counts, int32_t *__restrict__ perm)
{
    __shared__ int part[kOrderThreads];
    const int t = threadIdx.x;
    const int per = (n + kOrderThreads - 1) / kOrderThreads;
    const int j0 = min(n, t * per), j1 = min(n, j0 + per);
    for (int b = 0; b < kOrderBuckets; ++b) counts[b * kOrderThreads + t] = 0;
    for (int j = j0; j < j1; ++j) counts[extent_bucket(extent[j]) * kOrderThreads + t] += 1;
    __syncthreads();
    // exclusive scan of counts in (bucket, thread) order: thread t scans entries
    // [t * kOrderBuckets, (t + 1) * kOrderBuckets) of the flattened array
    const int e0 = t * kOrderBuckets, e1 = e0 + kOrderBuckets;
    int local = 0;
    for (int i = e0; i < e1; ++i) local += counts[i];
    part[t] = local;
    __syncthreads();
    for (int d = 1; d < kOrderThreads; d *= 2) {       // inclusive scan of the thread sums
        const int add = t >= d ? part[t - d] : 0;
        __syncthreads();
        part[t] += add;
        __syncthreads();
    }
    int run = part[t] - local;
    for (int i = e0; i < e1; ++i) {
        const int c = counts[i];
        counts[i] = run;
        run += c;
    }
    __syncthreads();
    for (int j = j0; j < j1; ++j) {
        int *slot = &counts[extent_bucket(extent[j]) * kOrderThreads + t];
        perm[*slot] = j;
        *slot += 1;
    }
}

// Baselines to walk per source: one past the last ordered position whose baseline
// can reach the facet window.  A baseline cannot when extent * s_min / du >= N / 2
// (with a 1e-12 margin): then at every row and channel |u| s / du or |v| s / du is at
// least N / 2, so floor(u s / du) or floor(v s / du) lies outside [-N/2, N/2).
__global__ void live_count_kernel(const float *__restrict__ extent, const int32_t *__restrict__ perm, int32_t n,
                                  const SrcRow *__restrict__ table, int32_t N, double s_min,
                                  int32_t *__restrict__ n_live)
{
    __shared__ int best[kThreads / 32];
    const double lim = 0.5 * N * table[blockIdx.x].du * (1.0 + 1.0e-12);
    int last = -1;
    for (int j = threadIdx.x; j < n; j += kThreads) {
        const int b = perm ? perm[j] : j;
        if ((double)extent[b] * s_min < lim) last = j;
    }
    for (int o = 16; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o));
    if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = last;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = -1;
        for (int w = 0; w < kThreads / 32; ++w) m = max(m, best[w]);
        n_live[blockIdx.x] = m + 1;
    }
}

// Cell of both coordinates from one paired FMA.  With off = 320 + N/2, m = fl(u) fl(s/du) +
// off, rounded once to the 2^-15 grid of [256, 512); a window coordinate t = u s / du in
// [-N/2, N/2) lands in [320, 320 + N), whose integer part minus 320 is the cell, and
// d = bits(m) - bits(320) holds it as d >> 15 with the fraction in the low 15 bits.  The
// product's error is below 2^-23 |t| < 4e-6 for |t| <= 33 (the window and one cell
// beyond), under half the grid step 2^-16, so away from an integer m rounds to the same
// side as the exact value and floor(t) is the definition's.  `edge` marks m on an
// integer (a zero fraction: t within ~2e-5 of a cell edge, including the window's own
// edges at 320 and 320 + N), where the caller takes the FP64 decision; `in` marks both
// coordinates inside the window.
__device__ __forceinline__ void cell_index2(float uh, float vh, float sdu, float off, int N, int &cell, bool &edge,
                                            bool &in)
{
    float mu, mv;
    up2(fma2(pk2(uh, vh), pk2(sdu, sdu), pk2(off, off)), mu, mv);
    const int du = __float_as_int(mu) - 0x43A00000, dv = __float_as_int(mv) - 0x43A00000;  // bits(320.0f)
    edge = ((du & 0x7fff) == 0) | ((dv & 0x7fff) == 0);
    in = max((unsigned)du, (unsigned)dv) < ((unsigned)N << 15);
    cell = (dv >> 15) * N + (du >> 15);
}

// A 16-byte shared-memory store under a predicate: the append of a finished run
// costs the same few instructions whether or not the lane appends, with no branch
// for the warp to diverge on.
__device__ __forceinline__ void st_shared_v4_if(uint32_t addr, bool p, int a, int b, int c, int d)
{
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared.v4.b32 [%1], {%2, %3, %4, %5}; }"
                 :: "r"((int)p), "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// ---- extraction by channel-pair lanes -------------------------------------------------
// A warp holds 32 / CL baselines x CL lanes; lane lc of a baseline walks two adjacent
// channels, k0 + 2 lc and k0 + 2 lc + 1 (k0 = the first channel of the lane group; more
// than 2 CL channels are split into groups), through time.  Each lane sums runs of equal
// cells of its two channels in registers (paired FP32 instructions: two channels per
// instruction for the phase, the rotation, the model and the run sums) and appends a
// finished run to its own ring in shared memory.  The per-row work of a baseline
// (float-pair phase argument, the group's phase f0 and step fd, the source's quadratic
// form, u and v in FP32) is shared by its CL lanes: for a block of CL time steps lane lc
// computes row t0 + lc and stores it in shared memory, and every lane then reads each
// row of the block (a broadcast).  The next row's residual is loaded one row ahead,
// across block boundaries.
constexpr int kPairThreads = 512;
constexpr int kPairWarps = kPairThreads / 32;
constexpr int kPairRing = 4;     // ring entries per lane: a row appends at most two runs, checked every row

// entry = {cell | k << 12, count (as a float), sum Re, sum Im}
__device__ __noinline__ void drain_pair_ring(const int4 *ring, int n_entries, int tid, float *sre, float *sim,
                                             int *scnt, float *ssp, const float *dsp_s)
{
    for (int j = 0; j < n_entries; ++j) {
        const int4 e = ring[j * kPairThreads + tid];
        const int cell = e.x & 0xfff;
        const float n = __int_as_float(e.y);
        atomicAdd(&sre[cell], __int_as_float(e.z));
        atomicAdd(&sim[cell], __int_as_float(e.w));
        atomicAdd(&scnt[cell], (int)n);
        atomicAdd(&ssp[cell], n * dsp_s[e.x >> 12]);
    }
}

template <int CL, bool kUniform, bool kSplit, bool kGauss>
__global__ void __launch_bounds__(kPairThreads, 2)
extract_pair_kernel(const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ w,
                    const float *__restrict__ us, int64_t n_rows, int32_t stride, int32_t n_parts, const ChanTable ch,
                    const float2 *__restrict__ resid, const SrcRow *__restrict__ table, int32_t N,
                    const int32_t *__restrict__ perm, const int32_t *__restrict__ n_live, int32_t n_tslices,
                    float *__restrict__ partial)
{
    constexpr int BW = 32 / CL;                // baselines per warp
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NN = N * N;
    int4 *ring = reinterpret_cast<int4 *>(smraw);                                   // [kPairRing][threads]
    float4 *rows = reinterpret_cast<float4 *>(ring + kPairRing * kPairThreads);     // [warps][32][2]
    float *dsp_s = reinterpret_cast<float *>(rows + kPairWarps * 32 * 2);           // [RLF_MAX_CHAN]
    float *sre = dsp_s + RLF_MAX_CHAN;
    float *sim = sre + NN;
    int *scnt = reinterpret_cast<int *>(sim + NN);
    float *ssp = reinterpret_cast<float *>(scnt + NN);
    const int s = blockIdx.x;
    const SrcRow S = table[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < NN; i += kPairThreads) {
        sre[i] = 0.0f;
        sim[i] = 0.0f;
        scnt[i] = 0;
        ssp[i] = 0.0f;
    }
    const int C = ch.n;
    for (int k = tid; k < C; k += kPairThreads) dsp_s[k] = (float)(ch.spec[k] - ch.spec_off);
    __syncthreads();
    const int lb = lane / CL, lc = lane % CL;  // this lane's baseline in the warp, lane in the group
    const int n_cg = (C + 2 * CL - 1) / (2 * CL);
    const int bpc = kPairWarps * BW;           // baselines per work unit
    const bool vec = (C & 1) == 0;             // channel pairs load as one 16-byte vector
    const double du = S.du;
    const int half = N / 2;
    const float coff = 320.0f + (float)half;
    const f32x2 two_pi2 = pk2(6.28318530717958647692f, 6.28318530717958647692f);
    const f32x2 one2 = pk2(1.0f, 1.0f);
    int cnt = 0;
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring) + (uint32_t)tid * 16u;
    float4 *my_rows = rows + (size_t)warp * 64;   // this warp's 32 rows x 2 float4

    if (S.flux > 0.0) {
        const float q0 = (float)S.q[0], q1 = (float)S.q[1], q2 = (float)S.q[2];
        float lh, ll, mh, ml, nh, nl;
        split_double(S.l, lh, ll);
        split_double(S.m, mh, ml);
        split_double(S.n1, nh, nl);
        const int64_t n_time = (n_rows + stride - 1) / stride;
        const int n_base = n_live[s];
        const int n_blocks = (n_base + bpc - 1) / bpc;
        const int n_units = n_blocks * n_cg * n_tslices;
        for (int wk = blockIdx.y; wk < n_units; wk += n_parts) {
            const int blk = wk % n_blocks;
            const int g = (wk / n_blocks) % n_cg;
            const int ts = wk / (n_blocks * n_cg);
            const int64_t t_begin = n_time * ts / n_tslices, t_end = n_time * (ts + 1) / n_tslices;
            const int j = blk * bpc + warp * BW + lb;         // position in the baseline order
            const bool base_on = j < n_base;
            const int bl = base_on ? (perm ? perm[j] : j) : 0;
            const int k0 = g * 2 * CL;                        // the group's first channel
            const int ka = k0 + 2 * lc, kb = ka + 1;          // this lane's channels
            const bool on_a = base_on && ka < C, on_b = base_on && kb < C;
            const int kac = on_a ? ka : 0, kbc = on_b ? kb : 0;
            // per-channel constants (pairs: channel a, channel b)
            const float sdu_a = (float)(ch.s[kac] / du), sdu_b = (float)(ch.s[kbc] / du);
            const f32x2 f2 = pk2((float)(ch.s[kac] * ch.s[kac]), (float)(ch.s[kbc] * ch.s[kbc]));
            const f32x2 fspec = pk2((float)(S.flux * ch.spec[kac]), (float)(S.flux * ch.spec[kbc]));
            const f32x2 cpos = pk2((float)(2 * lc), (float)(2 * lc + 1));
            const int kbits_a = ka << 12, kbits_b = kb << 12;
            int cell_a = -1, cell_b = -1;
            f32x2 run_re = pk2(0.0f, 0.0f), run_im = pk2(0.0f, 0.0f), run_n = pk2(0.0f, 0.0f);
            // split-baseline record of this lane's row of the next block, fetched a block ahead
            float4 rec_a = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 rec_b = make_float2(0.f, 0.f);
            auto fetch_record = [&](int64_t tt) {
                if (kSplit && base_on && tt < t_end && tt * stride + bl < n_rows) {
                    const int64_t c0 = tt * stride + j;
                    rec_a = reinterpret_cast<const float4 *>(us)[2 * c0];
                    rec_b = reinterpret_cast<const float2 *>(us)[4 * c0 + 2];
                }
            };
            const int nr32 = (int)n_rows;
            const int vstep = stride * C;
            float4 dnext = make_float4(0.f, 0.f, 0.f, 0.f);   // the residual of the lane's next row
            for (int64_t t0 = t_begin; t0 < t_end; t0 += CL) {
                // rows t0 .. t0 + CL - 1 of this lane's baseline: lane lc prepares row t0 + lc
                {
                    const int64_t tt = t0 + lc;
                    const int64_t r = tt * stride + bl;
                    const bool row_ok = base_on && tt < t_end && r < n_rows;
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
                    fetch_record(tt);
                    const float4 a4 = rec_a;
                    const float2 b2 = rec_b;
                    if (row_ok) {
                        float uh, vh;
                        float P = 0.0f, E = 0.0f, f0 = 0.0f, fd = 0.0f;
                        if (kSplit) {
                            uh = a4.x;
                            vh = a4.z;
                            phase_metres(a4.x, a4.y, a4.z, a4.w, b2.x, b2.y, lh, ll, mh, ml, nh, nl, P, E);
                            if (kUniform) {
                                f0 = frac_cycles(P, E, ch.s_hi[k0], ch.s_lo[k0]);
                                fd = frac_cycles(P, E, ch.ds_hi, ch.ds_lo);
                            }
                        } else {
                            const double ud = u[r], vd = v[r], wd = w[r];
                            const double ph = fma(wd, S.n1, fma(vd, S.m, ud * S.l));
                            uh = (float)ud;
                            vh = (float)vd;
                            // the FP64 phase (metres) kept in the two words P, E
                            P = __int_as_float(__double2hiint(ph));
                            E = __int_as_float(__double2loint(ph));
                            if (kUniform) {
                                const double t1 = ph * ch.s[k0];
                                f0 = (float)(t1 - rint(t1));
                                const double t2 = ph * ch.ds;
                                fd = (float)(t2 - rint(t2));
                            }
                        }
                        const float q = fmaf(q2, vh * vh, fmaf(q1, uh * vh, q0 * (uh * uh)));
                        a = make_float4(P, E, f0, fd);
                        b = make_float4(uh, vh, q, 1.0f);
                    }
                    my_rows[2 * lane] = a;
                    my_rows[2 * lane + 1] = b;
                }
                __syncwarp();
                const int nt = (int)min((int64_t)CL, t_end - t0);
                int r = (int)(t0 * stride + bl);
                const float2 *dp = resid + ((int64_t)r * C + kac);
                if (t0 == t_begin && r < nr32) {
                    // the unit's first row; later blocks start on the row the previous
                    // block's last iteration fetched
                    if (vec) {
                        dnext = *reinterpret_cast<const float4 *>(dp);
                    } else {
                        const float2 x = dp[0];
                        const float2 y = on_b ? dp[1] : make_float2(0.f, 0.f);
                        dnext = make_float4(x.x, x.y, y.x, y.y);
                    }
                }
#pragma unroll 2
                for (int tau = 0; tau < CL; ++tau) {
                    if (tau < nt) {
                        // a row appends at most two runs: make room first
                        if (__any_sync(0xffffffffu, cnt > kPairRing - 2)) {
                            drain_pair_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                            cnt = 0;
                        }
                        const float4 d = dnext;
                        {
                            // the next row (the next block's first after a block's last), or this
                            // row again past the last row (always in bounds)
                            const float2 *np = r + stride < nr32 ? dp + vstep : dp;
                            if (vec) {
                                dnext = *reinterpret_cast<const float4 *>(np);
                            } else {
                                const float2 x = np[0];
                                const float2 y = on_b ? np[1] : make_float2(0.f, 0.f);
                                dnext = make_float4(x.x, x.y, y.x, y.y);
                            }
                        }
                        const float4 ra = my_rows[2 * (lb * CL + tau)];
                        const float4 rb = my_rows[2 * (lb * CL + tau) + 1];
                        const bool row_on = rb.w != 0.0f;
                        // phases of the two channels, in cycles, reduced to [-1/2, 1/2]
                        float fa, fb;
                        if (kUniform) {
                            up2(fma2(cpos, pk2(ra.w, ra.w), pk2(ra.z, ra.z)), fa, fb);
                        } else if (kSplit) {
                            fa = frac_cycles(ra.x, ra.y, ch.s_hi[kac], ch.s_lo[kac]);
                            fb = frac_cycles(ra.x, ra.y, ch.s_hi[kbc], ch.s_lo[kbc]);
                        } else {
                            const double ph = __hiloint2double(__float_as_int(ra.x), __float_as_int(ra.y));
                            const double ta = ph * ch.s[kac], tb = ph * ch.s[kbc];
                            fa = (float)(ta - rint(ta));
                            fb = (float)(tb - rint(tb));
                        }
                        float xa, xb;
                        up2(mul2(add2(pk2(fa, fb), pk2(-rintf(fa), -rintf(fb))), two_pi2), xa, xb);
                        float sa, ca, sb, cb;
                        __sincosf(xa, &sa, &ca);
                        __sincosf(xb, &sb, &cb);
                        // cells of the two channels (FP64 decision within the FP32 error of an edge)
                        int ia, ib;
                        bool ea, eb, ina, inb;
                        cell_index2(rb.x, rb.y, sdu_a, coff, N, ia, ea, ina);
                        cell_index2(rb.x, rb.y, sdu_b, coff, N, ib, eb, inb);
                        // rows past the baseline list or the time slice hold u = v = 0: not edges
                        ea = ea && row_on && on_a;
                        eb = eb && row_on && on_b;
                        if (ea || eb) {
                            const double ku = u[r], kv = v[r];
                            if (ea) {
                                const int iu = (int)floor((ku * ch.s[kac]) / du) + half;
                                const int iv = (int)floor((kv * ch.s[kac]) / du) + half;
                                ina = (unsigned)iu < (unsigned)N && (unsigned)iv < (unsigned)N;
                                ia = iv * N + iu;
                            }
                            if (eb) {
                                const int iu = (int)floor((ku * ch.s[kbc]) / du) + half;
                                const int iv = (int)floor((kv * ch.s[kbc]) / du) + half;
                                inb = (unsigned)iu < (unsigned)N && (unsigned)iv < (unsigned)N;
                                ib = iv * N + iu;
                            }
                        }
                        ia = (row_on && on_a && ina) ? ia : -1;
                        ib = (row_on && on_b && inb) ? ib : -1;
                        // (rr + i ri) exp(-2 pi i f) plus the source's model S s M, two channels
                        const f32x2 rr = pk2(d.x, d.z), ri = pk2(d.y, d.w);
                        const f32x2 cs = pk2(ca, cb), sn = pk2(sa, sb), nsn = pk2(-sa, -sb);
                        f32x2 xr = fma2(rr, cs, mul2(ri, sn));
                        const f32x2 xi = fma2(ri, cs, mul2(rr, nsn));
                        xr = fma2(fspec, brightness2<kGauss>(pk2(rb.z, rb.z), f2), xr);
                        // runs: a run ends when the cell changes; runs of cell -1 are dropped
                        const bool cha = ia != cell_a, chb = ib != cell_b;
                        float re_a, re_b, im_a, im_b, n_a, n_b;
                        up2(run_re, re_a, re_b);
                        up2(run_im, im_a, im_b);
                        up2(run_n, n_a, n_b);
                        const bool app_a = cha && cell_a >= 0, app_b = chb && cell_b >= 0;
                        st_shared_v4_if(ring_s + (uint32_t)cnt * (kPairThreads * 16u), app_a, cell_a | kbits_a,
                                        __float_as_int(n_a), __float_as_int(re_a), __float_as_int(im_a));
                        cnt += app_a ? 1 : 0;
                        st_shared_v4_if(ring_s + (uint32_t)cnt * (kPairThreads * 16u), app_b, cell_b | kbits_b,
                                        __float_as_int(n_b), __float_as_int(re_b), __float_as_int(im_b));
                        cnt += app_b ? 1 : 0;
                        const f32x2 keep = pk2(cha ? 0.0f : 1.0f, chb ? 0.0f : 1.0f);
                        run_re = fma2(run_re, keep, xr);
                        run_im = fma2(run_im, keep, xi);
                        run_n = fma2(run_n, keep, one2);
                        cell_a = ia;
                        cell_b = ib;
                        r += stride;
                        dp += vstep;
                    }
                }
                __syncwarp();
            }
            // the unit's last runs
            if (__any_sync(0xffffffffu, cnt > kPairRing - 2)) {
                drain_pair_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                cnt = 0;
            }
            float re_a, re_b, im_a, im_b, n_a, n_b;
            up2(run_re, re_a, re_b);
            up2(run_im, im_a, im_b);
            up2(run_n, n_a, n_b);
            if (cell_a >= 0) {
                ring[cnt * kPairThreads + tid] = make_int4(cell_a | kbits_a, __float_as_int(n_a), __float_as_int(re_a),
                                                           __float_as_int(im_a));
                ++cnt;
            }
            if (cell_b >= 0) {
                ring[cnt * kPairThreads + tid] = make_int4(cell_b | kbits_b, __float_as_int(n_b), __float_as_int(re_b),
                                                           __float_as_int(im_b));
                ++cnt;
            }
        }
    }
    drain_pair_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
    __syncthreads();
    float *o = partial + ((size_t)s * n_parts + blockIdx.y) * 4 * NN;
    for (int i = tid; i < NN; i += kPairThreads) {
        o[i] = sre[i];
        o[NN + i] = sim[i];
        o[2 * NN + i] = __int_as_float(scnt[i]);
        o[3 * NN + i] = ssp[i];
    }
}

// Sum of the parts of every cell in FP64: a CTA takes 32 cells of one facet and
// eight groups of threads sum every eighth part each; the groups' sums are then
// added in group order (the result does not depend on timing).
constexpr int kReduceCells = 32, kReduceGroups = kThreads / kReduceCells;

__global__ void facet_reduce_kernel(const float *__restrict__ partial, int32_t n_parts, int32_t NN,
                                    double spec_off, double *__restrict__ facets)
{
    __shared__ double sre[kReduceGroups][kReduceCells], sim[kReduceGroups][kReduceCells],
        ssp[kReduceGroups][kReduceCells];
    __shared__ long long scnt[kReduceGroups][kReduceCells];
    const int s = blockIdx.y;
    const int lc = threadIdx.x % kReduceCells, grp = threadIdx.x / kReduceCells;
    const int cell = blockIdx.x * kReduceCells + lc;
    double re = 0.0, im = 0.0, sp = 0.0;
    long long n = 0;
    if (cell < NN) {
        for (int p = grp; p < n_parts; p += kReduceGroups) {
            const float *q = partial + ((size_t)s * n_parts + p) * 4 * NN;
            re += (double)q[cell];
            im += (double)q[NN + cell];
            n += __float_as_int(q[2 * NN + cell]);
            sp += (double)q[3 * NN + cell];
        }
    }
    sre[grp][lc] = re;
    sim[grp][lc] = im;
    ssp[grp][lc] = sp;
    scnt[grp][lc] = n;
    __syncthreads();
    if (grp == 0 && cell < NN) {
        for (int g = 1; g < kReduceGroups; ++g) {
            re += sre[g][lc];
            im += sim[g][lc];
            sp += ssp[g][lc];
            n += scnt[g][lc];
        }
        double *f = facets + (size_t)s * 4 * NN;
        f[cell] = re;
        f[NN + cell] = im;
        f[2 * NN + cell] = (double)n;
        f[3 * NN + cell] = sp + (double)n * spec_off;
    }
}

// FP64 extraction: every operation in double precision, one visibility at a time.
__global__ void __launch_bounds__(kThreads)
extract_fp64_kernel(const double *__restrict__ u, const double *__restrict__ v,
                    const double *__restrict__ w, int64_t n_rows, const ChanTable ch,
                    const float2 *__restrict__ data, const float2 *__restrict__ sky,
                    const SrcRow *__restrict__ table, int32_t N, int64_t rows_per_chunk,
                    double *__restrict__ facets)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    double *acc = reinterpret_cast<double *>(smraw);
    const int NN = N * N;
    const int s = blockIdx.x;
    const SrcRow S = table[s];
    for (int i = threadIdx.x; i < 4 * NN; i += kThreads) acc[i] = 0.0;
    __syncthreads();
    const int C = ch.n;
    const int half = N / 2;
    const double du = S.du;
    if (S.flux > 0.0) {
        const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
        const int64_t r1 = min(n_rows, r0 + rows_per_chunk);
        for (int64_t o = r0 * C + threadIdx.x; o < r1 * C; o += kThreads) {
            const int64_t r = o / C;
            const int k = (int)(o % C);
            const double ud = u[r], vd = v[r], wd = w[r];
            const double ku = ud * ch.s[k], kv = vd * ch.s[k];
            const double fu = floor(ku / du), fv = floor(kv / du);
            if (fu < -half || fu >= half || fv < -half || fv >= half) continue;
            const int iu = (int)fu + half, iv = (int)fv + half;
            const float2 dv = data[o];
            const float2 sv = sky[o];
            const double rr = (double)dv.x - (double)sv.x, ri = (double)dv.y - (double)sv.y;
            const double t = fma(wd, S.n1, fma(vd, S.m, ud * S.l)) * ch.s[k];
            double sn, cs;
            sincospi(2.0 * (t - rint(t)), &sn, &cs);
            double xr = rr * cs + ri * sn;
            const double xi = ri * cs - rr * sn;
            const double qs = (S.q[0] * ud * ud + S.q[1] * ud * vd + S.q[2] * vd * vd) * ch.s[k] * ch.s[k];
            xr += S.flux * ch.spec[k] * brightness64(qs, ch.profile);
            const int cell = iv * N + iu;
            atomicAdd(&acc[cell], xr);
            atomicAdd(&acc[NN + cell], xi);
            atomicAdd(&acc[2 * NN + cell], 1.0);
            atomicAdd(&acc[3 * NN + cell], ch.spec[k]);
        }
    }
    __syncthreads();
    double *f = facets + (size_t)s * 4 * NN;
    for (int i = threadIdx.x; i < NN; i += kThreads) {
        if (acc[2 * NN + i] != 0.0) {
            atomicAdd(&f[i], acc[i]);
            atomicAdd(&f[NN + i], acc[NN + i]);
            atomicAdd(&f[2 * NN + i], acc[2 * NN + i]);
            atomicAdd(&f[3 * NN + i], acc[3 * NN + i]);
        }
    }
}

int sm_count_x()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 152;
    }
    return n;
}

// Baseline order of an extraction: perm (null: identity) and per-source counts.
struct Order {
    const int32_t *perm;
    const int32_t *n_live;
};

// lanes per baseline of the channel-pair kernel: half the channel count rounded up to a
// power of two, at most 32 (more channels form groups of 64)
int pair_cl(int n_chan)
{
    int cl = 1;
    while (2 * cl < n_chan && cl < 32) cl *= 2;
    return cl;
}

size_t pair_smem(int N)
{
    return (size_t)kPairRing * kPairThreads * sizeof(int4) + (size_t)kPairWarps * 64 * sizeof(float4) +
           RLF_MAX_CHAN * sizeof(float) + 4 * (size_t)N * N * sizeof(float);
}

template <int CL, bool kSplit>
auto pick_pair_kernel(const ChanTable &ch)
{
    if (ch.profile == RLF_PROFILE_GAUSSIAN)
        return ch.uniform ? extract_pair_kernel<CL, true, kSplit, true> : extract_pair_kernel<CL, false, kSplit, true>;
    return ch.uniform ? extract_pair_kernel<CL, true, kSplit, false> : extract_pair_kernel<CL, false, kSplit, false>;
}

template <bool kSplit>
cudaError_t launch_pair(const rlf_uvw &uvw, const ChanTable &ch, const float *resid, const SrcRow *table,
                        int32_t count, int32_t N, const float *us, const Order &ord, float *partial,
                        int32_t max_partials, double *facets, int waves, cudaStream_t st)
{
    const size_t smem = pair_smem(N);
    const int CL = pair_cl(ch.n);
    decltype(&extract_pair_kernel<1, true, kSplit, false>) kern;
    switch (CL) {
    case 1: kern = pick_pair_kernel<1, kSplit>(ch); break;
    case 2: kern = pick_pair_kernel<2, kSplit>(ch); break;
    case 4: kern = pick_pair_kernel<4, kSplit>(ch); break;
    case 8: kern = pick_pair_kernel<8, kSplit>(ch); break;
    case 16: kern = pick_pair_kernel<16, kSplit>(ch); break;
    default: kern = pick_pair_kernel<32, kSplit>(ch); break;
    }
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPairThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int32_t stride = uvw.n_baselines > 0 ? uvw.n_baselines : 1024;
    const int n_cg = (ch.n + 2 * CL - 1) / (2 * CL);
    const int bpc = kPairWarps * (32 / CL);
    const int64_t n_blocks = ((int64_t)stride + bpc - 1) / bpc * n_cg;   // (baseline block, channel group) units
    const int64_t n_time = (uvw.n_rows + stride - 1) / stride;
    const int NN = N * N;
    const int64_t slots = (int64_t)sm_count_x() * per_sm;
    for (int32_t first = 0; first < count; first += max_partials) {
        const int32_t cnt = count - first < max_partials ? count - first : max_partials;
        // parts per source: about `waves` waves of CTAs; beyond one part per unit (few
        // sources) the time series are split too, into slices of at least 16 steps
        int64_t parts = ((int64_t)waves * slots + cnt - 1) / cnt;
        int64_t slices = 1;
        if (parts > n_blocks) {
            slices = (parts + n_blocks - 1) / n_blocks;
            const int64_t max_slices = n_time / 16 > 1 ? n_time / 16 : 1;
            if (slices > max_slices) slices = max_slices;
            if (slices > 32) slices = 32;
        }
        if (parts > n_blocks * slices) parts = n_blocks * slices;
        if (parts > max_partials / cnt) parts = max_partials / cnt;
        if (parts < 1) parts = 1;
        dim3 grid(cnt, (unsigned)parts);
        kern<<<grid, kPairThreads, smem, st>>>(uvw.u, uvw.v, uvw.w, us, uvw.n_rows, stride, (int32_t)parts, ch,
                                               reinterpret_cast<const float2 *>(resid), table + first, N, ord.perm,
                                               ord.n_live + first, (int32_t)slices, partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        dim3 rgrid((NN + kReduceCells - 1) / kReduceCells, cnt);
        facet_reduce_kernel<<<rgrid, kThreads, 0, st>>>(partial, (int32_t)parts, NN, ch.spec_off,
                                                        facets + (size_t)first * 4 * NN);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_fp64(const rlf_uvw &uvw, const ChanTable &ch, const float *data, const float *sky,
                        const SrcRow *table, int32_t count, int32_t N, double *facets, cudaStream_t st)
{
    const size_t smem = 4 * (size_t)N * N * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(extract_fp64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t target = (int64_t)sm_count_x() * 4;
    int64_t n_chunks = (target + count - 1) / count;
    const int64_t max_chunks = (uvw.n_rows * uvw.n_chan + kThreads - 1) / kThreads;
    if (n_chunks > max_chunks) n_chunks = max_chunks;
    if (n_chunks < 1) n_chunks = 1;
    if (n_chunks > 65535) n_chunks = 65535;
    const int64_t rows_per_chunk = (uvw.n_rows + n_chunks - 1) / n_chunks;
    dim3 grid(count, (unsigned)n_chunks);
    extract_fp64_kernel<<<grid, kThreads, smem, st>>>(uvw.u, uvw.v, uvw.w, uvw.n_rows, ch,
                                                     reinterpret_cast<const float2 *>(data),
                                                     reinterpret_cast<const float2 *>(sky), table, N,
                                                     rows_per_chunk, facets);
    return cudaGetLastError();
}

}  // namespace

namespace {

// rows are walked as [time][stride]; stride = baselines per time step when known
int32_t row_stride(const rlf_uvw &uvw) { return uvw.n_baselines > 0 ? uvw.n_baselines : 1024; }

// the order is used when the rows are exactly [time][baseline]
bool ordered(const rlf_uvw &uvw) { return uvw.n_baselines > 0 && uvw.n_rows % uvw.n_baselines == 0; }

int64_t grid_for(int64_t n, int64_t cap)
{
    const int64_t need = (n + kThreads - 1) / kThreads;
    return need < 1 ? 1 : (need < cap ? need : cap);
}

}  // namespace

// out = a - b over n_complex complex values of any count (float4 pairs, then the odd one)
__global__ void difference_tail_kernel(const float2 *__restrict__ a, const float2 *__restrict__ b, int64_t i,
                                       float2 *__restrict__ out)
{
    const float2 x = a[i], y = b[i];
    out[i] = make_float2(x.x - y.x, x.y - y.y);
}

cudaError_t launch_difference_any(const float *a, const float *b, int64_t n_complex, float *out, cudaStream_t st)
{
    const int64_t n4 = n_complex / 2;
    if (n4 > 0) {
        residual_kernel<<<(int)grid_for(n4, (int64_t)sm_count_x() * 16), kThreads, 0, st>>>(
            reinterpret_cast<const float4 *>(a), reinterpret_cast<const float4 *>(b), n4,
            reinterpret_cast<float4 *>(out));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_complex % 2 != 0) {
        difference_tail_kernel<<<1, 1, 0, st>>>(reinterpret_cast<const float2 *>(a), reinterpret_cast<const float2 *>(b),
                                                n_complex - 1, reinterpret_cast<float2 *>(out));
        return cudaGetLastError();
    }
    return cudaSuccess;
}

cudaError_t launch_difference(const float *a, const float *b, int64_t n_complex, float *out, cudaStream_t st)
{
    if (n_complex % 2 != 0) return cudaErrorInvalidValue;
    const int64_t n4 = n_complex / 2;
    residual_kernel<<<(int)grid_for(n4, (int64_t)sm_count_x() * 16), kThreads, 0, st>>>(
        reinterpret_cast<const float4 *>(a), reinterpret_cast<const float4 *>(b), n4, reinterpret_cast<float4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_split_uvw(const rlf_uvw &uvw, float *out, cudaStream_t st)
{
    split_uvw_kernel<<<(int)grid_for(uvw.n_rows, (int64_t)sm_count_x() * 8), kThreads, 0, st>>>(
        uvw.u, uvw.v, uvw.w, uvw.n_rows, 1, nullptr, out);
    return cudaGetLastError();
}

SplitRows split_rows(const rlf_uvw &uvw, const rlf_params &p, const Workspace &ws)
{
    SplitRows sr;
    if (p.precision != RLF_PREC_MIXED_SPLIT || !ws.uvw_split) return sr;
    sr.rec = ws.uvw_split;
    sr.perm = ordered(uvw) ? ws.perm : nullptr;
    sr.stride = row_stride(uvw);
    return sr;
}

cudaError_t launch_extract_prepare(const rlf_uvw &uvw, const rlf_params &p, const Workspace &ws, cudaStream_t st)
{
    if (p.precision == RLF_PREC_FP64) return cudaSuccess;
    const int32_t stride = row_stride(uvw);
    const int32_t n_b = (int64_t)stride < uvw.n_rows ? stride : (int32_t)uvw.n_rows;
    track_extent_kernel<<<(int)grid_for(n_b, (int64_t)sm_count_x() * 8), kThreads, 0, st>>>(uvw.u, uvw.v, uvw.n_rows,
                                                                                            n_b, ws.extent);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const bool ord = ordered(uvw);
    if (ord) {
        order_kernel<<<1, kOrderThreads, 0, st>>>(ws.extent, n_b, ws.order_counts, ws.perm);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (p.precision == RLF_PREC_MIXED_SPLIT) {
        split_uvw_kernel<<<(int)grid_for(uvw.n_rows, (int64_t)sm_count_x() * 8), kThreads, 0, st>>>(
            uvw.u, uvw.v, uvw.w, uvw.n_rows, stride, ord ? ws.perm : nullptr, ws.uvw_split);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_extract(const rlf_uvw &uvw, const ChanTable &ch, const float *data,
                           const float *sky, const SrcRow *table, int32_t count,
                           const rlf_params &p, const Workspace &ws, double *facets, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    if (p.precision == RLF_PREC_FP64) {
        e = cudaMemsetAsync(facets, 0, (size_t)count * 4 * p.facet_n * p.facet_n * sizeof(double), st);
        if (e != cudaSuccess) return e;
        return launch_fp64(uvw, ch, data, sky, table, count, p.facet_n, facets, st);
    }
    // the extraction reads R = D - V_sky: formed here in one streaming pass (every source
    // of the batch reads it), unless the caller passes the residual itself (sky null)
    if (sky) {
        if (!ws.resid) return cudaErrorInvalidValue;
        const int64_t n2 = uvw.n_rows * uvw.n_chan;   // complex values
        if ((e = launch_difference_any(data, sky, n2, ws.resid, st)) != cudaSuccess) return e;
        data = ws.resid;
    }
    // per source, how far along the baseline order its window can be reached
    const int32_t stride = row_stride(uvw);
    const int32_t n_b = (int64_t)stride < uvw.n_rows ? stride : (int32_t)uvw.n_rows;
    double s_min = ch.s[0];
    for (int k = 1; k < ch.n; ++k) s_min = ch.s[k] < s_min ? ch.s[k] : s_min;
    const Order ord{ordered(uvw) ? ws.perm : nullptr, ws.n_live};
    live_count_kernel<<<count, kThreads, 0, st>>>(ws.extent, ord.perm, n_b, table, p.facet_n, s_min, ws.n_live);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int waves = p.tune_extract_waves > 0 ? p.tune_extract_waves : 2;
    if (p.precision == RLF_PREC_MIXED)
        return launch_pair<false>(uvw, ch, data, table, count, p.facet_n, nullptr, ord, ws.partial, ws.n_partials,
                                  facets, waves, st);
    return launch_pair<true>(uvw, ch, data, table, count, p.facet_n, ws.uvw_split, ord, ws.partial, ws.n_partials,
                             facets, waves, st);
}

}  // namespace rlf
