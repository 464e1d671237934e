// Facet extraction (Sec. 2.3): residual isolation, phase shift to the source and
// averaging of the shifted visibilities into a facet_n x facet_n uv grid of
// cell side du = 1 / (K alpha).
//
// The residual of source i is D - V_sky + model_i; model_i carries the phase
// exp(+2 pi i phi_i), so after the shift it is the real number S s M(k) and
// x = (D - V_sky) exp(-2 pi i phi_i) + S s M(k).
//
// Mixed-precision kernel (extract_rl_kernel).  A CTA owns (source, part) and
// keeps a private copy of the facet in shared memory; the part is an
// interleaved share of the blocks of baselines.  Each thread walks one
// baseline's whole time series for a group of channels.  A baseline's uv track
// moves slowly (a few per cent of a cell per 60 s step at the facet sizes of the
// method), so consecutive visibilities of one channel usually fall in the same
// cell: the thread sums that run in registers and adds it to shared memory only
// when the cell changes.  At the end the CTA stores its partial facet with
// plain coalesced stores, and facet_reduce_kernel sums the parts of each cell in
// FP64 in a fixed order (no global atomics).  Inside a CTA the warps' shared-memory
// additions land in varying order, so repeated runs agree to FP32 rounding.  blockIdx.x runs over the sources, so the CTAs reading the same
// baselines run together and share them through L2.
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

// Run rings: a lane whose run of equal cells ends appends the run to its own
// ring of kRing entries in shared memory (slot-major, so a warp's appends are
// consecutive 16-byte words); no warp vote per visibility.  Once per row the warp
// checks whether any ring could overflow during the row (at most CG appends) and,
// if so, every lane adds its own entries to the shared-memory facet.
constexpr int kRing = 12;    // entries per lane

// Add lane `tid`'s n_entries ring entries to the facet; entry = {cell | k << 12
// (cell < 4096, channel k < 128), count, sum Re, sum Im}; the spectral sum of a
// run is count * (spec_k - spec_off).
__device__ __noinline__ void drain_ring(const int4 *ring, int n_entries, int tid, float *sre, float *sim,
                                        int *scnt, float *ssp, const float *dsp_s)
{
    for (int j = 0; j < n_entries; ++j) {
        const int4 e = ring[j * kThreads + tid];
        const int cell = e.x & 0xfff;
        atomicAdd(&sre[cell], __int_as_float(e.z));
        atomicAdd(&sim[cell], __int_as_float(e.w));
        atomicAdd(&scnt[cell], e.y);
        atomicAdd(&ssp[cell], (float)e.y * dsp_s[e.x >> 12]);
    }
}

// Cell index of both coordinates, with paired FP32 instructions: floor(t) for
// |t| < 2^22 as round(t - 1/2), where the rounding to an integer is done by adding
// 1.5 * 2^23 (the integer lands in the low mantissa bits) and d = y - round(y) is
// exact.  Away from a cell edge round(t - 1/2) = floor(t).  With t = fl(u) *
// fl(nu/c/du) formed by one FMA, |error of t| <= 3 * 2^-24 |t| < 6e-6 for
// |t| <= 33 (every facet window here); `edge` flags values within 1e-5 of a
// cell edge, where the caller takes the FP64 decision instead.
__device__ __forceinline__ void cell_floor2(float uh, float vh, float sdu, int &iu, int &iv, bool &edge)
{
    constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
    const f32x2 y = fma2(pk2(uh, vh), pk2(sdu, sdu), pk2(-0.5f, -0.5f));
    const f32x2 m = add2(y, pk2(kMagic, kMagic));
    const f32x2 d = add2(y, add2(m, pk2(-kMagic, -kMagic)) ^ 0x8000000080000000ull);
    float du_, dv_, mu_, mv_;
    up2(d, du_, dv_);
    up2(m, mu_, mv_);
    edge = fmaxf(fabsf(du_), fabsf(dv_)) > 0.5f - 1.0e-5f;
    iu = __float_as_int(mu_) - 0x4B400000;
    iv = __float_as_int(mv_) - 0x4B400000;
}

// A 16-byte shared-memory store under a predicate: the append of a finished run
// costs the same few instructions whether or not the lane appends, with no branch
// for the warp to diverge on.
__device__ __forceinline__ void st_shared_v4_if(uint32_t addr, bool p, int a, int b, int c, int d)
{
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared.v4.b32 [%1], {%2, %3, %4, %5}; }"
                 :: "r"((int)p), "r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

// kResid: `data` already holds D - V_sky (one load per visibility), `sky` is unused.
// kGauss: the Gaussian source profile instead of the exponential one.
template <int CG, bool kUniform, bool kSplit, bool kResid, bool kGauss>
__global__ void __launch_bounds__(kThreads, CG >= 8 ? 2 : 3)
extract_rl_kernel(const double *__restrict__ u, const double *__restrict__ v,
                  const double *__restrict__ w, const float *__restrict__ us, int64_t n_rows,
                  int32_t stride, int32_t n_parts, const ChanTable ch,
                  const float2 *__restrict__ data, const float2 *__restrict__ sky,
                  const SrcRow *__restrict__ table, int32_t N, const int32_t *__restrict__ perm,
                  const int32_t *__restrict__ n_live, int32_t n_tslices, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NN = N * N;
    (void)sky;
    int4 *ring = reinterpret_cast<int4 *>(smraw);                       // [kRing][kThreads]
    float *dsp_s = reinterpret_cast<float *>(ring + kRing * kThreads);  // [RLF_MAX_CHAN]
    float *sre = dsp_s + RLF_MAX_CHAN;
    float *sim = sre + NN;
    int *scnt = reinterpret_cast<int *>(sim + NN);
    float *ssp = reinterpret_cast<float *>(scnt + NN);
    const int s = blockIdx.x;
    const SrcRow S = table[s];
    const int tid = threadIdx.x;

    for (int i = tid; i < NN; i += kThreads) {
        sre[i] = 0.0f;
        sim[i] = 0.0f;
        scnt[i] = 0;
        ssp[i] = 0.0f;
    }
    const int C = ch.n;
    const int n_groups = (C + CG - 1) / CG;
    const int bpc = kThreads / n_groups;           // baselines per block
    const int g = tid / bpc;
    const int lane_b = tid % bpc;
    const bool group_on = g < n_groups;
    const int k0 = group_on ? g * CG : 0;
    for (int k = tid; k < C; k += kThreads) dsp_s[k] = (float)(ch.spec[k] - ch.spec_off);
    __syncthreads();
    const int half = N / 2;
    const double du = S.du;
    constexpr float kTwoPi = 6.28318530717958647692f;
    int cnt = 0;                                   // entries in this lane's ring
    const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);

    auto append = [&](int cell, int k, int n, float re, float im) {
        ring[cnt * kThreads + tid] = make_int4(cell | (k << 12), n, __float_as_int(re), __float_as_int(im));
        ++cnt;
    };

    if (S.flux > 0.0) {
        // per-channel constants used for every visibility stay in registers
        float sdu[CG], f2[CG], fspec[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) {
            const int k = min(k0 + c, C - 1);
            sdu[c] = (float)(ch.s[k] / du);
            f2[c] = (float)(ch.s[k] * ch.s[k]);
            fspec[c] = (float)(S.flux * ch.spec[k]);
        }
        const float q0 = (float)S.q[0], q1 = (float)S.q[1], q2 = (float)S.q[2];
        float lh, ll, mh, ml, nh, nl;
        split_double(S.l, lh, ll);
        split_double(S.m, mh, ml);
        split_double(S.n1, nh, nl);
        const int64_t n_time = (n_rows + stride - 1) / stride;
        // the source's baselines, in extent order, that can reach its window
        const int n_base = n_live[s];
        const int n_blocks = (n_base + bpc - 1) / bpc;
        // the residual of a row's channel group is read as float4 pairs when the
        // layout allows (even channel count, groups of >= 2 channels)
        const bool vec = kResid && CG >= 2 && (C % 2 == 0);

        int run_cell[CG], run_n[CG];
        float run_re[CG], run_im[CG];
        // every lane runs every iteration (the per-row ring check is a warp vote);
        // lanes without a visibility carry cell = -1, whose runs are never appended
        // work units: (block of baselines, slice of the time series); a few sources at a
        // time also split each baseline's time series so that the grid fills the GPU
        for (int wk = blockIdx.y; wk < n_blocks * n_tslices; wk += n_parts) {
            const int blk = wk % n_blocks, ts = wk / n_blocks;
            const int64_t t_begin = n_time * ts / n_tslices, t_end = n_time * (ts + 1) / n_tslices;
            // lane position j in the order; bl the baseline (data rows bl + t * stride);
            // the split baselines are stored in order, at column j
            const int j = blk * bpc + lane_b;
            const bool lane_on = group_on && j < n_base;
            const int bl = lane_on ? (perm ? perm[j] : j) : 0;
#pragma unroll
            for (int c = 0; c < CG; ++c) {
                run_cell[c] = -1;
                run_n[c] = 0;
                run_re[c] = run_im[c] = 0.0f;
            }
            // split baselines of the next row are fetched one iteration ahead
            float nuh = 0, nul = 0, nvh = 0, nvl = 0, nwh = 0, nwl = 0;
            if (kSplit && lane_on && t_begin < t_end && t_begin * stride + bl < n_rows) {
                const int64_t c0 = t_begin * stride + j;
                const float4 a4 = reinterpret_cast<const float4 *>(us)[2 * c0];
                const float2 b2 = reinterpret_cast<const float2 *>(us)[4 * c0 + 2];
                nuh = a4.x;
                nul = a4.y;
                nvh = a4.z;
                nvl = a4.w;
                nwh = b2.x;
                nwl = b2.y;
            }
            for (int64_t t = t_begin; t < t_end; ++t) {
                // a row appends at most CG runs: make room first
                if (__any_sync(0xffffffffu, cnt > kRing - CG)) {
                    drain_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                    cnt = 0;
                }
                const int64_t r = t * stride + bl;
                const bool row_on = lane_on && r < n_rows;
                float2 rv[CG];
#pragma unroll
                for (int c = 0; c < CG; ++c) rv[c] = make_float2(0.0f, 0.0f);
                if (vec && row_on) {
                    const float4 *src4 = reinterpret_cast<const float4 *>(data + (r * C + k0));
#pragma unroll
                    for (int j = 0; j < CG / 2; ++j) {
                        if (k0 + 2 * j < C) {
                            const float4 q4 = src4[j];
                            rv[2 * j] = make_float2(q4.x, q4.y);
                            rv[2 * j + 1] = make_float2(q4.z, q4.w);
                        }
                    }
                }
                float uh = 0, ul = 0, vh = 0, vl = 0, wh = 0, wl = 0;
                double ph = 0.0;
                if (kSplit) {
                    uh = nuh;
                    ul = nul;
                    vh = nvh;
                    vl = nvl;
                    wh = nwh;
                    wl = nwl;
                    const int64_t rn = r + stride;
                    const int64_t cn = (t + 1) * stride + j;
                    if (lane_on && t + 1 < t_end && rn < n_rows) {
                        const float4 a4 = reinterpret_cast<const float4 *>(us)[2 * cn];
                        const float2 b2 = reinterpret_cast<const float2 *>(us)[4 * cn + 2];
                        nuh = a4.x;
                        nul = a4.y;
                        nvh = a4.z;
                        nvl = a4.w;
                        nwh = b2.x;
                        nwl = b2.y;
                    }
                } else if (row_on) {
                    const double ud = u[r], vd = v[r], wd = w[r];
                    ph = fma(wd, S.n1, fma(vd, S.m, ud * S.l));
                    uh = (float)ud;
                    vh = (float)vd;
                }
                const float uu = uh * uh, uv = uh * vh, vv = vh * vh;
                const float q = fmaf(q2, vv, fmaf(q1, uv, q0 * uu));
                float P = 0.0f, E = 0.0f;
                if (kSplit) phase_metres(uh, ul, vh, vl, wh, wl, lh, ll, mh, ml, nh, nl, P, E);
                // uniform channels: the phase of channel c is frac(f0 + c fd) cycles, each
                // channel's sincos independent of the others (f0 + c fd in FP32 is within
                // 2^-24 * CG cycles of the exact value)
                float sn = 0.0f, cs = 1.0f;
                float f0_keep = 0.0f, fd_keep = 0.0f;
                if (kUniform) {
                    float f0, fd = 0.0f;
                    if (kSplit) {
                        f0 = frac_cycles(P, E, ch.s_hi[k0], ch.s_lo[k0]);
                        if (CG > 1) fd = frac_cycles(P, E, ch.ds_hi, ch.ds_lo);
                    } else {
                        const double tt = ph * ch.s[k0];
                        f0 = (float)(tt - rint(tt));
                        if (CG > 1) {
                            const double td = ph * ch.ds;
                            fd = (float)(td - rint(td));
                        }
                    }
                    f0_keep = f0;
                    fd_keep = fd;
                }
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int k = k0 + c;
                    if (kUniform) {
                        float fk = fmaf((float)c, fd_keep, f0_keep);
                        fk -= rintf(fk);
                        __sincosf(fk * kTwoPi, &sn, &cs);
                    }
                    if (!kUniform) {
                        const int kk = min(k, C - 1);
                        float f;
                        if (kSplit) {
                            f = frac_cycles(P, E, ch.s_hi[kk], ch.s_lo[kk]);
                        } else {
                            const double tt = ph * ch.s[kk];
                            f = (float)(tt - rint(tt));
                        }
                        __sincosf(f * kTwoPi, &sn, &cs);
                    }
                    int cell = -1;
                    if (row_on && k < C) {
                        int iu, iv;
                        bool edge;
                        cell_floor2(uh, vh, sdu[c], iu, iv, edge);
                        if (edge) {
                            iu = (int)floor((u[r] * ch.s[k]) / du);
                            iv = (int)floor((v[r] * ch.s[k]) / du);
                        }
                        iu += half;
                        iv += half;
                        if ((unsigned)iu < (unsigned)N && (unsigned)iv < (unsigned)N) cell = iv * N + iu;
                    }
                    float rr, ri;
                    if (vec) {
                        rr = rv[c].x;
                        ri = rv[c].y;
                    } else {
                        rr = ri = 0.0f;
                        if (cell >= 0) {
                            const float2 dv = data[r * C + k];
                            rr = dv.x;
                            ri = dv.y;
                            if (!kResid) {
                                const float2 sv = sky[r * C + k];
                                rr -= sv.x;
                                ri -= sv.y;
                            }
                        }
                    }
                    // (rr + i ri) exp(-2 pi i f) = (rr + i ri)(cs - i sn), plus the source's model
                    float xr = fmaf(rr, cs, ri * sn);
                    const float xi = fmaf(ri, cs, -rr * sn);
                    xr = fmaf(fspec[c], brightness<kGauss>(q, f2[c]), xr);
                    // a run ends when the cell changes; runs of cell -1 are dropped
                    const bool change = cell != run_cell[c];
                    {
                        const bool app = change && run_cell[c] >= 0;
                        st_shared_v4_if(ring_s + (uint32_t)(cnt * kThreads + tid) * 16u, app,
                                        run_cell[c] | ((k0 + c) << 12), run_n[c], __float_as_int(run_re[c]),
                                        __float_as_int(run_im[c]));
                        cnt += app ? 1 : 0;
                    }
                    const float keep = change ? 0.0f : 1.0f;
                    run_re[c] = fmaf(run_re[c], keep, xr);
                    run_im[c] = fmaf(run_im[c], keep, xi);
                    run_n[c] = change ? 1 : run_n[c] + 1;
                    run_cell[c] = cell;

                }
            }
            if (__any_sync(0xffffffffu, cnt > kRing - CG)) {
                drain_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                cnt = 0;
            }
#pragma unroll
            for (int c = 0; c < CG; ++c)
                if (run_cell[c] >= 0) append(run_cell[c], k0 + c, run_n[c], run_re[c], run_im[c]);
        }
    }
    // the rings' remainders
    drain_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
    __syncthreads();
    // this CTA's partial facet: plain stores; planes Re, Im, count (int bits), spec - spec_off
    float *o = partial + ((size_t)s * n_parts + blockIdx.y) * 4 * NN;
    for (int i = tid; i < NN; i += kThreads) {
        o[i] = sre[i];
        o[NN + i] = sim[i];
        o[2 * NN + i] = __int_as_float(scnt[i]);
        o[3 * NN + i] = ssp[i];
    }
}

// ---- lane-per-track extraction ------------------------------------------------------
// A warp holds 32 / CL baselines x CL channels (CL = the channel count rounded up to a
// power of two, at most 32; more channels are split into groups of 32): each lane walks
// one (baseline, channel) track through time, sums runs of equal cells in registers and
// appends a finished run to its own ring in shared memory.  The per-row work of a
// baseline (float-pair phase argument, the channel group's phase f0 and step fd, the
// source's quadratic form, u and v in FP32) is shared by its CL lanes: for a block of
// CL time steps lane c computes row t0 + c and stores it in shared memory, then every
// lane reads each row of the block (a broadcast).  One channel per thread keeps the
// registers low enough for 512-thread CTAs, two per SM.
constexpr int kLaneThreads = 512;
constexpr int kLaneWarps = kLaneThreads / 32;
constexpr int kLaneRing = 4;     // ring entries per lane: one append per row at most, drained every two rows
constexpr int kRowWords = 8;     // per row: P, E (or the FP64 phase), f0, fd, q, u, v, valid

__device__ __noinline__ void drain_lane_ring(const int4 *ring, int n_entries, int tid, float *sre, float *sim,
                                             int *scnt, float *ssp, const float *dsp_s)
{
    for (int j = 0; j < n_entries; ++j) {
        const int4 e = ring[j * kLaneThreads + tid];
        const int cell = e.x & 0xfff;
        atomicAdd(&sre[cell], __int_as_float(e.z));
        atomicAdd(&sim[cell], __int_as_float(e.w));
        atomicAdd(&scnt[cell], e.y);
        atomicAdd(&ssp[cell], (float)e.y * dsp_s[e.x >> 12]);
    }
}

template <bool kUniform, bool kSplit, bool kResid, bool kGauss>
__global__ void __launch_bounds__(kLaneThreads, 2)
extract_lane_kernel(const double *__restrict__ u, const double *__restrict__ v, const double *__restrict__ w,
                    const float *__restrict__ us, int64_t n_rows, int32_t stride, int32_t n_parts, const ChanTable ch,
                    const float2 *__restrict__ data, const float2 *__restrict__ sky, const SrcRow *__restrict__ table,
                    int32_t N, const int32_t *__restrict__ perm, const int32_t *__restrict__ n_live,
                    int32_t n_tslices, int32_t CL, float *__restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int NN = N * N;
    int4 *ring = reinterpret_cast<int4 *>(smraw);                                   // [kLaneRing][threads]
    float4 *rows = reinterpret_cast<float4 *>(ring + kLaneRing * kLaneThreads);     // [warps][32][2]
    float *dsp_s = reinterpret_cast<float *>(rows + kLaneWarps * 32 * 2);           // [RLF_MAX_CHAN]
    float *sre = dsp_s + RLF_MAX_CHAN;
    float *sim = sre + NN;
    int *scnt = reinterpret_cast<int *>(sim + NN);
    float *ssp = reinterpret_cast<float *>(scnt + NN);
    const int s = blockIdx.x;
    const SrcRow S = table[s];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < NN; i += kLaneThreads) {
        sre[i] = 0.0f;
        sim[i] = 0.0f;
        scnt[i] = 0;
        ssp[i] = 0.0f;
    }
    const int C = ch.n;
    for (int k = tid; k < C; k += kLaneThreads) dsp_s[k] = (float)(ch.spec[k] - ch.spec_off);
    __syncthreads();
    const int BW = 32 / CL;                    // baselines per warp
    const int lb = lane / CL, lc = lane % CL;  // this lane's baseline in the warp, channel in the group
    const int n_cg = (C + CL - 1) / CL;
    const int bpc = kLaneWarps * BW;           // baselines per work unit
    const double du = S.du;
    const int half = N / 2;
    constexpr float kTwoPi = 6.28318530717958647692f;
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
            const int k0 = g * CL;                            // the group's first channel
            const int k = k0 + lc;                            // this lane's channel
            const bool lane_on = base_on && k < C;
            const int kk = k < C ? k : C - 1;
            // per-channel constants
            const float sdu = (float)(ch.s[kk] / du);
            const float f2 = (float)(ch.s[kk] * ch.s[kk]);
            const float fspec = (float)(S.flux * ch.spec[kk]);
            const float cpos = (float)lc;
            int run_cell = -1, run_n = 0;
            float run_re = 0.0f, run_im = 0.0f;
            for (int64_t t0 = t_begin; t0 < t_end; t0 += CL) {
                // rows t0 .. t0 + CL - 1 of this lane's baseline: lane lc prepares row t0 + lc
                {
                    const int64_t tt = t0 + lc;
                    const int64_t r = tt * stride + bl;
                    const bool row_ok = base_on && tt < t_end && r < n_rows;
                    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (row_ok) {
                        float uh, ul, vh, vl, wh, wl;
                        float P = 0.0f, E = 0.0f, f0 = 0.0f, fd = 0.0f;
                        if (kSplit) {
                            const int64_t c0 = tt * stride + j;
                            const float4 a4 = reinterpret_cast<const float4 *>(us)[2 * c0];
                            const float2 b2 = reinterpret_cast<const float2 *>(us)[4 * c0 + 2];
                            uh = a4.x; ul = a4.y; vh = a4.z; vl = a4.w; wh = b2.x; wl = b2.y;
                            phase_metres(uh, ul, vh, vl, wh, wl, lh, ll, mh, ml, nh, nl, P, E);
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
                            (void)ul; (void)vl; (void)wh; (void)wl;
                        }
                        const float q = fmaf(q2, vh * vh, fmaf(q1, uh * vh, q0 * (uh * uh)));
                        a = make_float4(P, E, f0, fd);
                        b = make_float4(q, uh, vh, 1.0f);
                    }
                    my_rows[2 * lane] = a;
                    my_rows[2 * lane + 1] = b;
                }
                __syncwarp();
                const int nt = (int)min((int64_t)CL, t_end - t0);
                for (int tau = 0; tau < nt; ++tau) {
                    // two rows append at most two runs: make room every other row
                    if ((tau & 1) == 0 && __any_sync(0xffffffffu, cnt > kLaneRing - 2)) {
                        drain_lane_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                        cnt = 0;
                    }
                    const float4 ra = my_rows[2 * (lb * CL + tau)];
                    const float4 rb = my_rows[2 * (lb * CL + tau) + 1];
                    const bool on = lane_on && rb.w != 0.0f;
                    const int64_t r = (t0 + tau) * stride + bl;
                    float rr = 0.0f, ri = 0.0f;
                    if (on) {
                        const float2 dv = data[r * C + k];
                        rr = dv.x;
                        ri = dv.y;
                        if (!kResid) {
                            const float2 sv = sky[r * C + k];
                            rr -= sv.x;
                            ri -= sv.y;
                        }
                    }
                    float f;
                    if (kUniform) {
                        f = fmaf(cpos, ra.w, ra.z);
                    } else if (kSplit) {
                        f = frac_cycles(ra.x, ra.y, ch.s_hi[kk], ch.s_lo[kk]);
                    } else {
                        const double ph = __hiloint2double(__float_as_int(ra.x), __float_as_int(ra.y));
                        const double tt = ph * ch.s[kk];
                        f = (float)(tt - rint(tt));
                    }
                    f -= rintf(f);
                    float sn, cs;
                    __sincosf(f * kTwoPi, &sn, &cs);
                    int cell = -1;
                    if (on) {
                        int iu, iv;
                        bool edge;
                        cell_floor2(rb.y, rb.z, sdu, iu, iv, edge);
                        if (edge) {
                            iu = (int)floor((u[r] * ch.s[k]) / du);
                            iv = (int)floor((v[r] * ch.s[k]) / du);
                        }
                        iu += half;
                        iv += half;
                        if ((unsigned)iu < (unsigned)N && (unsigned)iv < (unsigned)N) cell = iv * N + iu;
                    }
                    // (rr + i ri) exp(-2 pi i f) plus the source's model S s M
                    float xr = fmaf(rr, cs, ri * sn);
                    const float xi = fmaf(ri, cs, -rr * sn);
                    xr = fmaf(fspec, brightness<kGauss>(rb.x, f2), xr);
                    const bool change = cell != run_cell;
                    const bool app = change && run_cell >= 0;
                    st_shared_v4_if(ring_s + (uint32_t)cnt * (kLaneThreads * 16u), app, run_cell | (k << 12), run_n,
                                    __float_as_int(run_re), __float_as_int(run_im));
                    cnt += app ? 1 : 0;
                    const float keep = change ? 0.0f : 1.0f;
                    run_re = fmaf(run_re, keep, xr);
                    run_im = fmaf(run_im, keep, xi);
                    run_n = change ? 1 : run_n + 1;
                    run_cell = cell;
                }
                __syncwarp();
            }
            // the unit's last run
            if (__any_sync(0xffffffffu, cnt > kLaneRing - 1)) {
                drain_lane_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
                cnt = 0;
            }
            if (run_cell >= 0) {
                ring[cnt * kLaneThreads + tid] = make_int4(run_cell | (k << 12), run_n, __float_as_int(run_re),
                                                           __float_as_int(run_im));
                ++cnt;
            }
        }
    }
    drain_lane_ring(ring, cnt, tid, sre, sim, scnt, ssp, dsp_s);
    __syncthreads();
    float *o = partial + ((size_t)s * n_parts + blockIdx.y) * 4 * NN;
    for (int i = tid; i < NN; i += kLaneThreads) {
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

template <int CG, bool kSplit>
cudaError_t launch_rl(const rlf_uvw &uvw, const ChanTable &ch, const float *data, const float *sky,
                      const SrcRow *table, int32_t count, int32_t N, const float *us, const Order &ord,
                      float *partial, int32_t max_partials, double *facets, int waves, cudaStream_t st)
{
    const size_t smem = (size_t)kRing * kThreads * sizeof(int4) + RLF_MAX_CHAN * sizeof(float) +
                        4 * (size_t)N * N * sizeof(float);
    const bool resid = sky == nullptr;
    decltype(&extract_rl_kernel<CG, true, kSplit, true, false>) kern;
    if (ch.profile == RLF_PROFILE_GAUSSIAN)
        kern = ch.uniform ? (resid ? extract_rl_kernel<CG, true, kSplit, true, true> : extract_rl_kernel<CG, true, kSplit, false, true>)
                          : (resid ? extract_rl_kernel<CG, false, kSplit, true, true> : extract_rl_kernel<CG, false, kSplit, false, true>);
    else
        kern = ch.uniform ? (resid ? extract_rl_kernel<CG, true, kSplit, true, false> : extract_rl_kernel<CG, true, kSplit, false, false>)
                          : (resid ? extract_rl_kernel<CG, false, kSplit, true, false> : extract_rl_kernel<CG, false, kSplit, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // rows are walked as [time][stride]; stride = baselines per time step when known
    const int32_t stride = uvw.n_baselines > 0 ? uvw.n_baselines : 1024;
    const int n_groups = (ch.n + CG - 1) / CG;
    const int bpc = kThreads / n_groups;
    const int64_t n_blocks = (stride + bpc - 1) / bpc;
    const int64_t n_time = (uvw.n_rows + stride - 1) / stride;
    const int NN = N * N;
    const int64_t slots = (int64_t)sm_count_x() * per_sm;
    // sources are handled in batches whose partial facets fit the workspace
    for (int32_t first = 0; first < count; first += max_partials) {
        const int32_t cnt = count - first < max_partials ? count - first : max_partials;
        // parts per source: about `waves` waves of CTAs; beyond one part per baseline block
        // (few sources) the time series are split too, into slices of at least 16 steps
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
        kern<<<grid, kThreads, smem, st>>>(uvw.u, uvw.v, uvw.w, us, uvw.n_rows, stride, (int32_t)parts, ch,
                                           reinterpret_cast<const float2 *>(data),
                                           reinterpret_cast<const float2 *>(sky), table + first, N, ord.perm,
                                           ord.n_live + first, (int32_t)slices, partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        dim3 rgrid((NN + kReduceCells - 1) / kReduceCells, cnt);
        facet_reduce_kernel<<<rgrid, kThreads, 0, st>>>(partial, (int32_t)parts, NN, ch.spec_off,
                                                        facets + (size_t)first * 4 * NN);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <bool kSplit>
cudaError_t launch_rl_cg(const rlf_uvw &uvw, const ChanTable &ch, const float *data, const float *sky,
                         const SrcRow *table, int32_t count, int32_t N, const float *us, const Order &ord,
                         float *partial, int32_t max_partials, double *facets, int waves, cudaStream_t st)
{
    if (ch.n == 1) return launch_rl<1, kSplit>(uvw, ch, data, sky, table, count, N, us, ord, partial, max_partials, facets, waves, st);
    if (ch.n == 2) return launch_rl<2, kSplit>(uvw, ch, data, sky, table, count, N, us, ord, partial, max_partials, facets, waves, st);
    if (ch.n <= 4) return launch_rl<4, kSplit>(uvw, ch, data, sky, table, count, N, us, ord, partial, max_partials, facets, waves, st);
    return launch_rl<8, kSplit>(uvw, ch, data, sky, table, count, N, us, ord, partial, max_partials, facets, waves, st);
}

// channel lanes of the lane-per-track kernel: the channel count rounded up to a power of
// two, at most 32
int lane_cl(int n_chan)
{
    int cl = 1;
    while (cl < n_chan && cl < 32) cl *= 2;
    return cl;
}

size_t lane_smem(int N)
{
    return (size_t)kLaneRing * kLaneThreads * sizeof(int4) + (size_t)kLaneWarps * 64 * sizeof(float4) +
           RLF_MAX_CHAN * sizeof(float) + 4 * (size_t)N * N * sizeof(float);
}

template <bool kSplit>
cudaError_t launch_lane(const rlf_uvw &uvw, const ChanTable &ch, const float *data, const float *sky,
                        const SrcRow *table, int32_t count, int32_t N, const float *us, const Order &ord,
                        float *partial, int32_t max_partials, double *facets, int waves, cudaStream_t st)
{
    const size_t smem = lane_smem(N);
    const bool resid = sky == nullptr;
    decltype(&extract_lane_kernel<true, kSplit, true, false>) kern;
    if (ch.profile == RLF_PROFILE_GAUSSIAN)
        kern = ch.uniform ? (resid ? extract_lane_kernel<true, kSplit, true, true> : extract_lane_kernel<true, kSplit, false, true>)
                          : (resid ? extract_lane_kernel<false, kSplit, true, true> : extract_lane_kernel<false, kSplit, false, true>);
    else
        kern = ch.uniform ? (resid ? extract_lane_kernel<true, kSplit, true, false> : extract_lane_kernel<true, kSplit, false, false>)
                          : (resid ? extract_lane_kernel<false, kSplit, true, false> : extract_lane_kernel<false, kSplit, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLaneThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int32_t stride = uvw.n_baselines > 0 ? uvw.n_baselines : 1024;
    const int CL = lane_cl(ch.n);
    const int n_cg = (ch.n + CL - 1) / CL;
    const int bpc = kLaneWarps * (32 / CL);
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
        kern<<<grid, kLaneThreads, smem, st>>>(uvw.u, uvw.v, uvw.w, us, uvw.n_rows, stride, (int32_t)parts, ch,
                                               reinterpret_cast<const float2 *>(data),
                                               reinterpret_cast<const float2 *>(sky), table + first, N, ord.perm,
                                               ord.n_live + first, (int32_t)slices, CL, partial);
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
    // several sources read every visibility: form D - V_sky once (one streaming pass)
    if (sky && ws.resid && count >= 3) {
        const int64_t n2 = uvw.n_rows * uvw.n_chan;   // complex values
        if (n2 % 2 == 0) {
            const int64_t n4 = n2 / 2;
            residual_kernel<<<(int)grid_for(n4, (int64_t)sm_count_x() * 16), kThreads, 0, st>>>(
                reinterpret_cast<const float4 *>(data), reinterpret_cast<const float4 *>(sky), n4,
                reinterpret_cast<float4 *>(ws.resid));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            data = ws.resid;
            sky = nullptr;
        }
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
        return launch_lane<false>(uvw, ch, data, sky, table, count, p.facet_n, nullptr, ord, ws.partial, ws.n_partials,
                                  facets, waves, st);
    return launch_lane<true>(uvw, ch, data, sky, table, count, p.facet_n, ws.uvw_split, ord, ws.partial, ws.n_partials,
                             facets, waves, st);
}

}  // namespace rlf
