// Per-source constants and the sky model (Sec. 2.2, Eq. 1, Eq. 2, Eq. 4).
//
// Sky model layout: one thread owns one (row, channel group) output and walks
// the catalogue, which every CTA stages through shared memory in tiles; rows
// are visited with a grid-stride loop so the staging is amortised over many
// rows.  Mixed precision keeps the phase argument u l + v m + w (n - 1) and its
// range reduction in FP64 once per (row, source) and steps it across the
// channels of the group by an FP32 complex rotation; the brightness factor
// (1 + x)^{-3/2} is one MUFU rsqrt and two multiplies per term.  The split
// variant carries the phase argument as a float pair (error-free FP32 products
// and sums), which GB300 executes at its FP32 rate.
#include <cmath>
#include <type_traits>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

struct PrepConst {
    double add, esp, psf_nat;
    int32_t update, update_mode;
};

__device__ inline void shape_coeffs(double e1, double e2, double alpha_rad, double q[3])
{
    // |A^{-T} k|^2 for A = [[1 - e1, -e2], [-e2, 1 + e1]] (Eq. 2):
    // ((1 + e1)^2 + e2^2) u^2 + 4 e2 u v + ((1 - e1)^2 + e2^2) v^2, over det(A)^2
    const double det = 1.0 - e1 * e1 - e2 * e2;
    const double c = 4.0 * kPi * kPi * alpha_rad * alpha_rad / (det * det);
    q[0] = c * ((1.0 + e1) * (1.0 + e1) + e2 * e2);
    q[1] = c * 4.0 * e2;
    q[2] = c * ((1.0 - e1) * (1.0 - e1) + e2 * e2);
}

__global__ void prepare_kernel(rlf_sources src, int32_t first, int32_t count,
                               const double *__restrict__ e1, const double *__restrict__ e2,
                               const double *__restrict__ e1n, const double *__restrict__ e2n,
                               const int32_t *__restrict__ flag, double *__restrict__ e1c,
                               double *__restrict__ e2c, PrepConst pc,
                               SrcRow *__restrict__ out, int32_t *__restrict__ status,
                               const int32_t *__restrict__ list)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    // row t is source first + t, or source list[t] when a list is given
    const int i = list ? list[t] : first + t;
    const double l = src.l[i], m = src.m[i], S = src.flux_jy[i];
    const double acat = src.alpha_arcsec ? src.alpha_arcsec[i] : 0.0;
    const double a1 = e1[i], a2 = e2[i];
    bool ok = isfinite(l) && isfinite(m) && (l * l + m * m < 1.0) && isfinite(S) && S > 0.0 &&
              isfinite(a1) && isfinite(a2) && (a1 * a1 + a2 * a2 < 1.0) && isfinite(acat);
    double b1 = 0.0, b2 = 0.0;
    bool selected = true;
    if (pc.update) {
        b1 = e1n[t];
        b2 = e2n[t];
        ok = ok && isfinite(b1) && isfinite(b2) && (b1 * b1 + b2 * b2 < 1.0);
        if (pc.update_mode == 0 && flag) selected = (flag[t] & (RLF_FLAG_BAD | RLF_FLAG_INVALID | RLF_FLAG_EMPTY)) == 0;
    }
    SrcRow row;
    const double lnS = log(S * 1.0e6);
    // Eq. 4 median scalelength unless the catalogue gives one (Sec. 2.3)
    const double alpha_as = acat > 0.0 ? acat : exp(pc.add + pc.esp * lnS);
    row.l = l;
    row.m = m;
    const double r2 = l * l + m * m;
    row.n1 = -r2 / (1.0 + sqrt(1.0 - r2));
    row.alpha_rad = alpha_as * kArcsec;
    row.du = 1.0 / (pc.psf_nat * alpha_as * kArcsec);
    row.mu = pc.add + pc.esp * lnS;
    row.flux = (ok && selected) ? S : 0.0;
    row.invalid = ok ? 0 : 1;
    row.pad = 0;
    if (ok) {
        shape_coeffs(a1, a2, row.alpha_rad, row.q);
        if (pc.update) shape_coeffs(b1, b2, row.alpha_rad, row.qn);
        else row.qn[0] = row.qn[1] = row.qn[2] = 0.0;
    } else {
        row.q[0] = row.q[1] = row.q[2] = 0.0;
        row.qn[0] = row.qn[1] = row.qn[2] = 0.0;
        atomicOr(status, RLF_DEV_INVALID_SOURCE);
    }
    out[t] = row;
    // the shapes now in the sky model (the whole-chain driver keeps them)
    if (pc.update && e1c && ok && selected) {
        e1c[i] = b1;
        e2c[i] = b2;
    }
}

struct SkySrc {
    double l, m, n1;
    float lh, ll, mh, ml, nh, nl;       // direction cosines as float pairs (split phase)
    float flux, q0, q1, q2, qn0, qn1, qn2, pad;
};

// Mixed precision sky model / update.  CG channels per thread (up to 16: the per-(row,
// source) phase work, about 40 instructions in split mode, is shared by CG terms).  kSplit selects
// the float-pair phase argument instead of the FP64 one; kRec (split only) reads the
// call's split-baseline records instead of splitting u, v, w per row.
template <int CG, bool kUpdate, bool kUniform, bool kSplit, bool kGauss, bool kRec = false>
__global__ void __launch_bounds__(kThreads)
sky_mixed_kernel(const double *__restrict__ u, const double *__restrict__ v,
                 const double *__restrict__ w, int64_t n_rows, const ChanTable ch,
                 const SrcRow *__restrict__ table, int32_t n_src, float2 *__restrict__ vis, float sign,
                 const float *__restrict__ rec, const int32_t *__restrict__ perm, int32_t stride)
{
    __shared__ SkySrc sm[kSkyTile];
    const int C = ch.n;
    const int n_groups = (C + CG - 1) / CG;
    const int lanes = kThreads / n_groups;
    const int g = threadIdx.x % n_groups;
    const int lane = threadIdx.x / n_groups;
    const bool thread_on = lane < lanes;
    const int k0 = g * CG;

    float f2[CG], spec[CG], shi[CG], slo[CG];
    double sk[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) {
        const int k = k0 + c;
        const double s = k < C ? ch.s[k] : 0.0;
        sk[c] = s;
        f2[c] = (float)(s * s);
        spec[c] = k < C ? (float)ch.spec[k] : 0.0f;
        shi[c] = k < C ? ch.s_hi[k] : 0.0f;
        slo[c] = k < C ? ch.s_lo[k] : 0.0f;
    }
    // uniform channels in pairs: two channels per paired FP32 instruction
    constexpr bool kPair = kUniform && CG >= 2 && CG % 2 == 0;
    constexpr int NP2 = kPair ? CG / 2 : 1;
    f32x2 F2[NP2];
#pragma unroll
    for (int j = 0; j < NP2; ++j) F2[j] = kPair ? pk2(f2[2 * j], f2[2 * j + 1]) : pk2(0.0f, 0.0f);
    const double s_k0 = sk[0];
    const double ds = ch.ds;
    constexpr float kTwoPi = 6.28318530717958647692f;

    for (int64_t rb = (int64_t)blockIdx.x * lanes; rb < n_rows; rb += (int64_t)gridDim.x * lanes) {
        // with split records: lane position i in record order, r its row
        const int64_t i = rb + lane;
        const bool act = thread_on && i < n_rows;
        int64_t r = i;
        double ud = 0.0, vd = 0.0, wd = 0.0;
        float uh = 0, ul = 0, vh = 0, vl = 0, wh = 0, wl = 0;
        float uu, uv, vv;
        if constexpr (kSplit && kRec) {
            // the call's split records: no FP64 per row (u^2, uv, v^2 from the high parts,
            // within 1e-7 of the rounded FP64 products, far below the FP32 model's error)
            if (act) {
                if (perm) {
                    if (n_rows <= INT32_MAX) {
                        const int32_t i32 = (int32_t)i;
                        r = (int64_t)(i32 / stride) * stride + perm[i32 % stride];
                    } else {
                        r = (i / stride) * stride + perm[i % stride];
                    }
                }
                const float4 a4 = reinterpret_cast<const float4 *>(rec)[2 * i];
                const float2 b2 = reinterpret_cast<const float2 *>(rec)[4 * i + 2];
                uh = a4.x;
                ul = a4.y;
                vh = a4.z;
                vl = a4.w;
                wh = b2.x;
                wl = b2.y;
            }
            uu = uh * uh;
            uv = uh * vh;
            vv = vh * vh;
        } else {
            if (act) {
                ud = u[r];
                vd = v[r];
                wd = w[r];
            }
            if (kSplit) {
                split_double(ud, uh, ul);
                split_double(vd, vh, vl);
                split_double(wd, wh, wl);
            }
            uu = (float)(ud * ud);
            uv = (float)(ud * vd);
            vv = (float)(vd * vd);
        }
        float are[CG], aim[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) are[c] = aim[c] = 0.0f;
        f32x2 are2[NP2], aim2[NP2];
#pragma unroll
        for (int j = 0; j < NP2; ++j) are2[j] = aim2[j] = pk2(0.0f, 0.0f);

        for (int t0 = 0; t0 < n_src; t0 += kSkyTile) {
            const int nt = min(kSkyTile, n_src - t0);
            __syncthreads();
            for (int j = threadIdx.x; j < nt; j += kThreads) {
                const SrcRow &R = table[t0 + j];
                SkySrc s;
                s.l = R.l;
                s.m = R.m;
                s.n1 = R.n1;
                split_double(R.l, s.lh, s.ll);
                split_double(R.m, s.mh, s.ml);
                split_double(R.n1, s.nh, s.nl);
                s.flux = (float)R.flux;
                s.q0 = (float)R.q[0];
                s.q1 = (float)R.q[1];
                s.q2 = (float)R.q[2];
                s.qn0 = (float)R.qn[0];
                s.qn1 = (float)R.qn[1];
                s.qn2 = (float)R.qn[2];
                s.pad = 0.0f;
                sm[j] = s;
            }
            __syncthreads();
            if (!act) continue;
            for (int j = 0; j < nt; ++j) {
                const SkySrc &S = sm[j];
                if (S.flux == 0.0f) continue;
                const float q = fmaf(S.q2, vv, fmaf(S.q1, uv, S.q0 * uu));
                float qn = 0.0f;
                if (kUpdate) qn = fmaf(S.qn2, vv, fmaf(S.qn1, uv, S.qn0 * uu));
                // phase argument and its reduction to [-1/2, 1/2] cycles
                double ph = 0.0;
                float P = 0.0f, E = 0.0f;
                if (kSplit) phase_metres(uh, ul, vh, vl, wh, wl, S.lh, S.ll, S.mh, S.ml, S.nh, S.nl, P, E);
                else ph = fma(wd, S.n1, fma(vd, S.m, ud * S.l));
                float sn, cs, sd = 0.0f, cd = 1.0f;
                if (kUniform) {
                    float f0, fd = 0.0f;
                    if (kSplit) {
                        f0 = frac_cycles(P, E, shi[0], slo[0]);
                        if (CG > 1) fd = frac_cycles(P, E, ch.ds_hi, ch.ds_lo);
                    } else {
                        const double t = ph * s_k0;
                        f0 = (float)(t - rint(t));
                        if (CG > 1) {
                            const double td = ph * ds;
                            fd = (float)(td - rint(td));
                        }
                    }
                    __sincosf(f0 * kTwoPi, &sn, &cs);
                    if (CG > 1) __sincosf(fd * kTwoPi, &sd, &cd);
                }
                if constexpr (kPair) {
                    // channel pairs (2j, 2j + 1): phasors z_2j and z_2j+1 = z_2j d, then both
                    // turned by d^2 for the next pair; lane by lane the arithmetic of the
                    // scalar loop below
                    const float cs1 = cs * cd - sn * sd, sn1 = fmaf(cs, sd, sn * cd);
                    f32x2 C2 = pk2(cs, cs1), S2 = pk2(sn, sn1);
                    const float cdd = cd * cd - sd * sd, sdd = 2.0f * cd * sd;
                    const f32x2 CD = pk2(cdd, cdd), SD = pk2(sdd, sdd), NSD = pk2(-sdd, -sdd);
                    const f32x2 Q2 = pk2(q, q), QN2 = pk2(qn, qn), FL = pk2(S.flux, S.flux);
#pragma unroll
                    for (int pr = 0; pr < NP2; ++pr) {
                        f32x2 M2 = brightness2<kGauss>(Q2, F2[pr]);
                        if (kUpdate) M2 = fma2(M2, pk2(-1.0f, -1.0f), brightness2<kGauss>(QN2, F2[pr]));
                        const f32x2 A2 = mul2(FL, M2);
                        are2[pr] = fma2(A2, C2, are2[pr]);
                        aim2[pr] = fma2(A2, S2, aim2[pr]);
                        if (pr + 1 < NP2) {
                            const f32x2 Cn = fma2(C2, CD, mul2(S2, NSD));
                            S2 = fma2(C2, SD, mul2(S2, CD));
                            C2 = Cn;
                        }
                    }
                    continue;
                }
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    if (!kUniform) {
                        float f;
                        if (kSplit) {
                            f = frac_cycles(P, E, shi[c], slo[c]);
                        } else {
                            const double t = ph * sk[c];
                            f = (float)(t - rint(t));
                        }
                        __sincosf(f * kTwoPi, &sn, &cs);
                    }
                    float M = brightness<kGauss>(q, f2[c]);
                    if (kUpdate) M = brightness<kGauss>(qn, f2[c]) - M;
                    const float a = S.flux * M;
                    are[c] = fmaf(a, cs, are[c]);
                    aim[c] = fmaf(a, sn, aim[c]);
                    if (kUniform && c + 1 < CG) {
                        const float cn = cs * cd - sn * sd;
                        sn = fmaf(cs, sd, sn * cd);
                        cs = cn;
                    }
                }
            }
        }
        if constexpr (kPair) {
#pragma unroll
            for (int j = 0; j < NP2; ++j) {
                up2(are2[j], are[2 * j], are[2 * j + 1]);
                up2(aim2[j], aim[2 * j], aim[2 * j + 1]);
            }
        }
        if (act) {
            // channel pairs as one 16-byte access when the layout allows (even channel
            // count: a pair starts on an even complex index); the update adds sign * terms
            if (CG >= 2 && C % 2 == 0) {
#pragma unroll
                for (int c = 0; c < CG; c += 2) {
                    const int k = k0 + c;
                    if (k < C) {
                        float4 o = make_float4(are[c] * spec[c], aim[c] * spec[c], are[c + 1] * spec[c + 1],
                                               aim[c + 1] * spec[c + 1]);
                        float4 *dst = reinterpret_cast<float4 *>(vis + (r * C + k));
                        if (kUpdate) {
                            const float4 p = *dst;
                            o = make_float4(fmaf(sign, o.x, p.x), fmaf(sign, o.y, p.y), fmaf(sign, o.z, p.z),
                                            fmaf(sign, o.w, p.w));
                        }
                        *dst = o;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int k = k0 + c;
                    if (k < C) {
                        float2 o = make_float2(are[c] * spec[c], aim[c] * spec[c]);
                        if (kUpdate) {
                            const float2 p = vis[r * C + k];
                            o.x = fmaf(sign, o.x, p.x);
                            o.y = fmaf(sign, o.y, p.y);
                        }
                        vis[r * C + k] = o;
                    }
                }
            }
        }
    }
}

// FP64 sky model / update: every operation in double precision.
template <bool kUpdate>
__global__ void __launch_bounds__(kThreads)
sky_fp64_kernel(const double *__restrict__ u, const double *__restrict__ v,
                const double *__restrict__ w, int64_t n_rows, const ChanTable ch,
                const SrcRow *__restrict__ table, int32_t n_src, float2 *__restrict__ vis, double sign)
{
    __shared__ SrcRow sm[kSkyTile / 2];
    constexpr int kTile = kSkyTile / 2;
    const int C = ch.n;
    const int64_t n_out = n_rows * C;
    for (int64_t ob = (int64_t)blockIdx.x * kThreads; ob < n_out; ob += (int64_t)gridDim.x * kThreads) {
        const int64_t o = ob + threadIdx.x;
        const bool act = o < n_out;
        const int64_t r = act ? o / C : 0;
        const int k = act ? (int)(o % C) : 0;
        const double ud = act ? u[r] : 0.0, vd = act ? v[r] : 0.0, wd = act ? w[r] : 0.0;
        const double s = ch.s[k];
        const double f2 = s * s;
        double are = 0.0, aim = 0.0;
        for (int t0 = 0; t0 < n_src; t0 += kTile) {
            const int nt = min(kTile, n_src - t0);
            __syncthreads();
            for (int j = threadIdx.x; j < nt; j += kThreads) sm[j] = table[t0 + j];
            __syncthreads();
            if (!act) continue;
            for (int j = 0; j < nt; ++j) {
                const SrcRow &S = sm[j];
                if (S.flux == 0.0) continue;
                const double t = fma(wd, S.n1, fma(vd, S.m, ud * S.l)) * s;
                double sn, cs;
                sincospi(2.0 * (t - rint(t)), &sn, &cs);
                const double q = (S.q[0] * ud * ud + S.q[1] * ud * vd + S.q[2] * vd * vd) * f2;
                double M = brightness64(q, ch.profile);
                if (kUpdate)
                    M = brightness64((S.qn[0] * ud * ud + S.qn[1] * ud * vd + S.qn[2] * vd * vd) * f2, ch.profile) - M;
                are += S.flux * M * cs;
                aim += S.flux * M * sn;
            }
        }
        if (act) {
            const double sp = ch.spec[k];
            float2 out = make_float2((float)(are * sp), (float)(aim * sp));
            if (kUpdate) {
                const float2 p = vis[o];
                out.x = (float)((double)p.x + sign * are * sp);
                out.y = (float)((double)p.y + sign * aim * sp);
            }
            vis[o] = out;
        }
    }
}

int sm_count()
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

template <int CG, bool kUpdate, bool kSplit>
void launch_mixed(const rlf_uvw &uvw, const ChanTable &ch, const SrcRow *table, int32_t n_src,
                  float *vis, int blocks_per_sm, float sign, const SplitRows &sr, cudaStream_t st)
{
    const int n_groups = (ch.n + CG - 1) / CG;
    const int lanes = kThreads / n_groups;
    const int64_t blocks_needed = (uvw.n_rows + lanes - 1) / lanes;
    const int64_t cap = (int64_t)sm_count() * blocks_per_sm;
    const int grid = (int)(blocks_needed < cap ? blocks_needed : cap);
    float2 *out = reinterpret_cast<float2 *>(vis);
    const bool gauss = ch.profile == RLF_PROFILE_GAUSSIAN;
    auto pick = [&](auto rec_tag) {
        constexpr bool kRec = decltype(rec_tag)::value;
        if (ch.uniform && !gauss) return sky_mixed_kernel<CG, kUpdate, true, kSplit, false, kRec>;
        if (ch.uniform) return sky_mixed_kernel<CG, kUpdate, true, kSplit, true, kRec>;
        if (!gauss) return sky_mixed_kernel<CG, kUpdate, false, kSplit, false, kRec>;
        return sky_mixed_kernel<CG, kUpdate, false, kSplit, true, kRec>;
    };
    auto kern = pick(std::false_type{});
    if constexpr (kSplit) {
        if (sr.rec) kern = pick(std::true_type{});
    }
    kern<<<grid, kThreads, 0, st>>>(uvw.u, uvw.v, uvw.w, uvw.n_rows, ch, table, n_src, out, sign, sr.rec, sr.perm,
                                    sr.stride);
}

template <bool kUpdate, bool kSplit>
void launch_mixed_cg(const rlf_uvw &uvw, const ChanTable &ch, const SrcRow *table,
                     int32_t n_src, float *vis, int bps, float sign, const SplitRows &sr, cudaStream_t st)
{
    if (ch.n == 1) launch_mixed<1, kUpdate, kSplit>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
    else if (ch.n == 2) launch_mixed<2, kUpdate, kSplit>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
    else if (ch.n <= 4) launch_mixed<4, kUpdate, kSplit>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
    // 16 channels per thread share the per-(row, source) phase work when there are enough
    // sources to make the kernel compute bound; a few sources (the serial order's updates)
    // stream the visibilities, where 8 channels per thread (more warps) go faster
    else if (ch.n <= 8 || n_src < 32) launch_mixed<8, kUpdate, kSplit>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
    else launch_mixed<16, kUpdate, kSplit>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
}

}  // namespace

cudaError_t launch_prepare(const rlf_sources &src, int32_t first, int32_t count,
                           const double *e1, const double *e2, const double *e1n,
                           const double *e2n, const int32_t *flag, int32_t update_mode,
                           double *e1_commit, double *e2_commit,
                           const rlf_params &p, SrcRow *out, int32_t *status, cudaStream_t st,
                           const int32_t *list)
{
    PrepConst pc{p.add, p.esp, p.psf_nat, e1n != nullptr, update_mode};
    const int grid = (count + kThreads - 1) / kThreads;
    prepare_kernel<<<grid, kThreads, 0, st>>>(src, first, count, e1, e2, e1n, e2n, flag, e1_commit,
                                              e2_commit, pc, out, status, list);
    return cudaGetLastError();
}

cudaError_t launch_sky(const rlf_uvw &uvw, const ChanTable &ch, const SrcRow *table, int32_t n_src,
                       bool update, int32_t precision, float *vis, cudaStream_t st, int32_t blocks_per_sm,
                       float sign, const SplitRows &sr)
{
    const int bps = blocks_per_sm > 0 ? blocks_per_sm : 8;
    const SplitRows none;
    if (precision == RLF_PREC_MIXED) {
        if (update) launch_mixed_cg<true, false>(uvw, ch, table, n_src, vis, bps, sign, none, st);
        else launch_mixed_cg<false, false>(uvw, ch, table, n_src, vis, bps, 1.0f, none, st);
    } else if (precision == RLF_PREC_MIXED_SPLIT) {
        if (update) launch_mixed_cg<true, true>(uvw, ch, table, n_src, vis, bps, sign, sr, st);
        else launch_mixed_cg<false, true>(uvw, ch, table, n_src, vis, bps, 1.0f, sr, st);
    } else {
        const int64_t n_out = uvw.n_rows * ch.n;
        const int64_t need = (n_out + kThreads - 1) / kThreads;
        const int64_t cap = (int64_t)sm_count() * 8;
        const int grid = (int)(need < cap ? need : cap);
        if (update)
            sky_fp64_kernel<true><<<grid, kThreads, 0, st>>>(uvw.u, uvw.v, uvw.w, uvw.n_rows, ch, table,
                                                             n_src, reinterpret_cast<float2 *>(vis), (double)sign);
        else
            sky_fp64_kernel<false><<<grid, kThreads, 0, st>>>(uvw.u, uvw.v, uvw.w, uvw.n_rows, ch, table,
                                                              n_src, reinterpret_cast<float2 *>(vis), 1.0);
    }
    return cudaGetLastError();
}

}  // namespace rlf
