// Facet extraction (Sec. 2.3): residual isolation, phase shift to the source and
// averaging of the shifted visibilities into a facet_n x facet_n uv grid of
// cell side du = 1 / (K alpha).
//
// One CTA owns (source, chunk of rows) and accumulates a private copy of the
// facet in shared memory (4 planes: sum Re x, sum Im x, count, sum of the
// spectral factor) with shared-memory atomics; at the end the non-empty cells
// are added to the FP64 facet in global memory.  blockIdx.x runs over the
// sources so the CTAs that read the same row chunk run together and share it
// through L2.
//
// The residual of source i is D - V_sky + model_i; model_i carries the phase
// exp(+2 pi i phi_i), so after the shift it is the real number S s M(k) and
// x = (D - V_sky) exp(-2 pi i phi_i) + S s M(k).
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

__device__ __forceinline__ bool near_edge(float t)
{
    // |error| of t = fl(fl(u) * fl(s/du)) is below 3 * 2^-24 |t|; keep a 5x margin
    return fabsf(t - rintf(t)) <= 1.0e-6f * fmaxf(fabsf(t), 1.0f);
}

template <bool kMixed, int CG, bool kUniform>
__global__ void __launch_bounds__(kThreads)
extract_kernel(const double *__restrict__ u, const double *__restrict__ v,
               const double *__restrict__ w, int64_t n_rows, const ChanTable ch,
               const float2 *__restrict__ data, const float2 *__restrict__ sky,
               const SrcRow *__restrict__ table, int32_t N, int64_t rows_per_chunk,
               double *__restrict__ facets)
{
    using Acc = typename std::conditional<kMixed, float, double>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    Acc *acc = reinterpret_cast<Acc *>(smraw);
    const int NN = N * N;
    const int s = blockIdx.x;
    const SrcRow S = table[s];

    for (int i = threadIdx.x; i < 4 * NN; i += kThreads) acc[i] = Acc(0);
    __syncthreads();

    const int C = ch.n;
    const int n_groups = (C + CG - 1) / CG;
    const int lanes = kThreads / n_groups;
    const int g = threadIdx.x % n_groups;
    const int lane = threadIdx.x / n_groups;
    const int k0 = g * CG;
    const int half = N / 2;
    const double du = S.du;
    constexpr float kTwoPi = 6.28318530717958647692f;

    if (S.flux > 0.0 && lane < lanes) {
        double sk[CG];
        float sdu[CG], f2[CG], spec[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) {
            const int k = k0 + c;
            sk[c] = k < C ? ch.s[k] : 0.0;
            sdu[c] = (float)(sk[c] / du);
            f2[c] = (float)(sk[c] * sk[c]);
            spec[c] = k < C ? (float)ch.spec[k] : 0.0f;
        }
        const float sflux = (float)S.flux;
        const float q0 = (float)S.q[0], q1 = (float)S.q[1], q2 = (float)S.q[2];
        const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
        const int64_t r1 = min(n_rows, r0 + rows_per_chunk);
        for (int64_t r = r0 + lane; r < r1; r += lanes) {
            const double ud = u[r], vd = v[r], wd = w[r];
            const double ph = fma(wd, S.n1, fma(vd, S.m, ud * S.l));
            if (kMixed) {
                const float uf = (float)ud, vf = (float)vd;
                const float uu = (float)(ud * ud), uv = (float)(ud * vd), vv = (float)(vd * vd);
                const float q = fmaf(q2, vv, fmaf(q1, uv, q0 * uu));
                float sn = 0.0f, cs = 1.0f, sd = 0.0f, cd = 1.0f;
                if (kUniform) {
                    const double t = ph * sk[0];
                    __sincosf((float)(t - rint(t)) * kTwoPi, &sn, &cs);
                    if (CG > 1) {
                        const double td = ph * ch.ds;
                        __sincosf((float)(td - rint(td)) * kTwoPi, &sd, &cd);
                    }
                }
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int k = k0 + c;
                    if (!kUniform) {
                        const double t = ph * sk[c];
                        __sincosf((float)(t - rint(t)) * kTwoPi, &sn, &cs);
                    }
                    if (k < C) {
                        const float tu = uf * sdu[c], tv = vf * sdu[c];
                        if (fabsf(tu) < half + 1.0f && fabsf(tv) < half + 1.0f) {
                            int iu = (int)floorf(tu), iv = (int)floorf(tv);
                            if (near_edge(tu)) iu = (int)floor((ud * sk[c]) / du);
                            if (near_edge(tv)) iv = (int)floor((vd * sk[c]) / du);
                            iu += half;
                            iv += half;
                            if (iu >= 0 && iu < N && iv >= 0 && iv < N) {
                                const float2 dv = data[r * C + k];
                                const float2 sv = sky[r * C + k];
                                const float rr = dv.x - sv.x, ri = dv.y - sv.y;
                                // (rr + i ri) exp(-2 pi i f) = (rr + i ri)(cs - i sn)
                                float xr = fmaf(rr, cs, ri * sn);
                                const float xi = fmaf(ri, cs, -rr * sn);
                                const float rq = rsqrtf(fmaf(q, f2[c], 1.0f));
                                xr = fmaf(sflux * spec[c], rq * rq * rq, xr);
                                const int cell = iv * N + iu;
                                atomicAdd(&acc[cell], xr);
                                atomicAdd(&acc[NN + cell], xi);
                                atomicAdd(&acc[2 * NN + cell], 1.0f);
                                atomicAdd(&acc[3 * NN + cell], spec[c]);
                            }
                        }
                    }
                    if (kUniform && c + 1 < CG) {
                        const float cn = cs * cd - sn * sd;
                        sn = fmaf(cs, sd, sn * cd);
                        cs = cn;
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int k = k0 + c;
                    if (k >= C) continue;
                    const double ku = ud * sk[c], kv = vd * sk[c];
                    const double fu = floor(ku / du), fv = floor(kv / du);
                    if (fu < -half || fu >= half || fv < -half || fv >= half) continue;
                    const int iu = (int)fu + half, iv = (int)fv + half;
                    const float2 dv = data[r * C + k];
                    const float2 sv = sky[r * C + k];
                    const double rr = (double)dv.x - (double)sv.x, ri = (double)dv.y - (double)sv.y;
                    const double t = ph * sk[c];
                    double sn, cs;
                    sincospi(2.0 * (t - rint(t)), &sn, &cs);
                    double xr = rr * cs + ri * sn;
                    const double xi = ri * cs - rr * sn;
                    const double x = 1.0 + (S.q[0] * ud * ud + S.q[1] * ud * vd + S.q[2] * vd * vd) * sk[c] * sk[c];
                    xr += S.flux * ch.spec[k] / (x * sqrt(x));
                    const int cell = iv * N + iu;
                    atomicAdd(&acc[cell], (Acc)xr);
                    atomicAdd(&acc[NN + cell], (Acc)xi);
                    atomicAdd(&acc[2 * NN + cell], Acc(1));
                    atomicAdd(&acc[3 * NN + cell], (Acc)ch.spec[k]);
                }
            }
        }
    }
    __syncthreads();
    double *f = facets + (size_t)s * 4 * NN;
    for (int i = threadIdx.x; i < NN; i += kThreads) {
        if (acc[2 * NN + i] != Acc(0)) {
            atomicAdd(&f[i], (double)acc[i]);
            atomicAdd(&f[NN + i], (double)acc[NN + i]);
            atomicAdd(&f[2 * NN + i], (double)acc[2 * NN + i]);
            atomicAdd(&f[3 * NN + i], (double)acc[3 * NN + i]);
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

template <bool kMixed, int CG>
cudaError_t launch_cg(const rlf_uvw &uvw, const ChanTable &ch, const float *data, const float *sky,
                      const SrcRow *table, int32_t count, int32_t N, double *facets,
                      cudaStream_t st)
{
    const size_t acc_bytes = kMixed ? sizeof(float) : sizeof(double);
    const size_t smem = 4 * (size_t)N * N * acc_bytes;
    auto kern = ch.uniform ? extract_kernel<kMixed, CG, true> : extract_kernel<kMixed, CG, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // Row chunks: enough CTAs for several waves, and a chunk of rows small enough
    // (about 16 MB of visibilities and baselines) that the CTAs of all sources
    // reading it at the same time find it in L2.
    const int n_groups = (ch.n + CG - 1) / CG;
    const int64_t lanes = kThreads / n_groups;
    const int64_t target = (int64_t)sm_count_x() * per_sm * 4;
    int64_t n_chunks = (target + count - 1) / count;
    const double bytes = (double)uvw.n_rows * (16.0 * ch.n + 24.0);
    const int64_t by_l2 = (int64_t)(bytes / 16.0e6) + 1;
    if (by_l2 > n_chunks) n_chunks = by_l2;
    const int64_t max_chunks = (uvw.n_rows + lanes - 1) / lanes;
    if (n_chunks > max_chunks) n_chunks = max_chunks;
    if (n_chunks < 1) n_chunks = 1;
    if (n_chunks > 65535) n_chunks = 65535;
    const int64_t rows_per_chunk = (uvw.n_rows + n_chunks - 1) / n_chunks;
    dim3 grid(count, (unsigned)n_chunks);
    kern<<<grid, kThreads, smem, st>>>(uvw.u, uvw.v, uvw.w, uvw.n_rows, ch,
                                       reinterpret_cast<const float2 *>(data),
                                       reinterpret_cast<const float2 *>(sky), table, N,
                                       rows_per_chunk, facets);
    return cudaGetLastError();
}

template <bool kMixed>
cudaError_t launch_prec(const rlf_uvw &uvw, const ChanTable &ch, const float *data,
                        const float *sky, const SrcRow *table, int32_t count, int32_t N,
                        double *facets, cudaStream_t st)
{
    if (ch.n == 1) return launch_cg<kMixed, 1>(uvw, ch, data, sky, table, count, N, facets, st);
    if (ch.n == 2) return launch_cg<kMixed, 2>(uvw, ch, data, sky, table, count, N, facets, st);
    if (ch.n <= 4) return launch_cg<kMixed, 4>(uvw, ch, data, sky, table, count, N, facets, st);
    return launch_cg<kMixed, 8>(uvw, ch, data, sky, table, count, N, facets, st);
}

}  // namespace

cudaError_t launch_extract(const rlf_uvw &uvw, const ChanTable &ch, const float *data,
                           const float *sky, const SrcRow *table, int32_t count,
                           const rlf_params &p, double *facets, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(facets, 0, (size_t)count * 4 * p.facet_n * p.facet_n * sizeof(double), st);
    if (e != cudaSuccess) return e;
    if (p.precision == RLF_PREC_MIXED)
        return launch_prec<true>(uvw, ch, data, sky, table, count, p.facet_n, facets, st);
    return launch_prec<false>(uvw, ch, data, sky, table, count, p.facet_n, facets, st);
}

}  // namespace rlf
