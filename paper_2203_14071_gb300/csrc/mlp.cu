// Learned proposal of the likelihood sub-grid (an addition to the method; no
// counterpart in the paper): a 8192-256-256-6 perceptron reads a facet and
// predicts the mean and log-variance of (e1, e2, ln alpha); the fit then
// evaluates only a 7 x 7 x 5 box of the grid around the prediction.
//
// Kernels: the first layer's forward GEMM and its weight gradient on tcgen05
// (mlp_umma.cu); the other GEMMs on mma.sync m16n8k16 (f16 inputs, f32
// accumulation; K = 256 or the batch)
// with fused epilogues for the forward and backward passes, the Gaussian NLL and
// its gradient, bias-gradient column sums, Adam, the facet encoder, the training
// facet simulator and the proposal rule.  Weights: f32 masters + f16 copies.
#include <cuda_fp16.h>

#include <cmath>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8, GTHREADS = 128;
constexpr int kL1Slices = 16;   // K slices of the first layer's forward GEMM

enum { EPI_F32 = 0, EPI_F32_BIAS = 1, EPI_F16_BIAS_RELU = 2, EPI_F16_MASK = 3 };

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[M x N] = op(A)[M x K] op(B)[K x N]; op = transpose when TA / TB.  Row-major
// storage: A(m, k) = TA ? A[k * lda + m] : A[m * lda + k];
//          B(k, n) = TB ? B[n * ldb + k] : B[k * ldb + n].
// Tiles of 64 x 64 x 32 staged in shared memory as As[m][k] and Bt[n][k]; four
// warps each own a 32 x 32 block of mma tiles.  Ragged edges are zero-filled.
// Staging moves 8 halves per 16-byte load when `vec` (both matrices 16-byte
// aligned, leading dimensions multiples of 8).  With gridDim.z > 1 the K range is
// split: slice z sums its share into the f32 partial C32 + z * M * ldc (EPI_F32),
// and splitk_reduce_kernel adds the slices and applies the epilogue.
__device__ __forceinline__ uint4 load8h(const __half *p, int avail, bool vec)
{
    if (vec && avail >= 8) return *reinterpret_cast<const uint4 *>(p);
    __align__(16) __half t[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) t[j] = j < avail ? p[j] : __float2half(0.0f);
    return *reinterpret_cast<const uint4 *>(t);
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(GTHREADS)
gemm_kernel(int M, int N, int K, const __half *__restrict__ A, int lda, const __half *__restrict__ B, int ldb,
            const float *__restrict__ bias, const __half *__restrict__ mask, int ldm, float *__restrict__ C32,
            __half *__restrict__ C16, int ldc, int k_slice, bool vec)
{
    __shared__ __align__(16) __half As[GBM][GBK + GPAD];
    __shared__ __align__(16) __half Bt[GBN][GBK + GPAD];
    const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
    const int kb = blockIdx.z * k_slice, ke = min(K, kb + k_slice);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += GBK) {
        // 64 x 32 halves per operand = 256 groups of 8; two groups per thread
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int i = threadIdx.x + rep * GTHREADS;
            if (!TA) {
                const int m = i >> 2, kq = (i & 3) * 8;
                const int gm = m0 + m, gk = k0 + kq;
                uint4 q = make_uint4(0, 0, 0, 0);
                if (gm < M) q = load8h(A + (size_t)gm * lda + gk, min(8, ke - gk), vec);
                *reinterpret_cast<uint4 *>(&As[m][kq]) = q;
            } else {
                const int k = i >> 3, mq = (i & 7) * 8;
                const int gk = k0 + k, gm = m0 + mq;
                uint4 q = make_uint4(0, 0, 0, 0);
                if (gk < ke) q = load8h(A + (size_t)gk * lda + gm, min(8, M - gm), vec);
                const __half *h = reinterpret_cast<const __half *>(&q);
#pragma unroll
                for (int j = 0; j < 8; ++j) As[mq + j][k] = h[j];
            }
            if (TB) {
                const int n = i >> 2, kq = (i & 3) * 8;
                const int gn = n0 + n, gk = k0 + kq;
                uint4 q = make_uint4(0, 0, 0, 0);
                if (gn < N) q = load8h(B + (size_t)gn * ldb + gk, min(8, ke - gk), vec);
                *reinterpret_cast<uint4 *>(&Bt[n][kq]) = q;
            } else {
                const int k = i >> 3, nq = (i & 7) * 8;
                const int gk = k0 + k, gn = n0 + nq;
                uint4 q = make_uint4(0, 0, 0, 0);
                if (gk < ke) q = load8h(B + (size_t)gk * ldb + gn, min(8, N - gn), vec);
                const __half *h = reinterpret_cast<const __half *>(&q);
#pragma unroll
                for (int j = 0; j < 8; ++j) Bt[nq + j][k] = h[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GBK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int im = 0; im < 2; ++im) {
                const int r = wm + im * 16 + g;
                af[im][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 2 * t]);
                af[im][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 2 * t]);
                af[im][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + 8 + 2 * t]);
                af[im][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int in = 0; in < 4; ++in) {
                const int c = wn + in * 8 + g;
                bf[in][0] = *reinterpret_cast<const uint32_t *>(&Bt[c][kk + 2 * t]);
                bf[in][1] = *reinterpret_cast<const uint32_t *>(&Bt[c][kk + 8 + 2 * t]);
            }
#pragma unroll
            for (int im = 0; im < 2; ++im)
#pragma unroll
                for (int in = 0; in < 4; ++in) mma16816(acc[im][in], af[im], bf[in]);
        }
        __syncthreads();
    }
    float *C32z = C32 ? C32 + (size_t)blockIdx.z * M * ldc : nullptr;
#pragma unroll
    for (int im = 0; im < 2; ++im)
#pragma unroll
        for (int in = 0; in < 4; ++in)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + wm + im * 16 + g + 8 * h;
                if (r >= M) continue;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = n0 + wn + in * 8 + 2 * t + q;
                    if (c >= N) continue;
                    float v = acc[im][in][2 * h + q];
                    if (EPI == EPI_F32) {
                        C32z[(size_t)r * ldc + c] = v;
                    } else if (EPI == EPI_F32_BIAS) {
                        C32[(size_t)r * ldc + c] = v + bias[c];
                    } else if (EPI == EPI_F16_BIAS_RELU) {
                        v += bias[c];
                        C16[(size_t)r * ldc + c] = __float2half(v > 0.0f ? v : 0.0f);
                    } else {
                        const bool on = __half2float(mask[(size_t)r * ldm + c]) > 0.0f;
                        C16[(size_t)r * ldc + c] = __float2half(on ? v : 0.0f);
                    }
                }
            }
}

// h = relu(sum over slices of part[z][M][N] + bias) as f16, slices added in order.
__global__ void splitk_reduce_kernel(const float *__restrict__ part, int n_slices, int M, int N,
                                     const float *__restrict__ bias, __half *__restrict__ h)
{
    const int64_t MN = (int64_t)M * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += (int64_t)gridDim.x * blockDim.x) {
        float v = bias[i % N];
        for (int z = 0; z < n_slices; ++z) v += part[z * MN + i];
        h[i] = __float2half(v > 0.0f ? v : 0.0f);
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const __half *A, int lda, const __half *B, int ldb, const float *bias,
                 const __half *mask, int ldm, float *C32, __half *C16, int ldc, cudaStream_t st, int n_slices = 1)
{
    const int k_slice = ((K + n_slices - 1) / n_slices + GBK - 1) / GBK * GBK;
    const bool vec = aligned16(A) && aligned16(B) && lda % 8 == 0 && ldb % 8 == 0;
    dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM, n_slices);
    gemm_kernel<TA, TB, EPI><<<grid, GTHREADS, 0, st>>>(M, N, K, A, lda, B, ldb, bias, mask, ldm, C32, C16, ldc,
                                                         k_slice, vec);
    return cudaGetLastError();
}

// Gaussian NLL of a batch and its gradient d nll / d o (1/B of the batch mean),
// as f32 and f16 [B][8] (columns 6, 7 zero).  loss (optional) accumulates the mean.
// The log-variance is clamped to [-8, 8] (zero gradient outside), which keeps the
// f16 gradients finite; a spread below e^-4 is finer than the grid needs.
__global__ void nll_kernel(const float *__restrict__ o, const float *__restrict__ y, int B,
                           float *__restrict__ g32, __half *__restrict__ g16, float *__restrict__ loss)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float l = 0.0f;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float mu = o[b * 8 + j], raw = o[b * 8 + 3 + j];
        const float lv = fminf(fmaxf(raw, -8.0f), 8.0f);
        const float r = y[b * 3 + j] - mu;
        const float iv = expf(-lv);
        l += 0.5f * (lv + r * r * iv);
        const float gm = -r * iv / B;
        const float gv = (raw > -8.0f && raw < 8.0f) ? 0.5f * (1.0f - r * r * iv) / B : 0.0f;
        g32[b * 8 + j] = gm;
        g32[b * 8 + 3 + j] = gv;
        g16[b * 8 + j] = __float2half(gm);
        g16[b * 8 + 3 + j] = __float2half(gv);
    }
    g32[b * 8 + 6] = g32[b * 8 + 7] = 0.0f;
    g16[b * 8 + 6] = g16[b * 8 + 7] = __float2half(0.0f);
    if (loss) atomicAdd(loss, l / B);
}

// out[n] = sum over rows of X[B][N] (f16 or f32), in row order.
template <typename T>
__global__ void colsum_kernel(const T *__restrict__ X, int B, int N, float *__restrict__ out)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += (float)X[(size_t)b * N + n];
    out[n] = s;
}

// Adam (Kingma & Ba 2015) over every parameter; refreshes the f16 weight copies.
__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __half *__restrict__ w16, int64_t P, float lr, float bc1,
                            float bc2, MlpOffsets off)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
        w[i] = wi;
        int64_t h = -1;
        if (i < off.b1) h = i;
        else if (i >= off.W2 && i < off.b2) h = off.W1h_n + (i - off.W2);
        else if (i >= off.W3 && i < off.b3) h = off.W1h_n + off.W2h_n + (i - off.W3);
        if (h >= 0) w16[h] = __float2half(wi);
    }
}

// He initialisation from caller-supplied standard normals; biases zero.
__global__ void init_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            __half *__restrict__ w16, const float *__restrict__ z, int64_t P, MlpOffsets off)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float wi = 0.0f;
        int64_t h = -1;
        if (i < off.b1) {
            wi = z[i] * sqrtf(2.0f / kMlpIn);
            h = i;
        } else if (i >= off.W2 && i < off.b2) {
            wi = z[i] * sqrtf(2.0f / kMlpHidden);
            h = off.W1h_n + (i - off.W2);
        } else if (i >= off.W3 && i < off.b3) {
            const int col = (int)((i - off.W3) % kMlpOutPad);
            wi = col < kMlpOut ? z[i] * sqrtf(1.0f / kMlpHidden) : 0.0f;
            h = off.W1h_n + off.W2h_n + (i - off.W3);
        }
        w[i] = wi;
        m[i] = 0.0f;
        v[i] = 0.0f;
        if (h >= 0) w16[h] = __float2half(wi);
    }
}

// Network input of each facet: [Re D_c / S, Im D_c / S], empty cells 0, f16.
__global__ void encode_kernel(const double *__restrict__ facets, const SrcRow *__restrict__ table, int NN,
                              __half *__restrict__ x)
{
    const int s = blockIdx.y;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= NN) return;
    const double *f = facets + (size_t)s * 4 * NN;
    const double n = f[2 * NN + c];
    const double S = table[s].flux;
    float re = 0.0f, im = 0.0f;
    if (n > 0.0 && S > 0.0) {
        re = (float)(f[c] / n / S);
        im = (float)(f[NN + c] / n / S);
    }
    x[(size_t)s * 2 * NN + c] = __float2half(re);
    x[(size_t)s * 2 * NN + NN + c] = __float2half(im);
}

// Training facets: D_c / S = s_c M(k_c; e, alpha) + (sigma / S) z / sqrt(n_c), from a
// template facet's counts and spectral sums and its cell size.  The result is f16,
// so the arithmetic is FP32.
__global__ void simulate_kernel(const double *__restrict__ tmpl, int n_tmpl, int profile, double add, double esp,
                                double psf_nat, const double *__restrict__ tflux, const int32_t *__restrict__ tidx,
                                const double *__restrict__ e1, const double *__restrict__ e2,
                                const double *__restrict__ alpha_as, const float *__restrict__ z, int N,
                                double sigma, __half *__restrict__ x, float *__restrict__ y)
{
    const int b = blockIdx.y;
    const int NN = N * N;
    const int ti = tidx[b];
    const bool valid = ti >= 0 && ti < n_tmpl;   // an out-of-range template index gives an all-zero input
    const float a1 = (float)e1[b], a2 = (float)e2[b];
    const double flux = valid ? tflux[ti] : 1.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        y[b * 3 + 0] = a1;
        y[b * 3 + 1] = a2;
        y[b * 3 + 2] = (float)log(alpha_as[b]);
    }
    // the template's cell size du = 1 / (K alpha_med(S)) with Eq. 4, and the
    // quadratic form 4 pi^2 alpha^2 |A^-1 k|^2 in cell units (A symmetric)
    const float du = (float)(1.0 / (psf_nat * exp(add + esp * log(flux * 1.0e6)) * kArcsec));
    const float al = (float)(alpha_as[b] * kArcsec);
    const float idet = 1.0f / (1.0f - a1 * a1 - a2 * a2);
    const float c2 = 4.0f * (float)(kPi * kPi) * al * al * du * du * idet * idet;
    const float sr0 = (float)(sigma / flux);
    const double *f = tmpl + (size_t)(valid ? ti : 0) * 4 * NN;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < NN; c += gridDim.x * blockDim.x) {
        const double n = valid ? f[2 * NN + c] : 0.0;
        float re = 0.0f, im = 0.0f;
        if (n > 0.0) {
            const float cu = (float)((c % N) - N / 2) + 0.5f, cv = (float)((c / N) - N / 2) + 0.5f;
            const float x1 = (1.0f + a1) * cu + a2 * cv, x2 = a2 * cu + (1.0f - a1) * cv;
            const float M = profile == RLF_PROFILE_GAUSSIAN ? brightness<true>(c2, x1 * x1 + x2 * x2)
                                                            : brightness<false>(c2, x1 * x1 + x2 * x2);
            const float nf = (float)n;
            const float sbar = (float)(f[3 * NN + c] / n);
            const float sr = sr0 * rsqrtf(nf);
            re = fmaf(sbar, M, sr * z[((size_t)b * 2) * NN + c]);
            im = sr * z[((size_t)b * 2 + 1) * NN + c];
        }
        x[(size_t)b * 2 * NN + c] = __float2half(re);
        x[(size_t)b * 2 * NN + NN + c] = __float2half(im);
    }
}

// Sub-box of the grid centred on the node nearest the prediction, clamped inside
// the grid; `wide` when the predicted spread of e1 or e2 exceeds three node spacings.
__global__ void propose_kernel(const float *__restrict__ o, int count, GridConst gc, int32_t *__restrict__ origin,
                               int32_t *__restrict__ wide)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= count) return;
    const double de = 2.0 * gc.e_max / (gc.n_e - 1);
    int idx[2];
    for (int j = 0; j < 2; ++j) {
        const double mu = o[s * 8 + j];
        int best = 0;
        double bd = 1e300;
        for (int k = 0; k < gc.n_e; ++k) {
            const double d = fabs(-gc.e_max + k * de - mu);
            if (d < bd) {
                bd = d;
                best = k;
            }
        }
        idx[j] = best;
    }
    const double am = exp((double)o[s * 8 + 2]);
    int kb = 0;
    double bd = 1e300;
    for (int k = 0; k < gc.n_alpha; ++k) {
        const double tt = gc.n_alpha > 1 ? (double)k / (gc.n_alpha - 1) : 0.0;
        const double d = fabs(gc.r_min + (gc.r_max - gc.r_min) * tt * tt - am);
        if (d < bd) {
            bd = d;
            kb = k;
        }
    }
    origin[s * 3 + 0] = min(max(idx[0] - kBoxE / 2, 0), gc.n_e - kBoxE);
    origin[s * 3 + 1] = min(max(idx[1] - kBoxE / 2, 0), gc.n_e - kBoxE);
    origin[s * 3 + 2] = min(max(kb - kBoxA / 2, 0), gc.n_alpha - kBoxA);
    const double s1 = exp(0.5 * (double)o[s * 8 + 3]), s2 = exp(0.5 * (double)o[s * 8 + 4]);
    wide[s] = (s1 > 3.0 * de || s2 > 3.0 * de) ? 1 : 0;
}

int sm_count_m()
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

}  // namespace

MlpOffsets mlp_offsets()
{
    MlpOffsets o;
    o.W1 = 0;
    o.b1 = o.W1 + (int64_t)kMlpIn * kMlpHidden;
    o.W2 = o.b1 + kMlpHidden;
    o.b2 = o.W2 + (int64_t)kMlpHidden * kMlpHidden;
    o.W3 = o.b2 + kMlpHidden;
    o.b3 = o.W3 + (int64_t)kMlpHidden * kMlpOutPad;
    o.P = o.b3 + kMlpOutPad;
    o.W1h_n = (int64_t)kMlpIn * kMlpHidden;
    o.W2h_n = (int64_t)kMlpHidden * kMlpHidden;
    o.W3h_n = (int64_t)kMlpHidden * kMlpOutPad;
    return o;
}

MlpWeights mlp_weights(void *blob)
{
    const MlpOffsets o = mlp_offsets();
    MlpWeights w;
    char *b = static_cast<char *>(blob);
    w.w = reinterpret_cast<float *>(b);
    w.m = w.w + o.P;
    w.v = w.m + o.P;
    w.g = w.v + o.P;
    w.h = reinterpret_cast<__half *>(w.g + o.P);
    return w;
}

size_t mlp_weights_bytes()
{
    const MlpOffsets o = mlp_offsets();
    return (size_t)o.P * 4 * sizeof(float) + (size_t)(o.W1h_n + o.W2h_n + o.W3h_n) * sizeof(__half);
}

MlpScratch mlp_scratch(void *base, int32_t max_batch)
{
    MlpScratch s;
    char *b = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        char *p = b;
        b += (bytes + 255) / 256 * 256;
        return p;
    };
    s.h1 = reinterpret_cast<__half *>(take((size_t)max_batch * kMlpHidden * sizeof(__half)));
    s.h2 = reinterpret_cast<__half *>(take((size_t)max_batch * kMlpHidden * sizeof(__half)));
    s.o = reinterpret_cast<float *>(take((size_t)max_batch * kMlpOutPad * sizeof(float)));
    s.g32 = reinterpret_cast<float *>(take((size_t)max_batch * kMlpOutPad * sizeof(float)));
    s.g16 = reinterpret_cast<__half *>(take((size_t)max_batch * kMlpOutPad * sizeof(__half)));
    s.dz2 = reinterpret_cast<__half *>(take((size_t)max_batch * kMlpHidden * sizeof(__half)));
    s.dz1 = reinterpret_cast<__half *>(take((size_t)max_batch * kMlpHidden * sizeof(__half)));
    s.part = reinterpret_cast<float *>(take((size_t)kL1Slices * max_batch * kMlpHidden * sizeof(float)));
    s.w1t = reinterpret_cast<__half *>(take((size_t)kMlpIn * kMlpHidden * sizeof(__half)));
    s.xT = reinterpret_cast<__half *>(take((size_t)kMlpIn * mlp_batch_pad(max_batch) * sizeof(__half)));
    s.dzT = reinterpret_cast<__half *>(take((size_t)kMlpHidden * mlp_batch_pad(max_batch) * sizeof(__half)));
    s.status = reinterpret_cast<int32_t *>(take(sizeof(int32_t)));
    s.bytes = (size_t)(b - static_cast<char *>(base));
    return s;
}

cudaError_t mlp_forward(const MlpWeights &W, const __half *x, int32_t B, const MlpScratch &s, cudaStream_t st)
{
    const MlpOffsets o = mlp_offsets();
    const __half *W1h = W.h, *W2h = W.h + o.W1h_n, *W3h = W.h + o.W1h_n + o.W2h_n;
    // layer 1 (K = 8192) on tcgen05, split over K so that a small batch still fills the GPU
    cudaError_t e = mlp_layer1_umma(x, B, W1h, s.w1t, s.part, kL1Slices, s.status, st);
    if (e == cudaSuccess) {
        const int64_t mn = (int64_t)B * kMlpHidden;
        splitk_reduce_kernel<<<(int)((mn + 255) / 256 < 1024 ? (mn + 255) / 256 : 1024), 256, 0, st>>>(
            s.part, kL1Slices, B, kMlpHidden, W.w + o.b1, s.h1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<false, false, EPI_F16_BIAS_RELU>(B, kMlpHidden, kMlpHidden, s.h1, kMlpHidden, W2h, kMlpHidden,
                                                  W.w + o.b2, nullptr, 0, nullptr, s.h2, kMlpHidden, st);
    if (e == cudaSuccess)
        e = gemm<false, false, EPI_F32_BIAS>(B, kMlpOutPad, kMlpHidden, s.h2, kMlpHidden, W3h, kMlpOutPad,
                                             W.w + o.b3, nullptr, 0, s.o, nullptr, kMlpOutPad, st);
    return e;
}

cudaError_t mlp_train_step(const MlpWeights &W, const __half *x, const float *y, int32_t B, float lr, int32_t step,
                           float *loss, const MlpScratch &s, cudaStream_t st)
{
    const MlpOffsets o = mlp_offsets();
    const __half *W2h = W.h + o.W1h_n, *W3h = W.h + o.W1h_n + o.W2h_n;
    cudaError_t e = mlp_forward(W, x, B, s, st);
    if (e != cudaSuccess) return e;
    nll_kernel<<<(B + 127) / 128, 128, 0, st>>>(s.o, y, B, s.g32, s.g16, loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // layer 3: dW3 = h2^T g, db3 = sum g, dz2 = (g W3^T) * [h2 > 0]
    e = gemm<true, false, EPI_F32>(kMlpHidden, kMlpOutPad, B, s.h2, kMlpHidden, s.g16, kMlpOutPad, nullptr, nullptr,
                                   0, W.g + o.W3, nullptr, kMlpOutPad, st);
    if (e == cudaSuccess) {
        colsum_kernel<float><<<1, kMlpOutPad, 0, st>>>(s.g32, B, kMlpOutPad, W.g + o.b3);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<false, true, EPI_F16_MASK>(B, kMlpHidden, kMlpOutPad, s.g16, kMlpOutPad, W3h, kMlpOutPad, nullptr,
                                            s.h2, kMlpHidden, nullptr, s.dz2, kMlpHidden, st);
    // layer 2: dW2 = h1^T dz2, db2 = sum dz2, dz1 = (dz2 W2^T) * [h1 > 0]
    if (e == cudaSuccess)
        e = gemm<true, false, EPI_F32>(kMlpHidden, kMlpHidden, B, s.h1, kMlpHidden, s.dz2, kMlpHidden, nullptr,
                                       nullptr, 0, W.g + o.W2, nullptr, kMlpHidden, st);
    if (e == cudaSuccess) {
        colsum_kernel<__half><<<(kMlpHidden + 127) / 128, 128, 0, st>>>(s.dz2, B, kMlpHidden, W.g + o.b2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = gemm<false, true, EPI_F16_MASK>(B, kMlpHidden, kMlpHidden, s.dz2, kMlpHidden, W2h, kMlpHidden, nullptr,
                                            s.h1, kMlpHidden, nullptr, s.dz1, kMlpHidden, st);
    // layer 1: dW1 = x^T dz1 (on tcgen05), db1 = sum dz1
    if (e == cudaSuccess) e = mlp_dw1_umma(x, B, s.dz1, s.xT, s.dzT, W.g + o.W1, s.status, st);
    if (e == cudaSuccess) {
        colsum_kernel<__half><<<(kMlpHidden + 127) / 128, 128, 0, st>>>(s.dz1, B, kMlpHidden, W.g + o.b1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess || step <= 0) return e;
    const float bc1 = 1.0f - powf(0.9f, (float)step), bc2 = 1.0f - powf(0.999f, (float)step);
    adam_kernel<<<sm_count_m() * 8, 256, 0, st>>>(W.w, W.g, W.m, W.v, W.h, o.P, lr, bc1, bc2, o);
    return cudaGetLastError();
}

cudaError_t mlp_init(const MlpWeights &W, const float *z, cudaStream_t st)
{
    const MlpOffsets o = mlp_offsets();
    init_kernel<<<sm_count_m() * 8, 256, 0, st>>>(W.w, W.m, W.v, W.h, z, o.P, o);
    return cudaGetLastError();
}

cudaError_t mlp_encode(const double *facets, const SrcRow *table, int32_t count, int32_t N, __half *x,
                       cudaStream_t st)
{
    const int NN = N * N;
    dim3 grid((NN + 255) / 256, count);
    encode_kernel<<<grid, 256, 0, st>>>(facets, table, NN, x);
    return cudaGetLastError();
}

cudaError_t mlp_simulate(const double *tmpl, int32_t n_tmpl, const rlf_params &p, const double *tflux,
                         const int32_t *tidx, const double *e1, const double *e2, const double *alpha_as,
                         const float *z, int32_t B, int32_t N, double sigma, __half *x, float *y, cudaStream_t st)
{
    dim3 grid(4, B);
    simulate_kernel<<<grid, 256, 0, st>>>(tmpl, n_tmpl, p.profile, p.add, p.esp, p.psf_nat, tflux, tidx, e1, e2, alpha_as, z, N,
                                          sigma, x, y);
    return cudaGetLastError();
}

cudaError_t mlp_propose(const float *o, int32_t count, const GridConst &gc, int32_t *origin, int32_t *wide,
                        cudaStream_t st)
{
    propose_kernel<<<(count + 127) / 128, 128, 0, st>>>(o, count, gc, origin, wide);
    return cudaGetLastError();
}

}  // namespace rlf
