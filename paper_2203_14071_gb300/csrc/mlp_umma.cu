// First layer of the proposal network on the fifth-generation tensor cores:
//   part[z][m][n] = sum over k in slice z of x[m][k] W1[k][n],   m < M, n < 256,
// the 8192-long K range cut into n_slices equal slices (splitk_reduce_kernel then
// adds the slices in order with the bias and the ReLU).
//
// A CTA computes the 128 x 256 block (rows m0 .. m0 + 127, every n) of one slice with
// tcgen05.mma (kind::f16: f16 operands, f32 accumulation) into 256 TMEM columns.  Both
// operands are staged K-major in shared memory by TMA (cp.async.bulk.tensor, 128-byte
// swizzle) through a ring of four stages of 64 K-values; full/empty mbarriers pass the
// stages between thread 0 (issues the loads) and thread 32 (issues the MMAs and
// commits each stage back to the loader).  After the last MMA all four warps read the
// accumulator out with tcgen05.ld (warp w owns TMEM lanes, i.e. rows, 32w .. 32w + 31)
// and store their rows of the slice.  Rows past M read as zeros (TMA fills out of
// bounds) and are not stored.
//
// The MMA wants B as [n][k] (K-major); W1 is stored [k][n], so transpose_pad_kernel
// writes W1 transposed into the caller's scratch first (4 MB, a few microseconds).
// The same kernel computes the training's first-layer weight gradient
// dW1 = x^T dz1 (M = 8192, K = the batch): both operands are transposed first into
// zero-padded K-major copies (mlp_dw1_umma).
//
// Every mbarrier wait has a time limit (about 2 s); a wait that runs out sets
// RLF_DEV_TIMEOUT in *status, and the CTA still waits (bounded) for the copies it
// issued, frees its TMEM and returns.
#include <cuda.h>

#include <atomic>
#include <cstdint>

#include "rlf_internal.cuh"

namespace rlf {

namespace {

constexpr int UM = 128, UN = 256, UK = 64, UST = 4, UTHREADS = 128;
constexpr int kMaxDevices = 64;
constexpr uint32_t kTileA = UM * UK * 2, kTileB = UN * UK * 2, kStageBytes = kTileA + kTileB;
constexpr size_t kUmmaSmem = (size_t)UST * kStageBytes + 1024;   // + room to put the ring on a 1 KB boundary
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s of SM clock: the limit of every mbarrier wait
// instruction descriptor of kind::f16: D f32 (bits 4-5 = 1), A and B f16 (bits 7-9 and
// 10-12 = 0), both K-major (bits 15 and 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | ((uint32_t)(UN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);

static_assert(kMlpHidden == UN, "one CTA covers every hidden unit");
static_assert(kStageBytes % 1024 == 0, "stages stay on 1 KB boundaries");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase of the given parity has completed; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// a 2-D box of the tensor map at (c0 = inner element, c1 = row) into shared memory,
// counted on `bar` by its bytes
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128
// bytes (64 f16), groups of 8 rows 1024 bytes apart (stride byte offset), start address
// / 16 in bits 0-13, version 1 in bits 46-47, layout 2 (128-byte swizzle) in bits 61-63.
// The tile starts on a 1 KB boundary (base offset 0); a step of 16 K-values (32 bytes)
// inside the row adds 2 to the start-address field.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

// arrive on `bar` once every MMA this thread issued so far has completed
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 16 consecutive f32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__global__ void __launch_bounds__(UTHREADS, 1)
l1_umma_kernel(const __grid_constant__ CUtensorMap tx, const __grid_constant__ CUtensorMap tw, int M, int kb_per,
               float *__restrict__ part, int32_t *__restrict__ status)
{
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) uint64_t bar_full[UST], bar_empty[UST], bar_done;
    __shared__ uint32_t s_tmem;
    const uint32_t ring = (smem_u32(dsm) + 1023u) & ~1023u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * UM, z = blockIdx.y;
    const int k_first = z * kb_per * UK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < UST; ++s) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        mbar_init(smem_u32(&bar_done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();   // tcgen05.alloc, .ld and .dealloc are warp-wide (.sync.aligned): converge first
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(UN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    bool ok = true;
    if (threadIdx.x == 0) {
        // loader: stage s is free again once the MMAs that read it have committed
        int issued = 0;
        for (int kb = 0; kb < kb_per; ++kb) {
            const int s = kb % UST;
            if (kb >= UST && !mbar_wait(smem_u32(&bar_empty[s]), ((kb / UST) - 1) & 1)) {
                ok = false;
                break;
            }
            const uint32_t full = smem_u32(&bar_full[s]), dst = ring + (uint32_t)s * kStageBytes;
            mbar_expect_tx(full, kStageBytes);
            tma_load_2d(dst, &tx, full, k_first + kb * UK, m0);
            tma_load_2d(dst + kTileA, &tw, full, k_first + kb * UK, 0);
            issued = kb + 1;
        }
        // the copies of the last stages this thread issued have landed before the CTA can
        // leave (bounded; they have in any run whose MMAs completed)
        for (int kb = issued > UST ? issued - UST : 0; kb < issued; ++kb)
            if (!mbar_wait(smem_u32(&bar_full[kb % UST]), (kb / UST) & 1)) ok = false;
    } else if (threadIdx.x == 32) {
        // MMA issuer: four K-steps of 16 per stage, accumulating after the first
        for (int kb = 0; kb < kb_per; ++kb) {
            const int s = kb % UST;
            if (!mbar_wait(smem_u32(&bar_full[s]), (kb / UST) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = ring + (uint32_t)s * kStageBytes;
            const uint64_t da = desc_sw128(a), db = desc_sw128(a + kTileA);
#pragma unroll
            for (int k = 0; k < UK / 16; ++k)
                umma_f16(tmem, da + (uint64_t)(2 * k), db + (uint64_t)(2 * k), (kb | k) != 0 ? 1u : 0u);
            umma_commit(smem_u32(&bar_empty[s]));
        }
        umma_commit(smem_u32(&bar_done));
    }
    __syncwarp();
    if (!mbar_wait(smem_u32(&bar_done), 0)) ok = false;
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    const bool store = ok && row < M;
    float *dst = part + ((size_t)z * M + (store ? row : 0)) * UN;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < UN; c += 16) {
        uint32_t r[16];
        tmem_ld16(tl + (uint32_t)c, r);
        if (store) {
            float4 *o = reinterpret_cast<float4 *>(dst + c);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                   __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
    }
    if (!ok) atomicOr(status, RLF_DEV_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    __syncwarp();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(UN) : "memory");
}

// out[c][r] = in[r][c] (r < rows), 0 (rows <= r < ld_out), for an f16 matrix in
// [rows][cols] (cols and ld_out multiples of 32), through 32 x 32 shared tiles
__global__ void transpose_pad_kernel(const __half *__restrict__ in, int rows, int cols, __half *__restrict__ out,
                                     int ld_out)
{
    __shared__ __half t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int j = ty; j < 32; j += 8)
        t[j][tx] = r0 + j < rows ? in[(size_t)(r0 + j) * cols + c0 + tx] : __float2half(0.0f);
    __syncthreads();
    for (int j = ty; j < 32; j += 8) out[(size_t)(c0 + j) * ld_out + r0 + tx] = t[tx][j];
}

cudaError_t transpose_pad(const __half *in, int rows, int cols, __half *out, int ld_out, cudaStream_t st)
{
    transpose_pad_kernel<<<dim3(cols / 32, ld_out / 32), dim3(32, 8), 0, st>>>(in, rows, cols, out, ld_out);
    return cudaGetLastError();
}

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime (no -lcuda)
EncodeTiled encode_tiled()
{
    static const EncodeTiled fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<EncodeTiled>(p);
    }();
    return fn;
}

// row-major [outer][inner] f16 matrix, boxes of box_outer rows x box_inner (128 bytes)
bool tensor_map_2d(CUtensorMap *map, const __half *base, uint64_t inner, uint64_t outer, uint32_t box_inner,
                   uint32_t box_outer)
{
    const EncodeTiled enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {inner, outer}, strides[1] = {inner * sizeof(__half)};
    const cuuint32_t box[2] = {box_inner, box_outer}, estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// part[z][m][n] = sum over k in slice z of A[m][k] Bt[n][k], m < M, n < 256: A
// [M][K] and Bt [256][K] f16, K-major, 16-byte aligned, K a multiple of 64 n_slices
cudaError_t umma_gemm_nt(const __half *A, int32_t M, int32_t K, const __half *Bt, float *part, int32_t n_slices,
                         int32_t *status, cudaStream_t st)
{
    if (M <= 0 || K <= 0 || n_slices <= 0 || K % (n_slices * UK) != 0 || (reinterpret_cast<uintptr_t>(A) & 15u) != 0 ||
        (reinterpret_cast<uintptr_t>(Bt) & 15u) != 0)
        return cudaErrorInvalidValue;
    CUtensorMap ta, tb;
    if (!tensor_map_2d(&ta, A, (uint64_t)K, (uint64_t)M, UK, UM) || !tensor_map_2d(&tb, Bt, (uint64_t)K, UN, UK, UN))
        return cudaErrorNotSupported;
    // the kernel's shared-memory limit, raised once per device (setting a function
    // attribute on every launch can stall the host behind the kernel's running launches)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static std::atomic<bool> smem_set[kMaxDevices];
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!smem_set[dev].load(std::memory_order_acquire)) {
        e = cudaFuncSetAttribute(l1_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kUmmaSmem);
        if (e != cudaSuccess) return e;
        smem_set[dev].store(true, std::memory_order_release);
    }
    l1_umma_kernel<<<dim3((M + UM - 1) / UM, n_slices), UTHREADS, kUmmaSmem, st>>>(ta, tb, M, K / (n_slices * UK),
                                                                                  part, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_layer1_umma(const __half *x, int32_t M, const __half *W1h, __half *W1t, float *part, int32_t n_slices,
                            int32_t *status, cudaStream_t st)
{
    // B operand: W1 [8192][256] transposed to [256][8192]
    cudaError_t e = transpose_pad(W1h, kMlpIn, kMlpHidden, W1t, kMlpIn, st);
    if (e == cudaSuccess) e = umma_gemm_nt(x, M, kMlpIn, W1t, part, n_slices, status, st);
    return e;
}

cudaError_t mlp_dw1_umma(const __half *x, int32_t B, const __half *dz1, __half *xT, __half *dzT, float *dW1,
                         int32_t *status, cudaStream_t st)
{
    // dW1[k][n] = sum over b of x[b][k] dz1[b][n]: both operands transposed to K-major
    // ([8192][Bp] and [256][Bp], the batch zero-padded to Bp, a multiple of 64)
    const int Bp = mlp_batch_pad(B);
    if (B <= 0 || (reinterpret_cast<uintptr_t>(dW1) & 15u) != 0) return cudaErrorInvalidValue;   // 16-byte stores
    cudaError_t e = transpose_pad(x, B, kMlpIn, xT, Bp, st);
    if (e == cudaSuccess) e = transpose_pad(dz1, B, kMlpHidden, dzT, Bp, st);
    if (e == cudaSuccess) e = umma_gemm_nt(xT, kMlpIn, Bp, dzT, dW1, 1, status, st);
    return e;
}

}  // namespace rlf
