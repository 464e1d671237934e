/*
 * rlf_peaks.h - arithmetic-unit throughput microbenchmarks shipped in librlf.so.
 *
 * A measurement utility with no counterpart in the paper: it gives the measured
 * denominators (FP32 FMA as scalar and paired f32x2 instructions, FP64 FMA, MUFU
 * rsqrt and sin per second on the current GPU, at its current clocks) for the
 * ALU rooflines of the hot-path kernels.
 */
#ifndef RLF_PEAKS_H
#define RLF_PEAKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double fp32_fma_per_s;    /* FP32 fused multiply-adds per second (scalar FFMA) */
    double fp32x2_fma_per_s;  /* FP32 fused multiply-adds per second issued as f32x2 pairs */
    double fp64_fma_per_s;    /* FP64 fused multiply-adds per second */
    double mufu_rsqrt_per_s;  /* rsqrtf per second (multi-function unit) */
    double mufu_sin_per_s;    /* __sinf per second (multi-function unit) */
    int sm_count;
} rlf_peaks;

/* Run the five microbenchmarks on `stream` (cudaStream_t; waits for it).
 * scratch: device buffer of at least SMs * 8 * 256 * 8 bytes (the kernels'
 * results land there).  Returns 0 on success, 1 for null arguments, 2 for a
 * small scratch buffer, 3 for a CUDA error. */
int rlf_peaks_measure(void *scratch, size_t scratch_bytes, void *stream, rlf_peaks *out);

#ifdef __cplusplus
}
#endif

#endif /* RLF_PEAKS_H */
