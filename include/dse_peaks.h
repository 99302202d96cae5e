/* dse_peaks.h -- arithmetic-rate microbenchmark of the GPU that runs the solver.
 *
 * The paper has no counterpart: this measures the denominators of the
 * arithmetic roofline that the solver's kernels are reported against (they are
 * bound by the FP64 and FP32 arithmetic pipes, not by memory).  Part of the same
 * shared library as dse.h.
 */
#ifndef DSE_PEAKS_H
#define DSE_PEAKS_H

#ifdef __cplusplus
extern "C" {
#endif

/* Pipes that dse_alu_peak can measure. */
enum {
    DSE_PEAK_FP64_FMA = 0, /* FP64 fused multiply-add (2 flops each) */
    DSE_PEAK_FP32_FMA = 1, /* FP32 fused multiply-add (2 flops each) */
    DSE_PEAK_MUFU_EX2 = 2, /* FP32 base-2 exponential on the special-function unit */
    DSE_PEAK_MUFU_LG2 = 3, /* FP32 base-2 logarithm on the special-function unit */
    DSE_PEAK_FP64_DMMA = 4, /* FP64 tensor-core multiply-add (mma.sync m8n8k4): one 8x8x4
                               warp product counts as 256 FMAs, 8 per thread */
    DSE_PEAK_FP32X2_FMA = 5 /* FP32 fused multiply-add on float pairs (the paired f32x2
                               instruction): each instruction counts as 2 FMAs */
};

/* Rate of one arithmetic pipe on the current device, in operations per second
 * (thread-level: one FMA or one exp2 of one thread is one operation; for
 * DSE_PEAK_FP64_DMMA the FMAs of the warp's matrix products divided among its
 * threads, so that the rate compares with DSE_PEAK_FP64_FMA's; for
 * DSE_PEAK_FP32X2_FMA both lanes of a paired instruction, so that the rate
 * compares with DSE_PEAK_FP32_FMA's).
 *
 * kind:      one of the DSE_PEAK_* values.
 * target_ms: approximate duration of the timed launch in milliseconds (1 .. 5000);
 *            a short calibration launch sizes it.
 * stream:    cudaStream_t to run on (NULL: the legacy default stream).
 * ops_per_s: host pointer, out: operations per second of the timed launch.
 * ms:        host pointer (nullable), out: duration of the timed launch.
 *
 * Each thread of a grid of (SM count x resident blocks per SM) blocks runs eight
 * independent dependency chains of the operation; timing is by CUDA events on
 * `stream`, and the call synchronises the stream.  Allocates nothing.
 * Returns DSE_OK, DSE_ERR_ARG (unknown kind, target_ms out of range, null
 * ops_per_s) or DSE_ERR_CUDA. */
int dse_alu_peak(int kind, double target_ms, void* stream, double* ops_per_s, double* ms);

#ifdef __cplusplus
}
#endif

#endif /* DSE_PEAKS_H */
