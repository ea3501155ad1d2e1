/*
 * frbx_peaks.h -- peak-rate probes of the GPU (libfrbx_peaks), used as roofline denominators
 * by the bench.  The paper has no counterpart: these measure the hardware, not the method.
 */
#ifndef FRBX_PEAKS_H
#define FRBX_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Runs one rate probe on every SM of the current device, on `stream` (NULL = legacy default
 * stream), after a short warm-up launch, and times it with CUDA events.
 *  kind   0 = FP32 FMA pipe, scalar fma.rn.f32 (64 warps per SM, 16 independent chains each);
 *         1 = FP32 FMA pipe, packed fma.rn.f32x2 (two FMAs per instruction);
 *         2 = tensor pipe, dense BF16 tcgen05.mma kind::f16, M 128 x N 256 x K 16 per
 *             instruction, FP32 accumulation in tensor memory, one CTA per SM;
 *         3 = the same with E4M3 operands, tcgen05.mma kind::f8f6f4, K 32 per instruction.
 *  iters  inner iterations (FMA probes: FMAs per chain; MMA probes: groups of 4 MMAs).
 *  tflops out: dense TFLOP/s, 2 flop per multiply-add;  ms  out: elapsed device time.
 * Returns 0, -1 (bad argument), -2 (allocation failed), -3 (CUDA error) or -5 (the bounded
 * wait for the MMAs' completion gave up).
 */
int frbx_peak_probe(int32_t kind, int32_t iters, double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FRBX_PEAKS_H */
