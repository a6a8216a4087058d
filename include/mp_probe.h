/*
 * mp_probe.h -- measurement helpers of the benchmark (no counterpart in the
 * paper). They are not part of the filter's boundary and live in their own
 * library, libmp_probe.so, built beside libmp.so: ceilings that the rooflines
 * of the filter's kernels are read against, measured on the GPU at hand.
 *
 * Pointers are DEVICE pointers of the current device (host memory and other
 * devices' memory are refused with MP_EINVAL before anything is launched).
 * Work is enqueued on cuda_stream (NULL = legacy default stream); every call
 * synchronises on its own events and returns the mean time of one run. Return
 * codes are those of megaparticles.h; nothing is printed.
 */
#ifndef MP_PROBE_H
#define MP_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Independent, uniformly random 4-byte reads over a device buffer of n_words
 * uint32 (contents arbitrary, left unchanged; each read fetches one 32-byte
 * sector from DRAM when the buffer is much larger than L2): the rate at which
 * this GPU serves random sectors, the ceiling of a gather-bound kernel such as
 * the likelihood's nearest-neighbour-field lookups while particles are spread.
 * blocks CTAs of 256 threads; each thread keeps 16 linear congruential
 * sequences and issues their 16 reads before it uses any of them, so that
 * enough reads are in flight to cover the DRAM latency; reads_per_thread is
 * rounded up to a multiple of 16. Runs once to warm up, then `repeats` times
 * timed with CUDA events; *ms_out = mean ms per run, *reads_out (may be NULL)
 * = reads per run. Errors: MP_EINVAL (NULL or non-device pointer, sizes < 1,
 * n_words > 2^32), MP_ECUDA. */
int mp_probe_random_reads(const uint32_t* words, int64_t n_words, int blocks, int reads_per_thread, int repeats,
                          void* cuda_stream, float* ms_out, int64_t* reads_out);

/* Fused multiply-add throughput: blocks CTAs of 256 threads, each thread
 * `iters` rounds of 16 independent dependent-chain FMAs. kind 0: FP32
 * (fmaf); kind 1: FP32 in packed pairs (one f32x2 fma = two FMAs); kind 2:
 * FP64 (fma). *ms_out = mean ms of one run over `repeats` timed runs after a
 * warm-up; *flops_out = flops of one run (2 per FMA). Errors: MP_EINVAL
 * (unknown kind, sizes < 1), MP_ECUDA. */
int mp_probe_fma_rate(int kind, int blocks, int iters, int repeats, void* cuda_stream, float* ms_out,
                      double* flops_out);

#ifdef __cplusplus
}
#endif
#endif /* MP_PROBE_H */
