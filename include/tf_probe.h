/*
 * tf_probe.h -- calibration kernel of the benchmark (libtfprobe.so).
 *
 * Not part of the twofold method: the paper has no counterpart.  The twofold
 * kernels of libtf.so are bound by the FP64 pipe, and no measured FP64
 * peak exists for this GPU, so the benchmark measures one with this kernel and
 * uses it as the denominator of its roofline fraction.
 */
#ifndef TF_PROBE_H
#define TF_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Enqueue a DFMA throughput kernel on `stream`: `blocks` x `threads` threads,
 * each running 8 independent fused multiply-add chains for `iters` iterations
 * (8 * iters DFMA per thread, nothing else inside the loop).  `out` is a device
 * array of blocks * threads doubles owned by the caller; each thread stores its
 * chain sum there so the work cannot be removed.  Returns 0, 4 when the launch
 * is rejected, 6 for a bad argument (NULL out, non-positive sizes, threads > 1024). */
int tfp_dfma(double* out, int blocks, int threads, int iters, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TF_PROBE_H */
