/*
 * tf_probe.h -- calibration kernels of the benchmark (libtfprobe.so).
 *
 * Not part of the twofold method: the paper has no counterpart.  The twofold
 * kernels of libtf.so are bound by the FP64 pipe and the integer ALU pipe, and
 * no measured peak exists for either on this GPU, so the benchmark
 * measures both with these kernels and uses them as the denominators of its
 * roofline fractions.
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

/* Enqueue an integer throughput kernel on `stream`: `blocks` x `threads`
 * threads, each running 8 independent chains for `iters` iterations, 16
 * instructions per iteration and thread, nothing else inside the loop.
 * mode 0: a 32-bit funnel-shift rotate and a dependent three-input xor per
 * chain (instructions only the integer ALU pipe executes: its peak); mode 1: a
 * 32-bit add and a dependent three-input xor (the adds may issue on the
 * multiply-add pipe: the two integer pipes together).  `out` is a device
 * array of blocks * threads unsigned ints owned by the caller (one result per
 * thread, so the work cannot be removed).  Returns as tfp_dfma (6 also for an
 * unknown mode). */
int tfp_alu(unsigned* out, int blocks, int threads, int iters, int mode, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TF_PROBE_H */
