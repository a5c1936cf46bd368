// tf_probe.cu -- FP64 pipe calibration kernel for the benchmark (include/tf_probe.h).
#include <cuda_runtime.h>

#include "tf_probe.h"

namespace {

// Eight independent chains a <- a * m + c per thread.  m slightly below 1 and a
// small c keep the values bounded, so no special operands slow the pipe.  m and
// c arrive as kernel arguments: with a literal multiplier and a per-thread
// addend the same loop ran at only about 1.7 DFMA per clock per SM on GB300,
// against 2 with both operands uniform.
__global__ void dfma_chains(double* out, int iters, double m, double c) {
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 1.0 + 0.1 * k + 1e-9 * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __fma_rn(a[k], m, c);
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] =
        ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
}

}  // namespace

extern "C" int tfp_dfma(double* out, int blocks, int threads, int iters, void* stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return 6;
    dfma_chains<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.99999999999, 1e-12);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
