// tf_probe.cu -- FP64 pipe calibration kernel for the benchmark (include/tf_probe.h).
#include <cuda_runtime.h>

#include "tf_probe.h"

namespace {

__global__ void dfma_chains(double* out, int iters) {
    // Eight independent chains a <- a * m + c with m slightly below 1 and a small
    // c: the values stay bounded, so no special operands slow the pipe.
    const double m = 0.99999999999;
    const double c = 1e-12 * (threadIdx.x + 1);
    double a0 = 1.0, a1 = 1.1, a2 = 1.2, a3 = 1.3, a4 = 1.4, a5 = 1.5, a6 = 1.6, a7 = 1.7;
    for (int i = 0; i < iters; ++i) {
        a0 = __fma_rn(a0, m, c);
        a1 = __fma_rn(a1, m, c);
        a2 = __fma_rn(a2, m, c);
        a3 = __fma_rn(a3, m, c);
        a4 = __fma_rn(a4, m, c);
        a5 = __fma_rn(a5, m, c);
        a6 = __fma_rn(a6, m, c);
        a7 = __fma_rn(a7, m, c);
    }
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

}  // namespace

extern "C" int tfp_dfma(double* out, int blocks, int threads, int iters, void* stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return 6;
    dfma_chains<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
