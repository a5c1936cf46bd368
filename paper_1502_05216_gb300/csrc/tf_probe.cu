// tf_probe.cu -- FP64 and integer-ALU pipe calibration kernels for the benchmark
// (include/tf_probe.h).
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

// Integer-ALU throughput.  Eight independent chains per thread; every
// iteration applies to each chain one instruction of two kinds in turn, the
// second depending on the first, with c and d kernel arguments:
//   mode 0: a <- rotate-left(a, 7) (funnel shift), then a <- a ^ b ^ c (lop3);
//   mode 1: b <- b + a, then a <- a ^ b ^ d (lop3).
// Two logic operations in a row on the same inputs could merge into one lop3,
// and two adds in a row into one three-input add; alternating two kinds keeps
// every instruction.  16 instructions per iteration and thread.  Mode 0 uses
// instruction kinds that only the integer ALU pipe executes; the compiler may
// issue mode 1's adds on the multiply-add pipe (IMAD), so mode 1 measures the
// two integer pipes together.
__global__ void alu_chains(unsigned* out, int iters, int mode, unsigned c, unsigned d) {
    unsigned a[8], b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        a[k] = threadIdx.x * 2654435761u + 97u * k;
        b[k] = blockIdx.x * 40503u + 13u * k;
    }
    if (mode == 0) {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                asm volatile("shf.l.wrap.b32 %0, %0, %0, 7;" : "+r"(a[k]));
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(b[k]), "r"(c));
            }
        }
    } else {
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                asm volatile("add.u32 %0, %0, %1;" : "+r"(b[k]) : "r"(a[k]));
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(a[k]) : "r"(b[k]), "r"(d));
            }
        }
    }
    unsigned r = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) r ^= a[k] + b[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace

extern "C" int tfp_alu(unsigned* out, int blocks, int threads, int iters, int mode, void* stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0 || mode < 0 || mode > 1) return 6;
    alu_chains<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, mode, 0x9e3779b9u,
                                                                         0x7f4a7c15u);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

extern "C" int tfp_dfma(double* out, int blocks, int threads, int iters, void* stream) {
    if (!out || blocks <= 0 || threads <= 0 || threads > 1024 || iters <= 0) return 6;
    dfma_chains<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.99999999999, 1e-12);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}
