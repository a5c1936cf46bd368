// tf_capi.cu -- elementwise twofold kernels for sm_103a and the C ABI of include/tf.h.
//
// One thread evaluates two consecutive elements (two independent chains of
// FP64 work for the scheduler; texp and tlog take both in one straight-line
// call, OpPair) and moves them with 128-bit loads and stores when every pointer
// is 16-byte aligned (four elements per thread for float twofolds).  All 32
// lanes of a warp always run the element code -- lanes past the end work on a
// harmless dummy argument and store nothing -- so that the warp-uniform votes
// (__any_sync) that guard the rare special-case paths see a full warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "tf.h"
#include "tf_core.cuh"
#include "tf_core_f.cuh"

namespace {

constexpr int kThreads = 256;

struct OpExp {
    static constexpr int threads = 128;   // 56 registers: 36 warps per SM (4.6 % faster than at 64)
    static constexpr int min_blocks = 9;
    static constexpr double dummy = 0.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::texp1(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::texp_pair(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
struct OpExpm1 {
    static constexpr int threads = 128;   // 72 registers, no spills: 28 warps per SM (at 64 it
    static constexpr int min_blocks = 7;  // spilled 16 bytes and ran the 2^24 hard cases 2.4 % slower)
    static constexpr double dummy = 0.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::texpm11(a, b, z0, z1); }
};
struct OpLog {
    static constexpr int threads = 128;   // 72 registers, no spills: 28 warps per SM (1.2 % faster
    static constexpr int min_blocks = 7;  // than at 64 with 20 bytes of spills)
    static constexpr double dummy = 1.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog1(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::tlog_pair(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
struct OpLog1p {
    static constexpr int threads = 128;   // 72 registers: 28 warps per SM
    static constexpr int min_blocks = 7;
    static constexpr double dummy = 0.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog1p1(a, b, z0, z1); }
};
// Coupled results (pexp, pexpm1, plog, plog1p) and twofold results of coupled
// arguments (texpp, texpm1p, tlogp, tlog1pp).
struct OpPExp {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;  // as OpExp
    static constexpr int min_blocks = 9;
    __device__ static void eval(double a, double b, double& z0, double& z1) {
        tf::texp_impl<true>(a, b, z0, z1);
        tf::couple(z0, z1);
    }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::texp_pair(a0, b0, a1, b1, r0, r1, s0, s1);
        tf::couple(r0, r1);
        tf::couple(s0, s1);
    }
};
struct OpPExpm1 {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;  // as OpExpm1
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) {
        tf::texpm1_impl<true>(a, b, z0, z1);
        tf::couple(z0, z1);
    }
};
struct OpPLog {
    static constexpr double dummy = 1.0;
    static constexpr int threads = 128;  // as OpLog
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) {
        tf::tlog_impl<true>(a, b, z0, z1);
        tf::couple(z0, z1);
    }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::tlog_pair(a0, b0, a1, b1, r0, r1, s0, s1);
        tf::couple(r0, r1);
        tf::couple(s0, s1);
    }
};
struct OpPLog1p {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) {
        tf::tlog1p1(a, b, z0, z1);
        tf::couple(z0, z1);
    }
};
struct OpExpP {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;  // as OpExp
    static constexpr int min_blocks = 9;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::texp_impl<true, false>(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::texp_pair<false>(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
struct OpExpm1P {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;  // as OpExpm1
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::texpm1_impl<true, false>(a, b, z0, z1); }
};
struct OpLogP {
    static constexpr double dummy = 1.0;
    static constexpr int threads = 128;  // as OpLog
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog_impl<true, false>(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::tlog_pair<false>(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
struct OpLog1pP {
    static constexpr double dummy = 0.0;
    static constexpr int threads = 128;
    static constexpr int min_blocks = 7;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog1p_impl<false>(a, b, z0, z1); }
};
struct OpExpTables {
    static constexpr double dummy = 0.0;
    static constexpr int min_blocks = 4;  // 64 registers (at 56 it spilled and ran 2.5 % slower)
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::texp_impl<true, true, true>(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::texp_pair<true, true>(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
// The logarithms with the Newton step in binary64 (A/B variants of OpLog, OpLog1p).
struct OpLogN64 {
    static constexpr int threads = 128;  // as OpLog
    static constexpr int min_blocks = 7;
    static constexpr double dummy = 1.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog_impl<true, true, true>(a, b, z0, z1); }
    __device__ static void eval2(double a0, double b0, double a1, double b1, double& r0, double& r1, double& s0,
                                 double& s1) {
        tf::tlog_pair<true, true>(a0, b0, a1, b1, r0, r1, s0, s1);
    }
};
struct OpLog1pN64 {
    static constexpr int threads = 128;
    static constexpr int min_blocks = 7;
    static constexpr double dummy = 0.0;
    __device__ static void eval(double a, double b, double& z0, double& z1) { tf::tlog1p_impl<true, true>(a, b, z0, z1); }
};
struct OpAdd {
    __device__ static void eval(double a, double b, double c, double d, double& z0, double& z1) {
        tf::tadd1(a, b, c, d, z0, z1);
    }
};
struct OpMul {
    __device__ static void eval(double a, double b, double c, double d, double& z0, double& z1) {
        tf::tmul1(a, b, c, d, z0, z1);
    }
};

struct OpExpF {
    static constexpr int min_blocks = 8;  // 32 registers: 64 warps per SM
    static constexpr float dummy = 0.0f;
    __device__ static void eval(float a, float b, float& z0, float& z1) { tff::texpf_impl<true>(a, b, z0, z1); }
    __device__ static void eval4(const float (&a)[4], const float (&b)[4], float (&r)[4], float (&s)[4]) {
        tff::texpf_multi<2>(a, b, r, s);
        tff::texpf_multi<2>(a + 2, b + 2, r + 2, s + 2);
    }
};
struct OpExpm1F {
    static constexpr int min_blocks = 8;  // 32 registers: 64 warps per SM
    static constexpr float dummy = 0.0f;
    __device__ static void eval(float a, float b, float& z0, float& z1) { tff::texpm1f_impl<true>(a, b, z0, z1); }
};
struct OpLogF {
    static constexpr int min_blocks = 6;  // 40 registers: 48 warps per SM
    static constexpr float dummy = 1.0f;
    __device__ static void eval(float a, float b, float& z0, float& z1) { tff::tlogf_impl<true>(a, b, z0, z1); }
    __device__ static void eval4(const float (&a)[4], const float (&b)[4], float (&r)[4], float (&s)[4]) {
        tff::tlogf_quad(a, b, r, s);
    }
};
struct OpLog1pF {
    static constexpr int min_blocks = 6;  // 40 registers: 48 warps per SM
    static constexpr float dummy = 0.0f;
    __device__ static void eval(float a, float b, float& z0, float& z1) { tff::tlog1pf_impl<true>(a, b, z0, z1); }
};

// Inputs are read with ordinary (coherent) loads: the ABI lets z0 be x0 and z1
// be x1, so an input array may be written during the launch, which rules out
// the read-only (non-coherent) path and __restrict__ on the inputs.  Each
// thread reads its elements before it writes them.
__device__ __forceinline__ double2 ld2(const double* p) { return *reinterpret_cast<const double2*>(p); }
__device__ __forceinline__ void st2(double* p, double a, double b) {
    __stcs(reinterpret_cast<double2*>(p), make_double2(a, b));  // streaming: outputs are not re-read
}

// Block size of an op's vector kernel: Op::threads where the op sets it, else
// kThreads.  With min_blocks it sets the register budget: 256 x 4 blocks gives
// 64 registers (32 warps per SM); 128 x 9 gives 56 (36 warps: texp); 128 x 7
// gives 72 (28 warps), which tlog, tlog1p's two-table log and texpm1 need to
// run without spills.
template <class Op, class = void>
struct OpThreads {
    static constexpr int value = kThreads;
};
template <class Op>
struct OpThreads<Op, decltype((void)Op::threads)> {
    static constexpr int value = Op::threads;
};

// Whether an op evaluates the two elements of a thread in one call (Op::eval2:
// both main paths in straight-line code, so that their independent
// instruction streams interleave; measured 11 % faster for tlog and 1.3 % for
// texp at 64 registers, 6 % and 3 % slower at 78 registers and 24 warps).
// Whether a float op evaluates the four elements of a thread in one call
// (Op::eval4, as OpPair for the double ops).
template <class Op, class = void>
struct OpQuad {
    static constexpr bool value = false;
};
template <class Op>
struct OpQuad<Op, decltype((void)&Op::eval4)> {
    static constexpr bool value = true;
};

template <class Op, class = void>
struct OpPair {
    static constexpr bool value = false;
};
template <class Op>
struct OpPair<Op, decltype((void)&Op::eval2)> {
    static constexpr bool value = true;
};

// Unary, 2 elements per thread, 128-bit I/O.  Thread t covers elements 2t, 2t+1.
template <class Op>
__global__ void __launch_bounds__(OpThreads<Op>::value, Op::min_blocks) unary_v2(const double* x0, const double* x1,
                                                                                     double* z0, double* z1, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * OpThreads<Op>::value + threadIdx.x;
    int64_t i = 2 * t;
    double a0 = Op::dummy, a1 = Op::dummy, b0 = 0.0, b1 = 0.0;
    bool full = i + 1 < n;
    bool half = i + 1 == n;
    if (full) {
        double2 a = ld2(x0 + i);
        a0 = a.x;
        a1 = a.y;
        if (x1) {
            double2 b = ld2(x1 + i);
            b0 = b.x;
            b1 = b.y;
        }
    } else if (half) {
        a0 = x0[i];
        b0 = x1 ? x1[i] : 0.0;
    }
    double r0, r1, s0, s1;
    if constexpr (OpPair<Op>::value) {
        Op::eval2(a0, b0, a1, b1, r0, r1, s0, s1);
    } else {
        Op::eval(a0, b0, r0, r1);
        Op::eval(a1, b1, s0, s1);
    }
    if (full) {
        st2(z0 + i, r0, s0);
        st2(z1 + i, r1, s1);
    } else if (half) {
        z0[i] = r0;
        z1[i] = r1;
    }
}

// Unary, 1 element per thread, scalar I/O (pointers not 16-byte aligned).
template <class Op>
__global__ void __launch_bounds__(kThreads) unary_v1(const double* x0, const double* x1, double* z0, double* z1,
                                                     int64_t n) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    bool in = i < n;
    double a = in ? x0[i] : Op::dummy;
    double b = (in && x1) ? x1[i] : 0.0;
    double r0, r1;
    Op::eval(a, b, r0, r1);
    if (in) {
        z0[i] = r0;
        z1[i] = r1;
    }
}

// Float twofolds: 4 elements per thread, 128-bit loads and stores.  Op::min_blocks
// sets the register budget: texpf and texpm1f at 8 blocks of 256 (32 registers)
// measured 3 % and 1.4 % faster than at 6 (40 registers); the logarithms spill
// below 40.
template <class Op>
__global__ void __launch_bounds__(kThreads, Op::min_blocks)
    unary_f4(const float* x0, const float* x1, float* z0, float* z1, int64_t n) {
    int64_t i = 4 * ((int64_t)blockIdx.x * kThreads + threadIdx.x);
    float a[4], b[4], r[4], s[4];
    bool full = i + 3 < n;
    if (full) {
        float4 v = *reinterpret_cast<const float4*>(x0 + i);
        a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w;
        float4 w = x1 ? *reinterpret_cast<const float4*>(x1 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        b[0] = w.x, b[1] = w.y, b[2] = w.z, b[3] = w.w;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            bool in = i + q < n;
            a[q] = in ? x0[i + q] : Op::dummy;
            b[q] = (in && x1) ? x1[i + q] : 0.0f;
        }
    }
    if constexpr (OpQuad<Op>::value) {
        Op::eval4(a, b, r, s);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) Op::eval(a[q], b[q], r[q], s[q]);
    }
    if (full) {
        __stcs(reinterpret_cast<float4*>(z0 + i), make_float4(r[0], r[1], r[2], r[3]));
        __stcs(reinterpret_cast<float4*>(z1 + i), make_float4(s[0], s[1], s[2], s[3]));
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i + q < n) {
                z0[i + q] = r[q];
                z1[i + q] = s[q];
            }
        }
    }
}

// Float twofolds, 1 element per thread, scalar I/O (pointers not 16-byte aligned).
template <class Op>
__global__ void __launch_bounds__(kThreads) unary_f1(const float* x0, const float* x1, float* z0, float* z1,
                                                     int64_t n) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    bool in = i < n;
    float a = in ? x0[i] : Op::dummy;
    float b = (in && x1) ? x1[i] : 0.0f;
    float r0, r1;
    Op::eval(a, b, r0, r1);
    if (in) {
        z0[i] = r0;
        z1[i] = r1;
    }
}

template <class Op>
__global__ void __launch_bounds__(kThreads) binary_v2(const double* x0, const double* x1, const double* y0,
                                                      const double* y1, double* z0, double* z1, int64_t n) {
    int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    int64_t i = 2 * t;
    if (i + 1 < n) {
        double2 a = ld2(x0 + i), c = ld2(y0 + i);
        double2 b = x1 ? ld2(x1 + i) : make_double2(0.0, 0.0);
        double2 d = y1 ? ld2(y1 + i) : make_double2(0.0, 0.0);
        double r0, r1, s0, s1;
        Op::eval(a.x, b.x, c.x, d.x, r0, r1);
        Op::eval(a.y, b.y, c.y, d.y, s0, s1);
        st2(z0 + i, r0, s0);
        st2(z1 + i, r1, s1);
    } else if (i < n) {
        double r0, r1;
        Op::eval(x0[i], x1 ? x1[i] : 0.0, y0[i], y1 ? y1[i] : 0.0, r0, r1);
        z0[i] = r0;
        z1[i] = r1;
    }
}

template <class Op>
__global__ void __launch_bounds__(kThreads) binary_v1(const double* x0, const double* x1, const double* y0,
                                                      const double* y1, double* z0, double* z1, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (i < n) {
        double r0, r1;
        Op::eval(x0[i], x1 ? x1[i] : 0.0, y0[i], y1 ? y1[i] : 0.0, r0, r1);
        z0[i] = r0;
        z1[i] = r1;
    }
}

inline bool al(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

// Largest n accepted (1 TiB per array): grids stay below 2^31 - 1 blocks.
constexpr int64_t kMaxN = (int64_t)1 << 37;

int launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return TF_OK;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return TF_ERR_NODEVICE;
    return TF_ERR_LAUNCH;
}

template <class Op>
int run_unary(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    if (n < 0 || n > kMaxN) return TF_ERR_SIZE;
    if (n == 0) return TF_OK;
    if (!x0 || !z0 || !z1) return TF_ERR_NULL;
    if (!al(x0, 8) || !al(z0, 8) || !al(z1, 8) || (x1 && !al(x1, 8))) return TF_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool vec = al(x0, 16) && al(z0, 16) && al(z1, 16) && (!x1 || al(x1, 16));
    if (vec) {
        constexpr int T = OpThreads<Op>::value;
        int64_t threads = (n + 1) / 2;
        unsigned blocks = (unsigned)((threads + T - 1) / T);
        unary_v2<Op><<<blocks, T, 0, s>>>(x0, x1, z0, z1, n);
    } else {
        unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
        unary_v1<Op><<<blocks, kThreads, 0, s>>>(x0, x1, z0, z1, n);
    }
    return launch_status();
}

template <class Op>
int run_unary_f(const float* x0, const float* x1, float* z0, float* z1, int64_t n, void* stream) {
    if (n < 0 || n > kMaxN) return TF_ERR_SIZE;
    if (n == 0) return TF_OK;
    if (!x0 || !z0 || !z1) return TF_ERR_NULL;
    if (!al(x0, 4) || !al(z0, 4) || !al(z1, 4) || (x1 && !al(x1, 4))) return TF_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool vec = al(x0, 16) && al(z0, 16) && al(z1, 16) && (!x1 || al(x1, 16));
    if (vec) {
        int64_t threads = (n + 3) / 4;
        unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
        unary_f4<Op><<<blocks, kThreads, 0, s>>>(x0, x1, z0, z1, n);
    } else {
        unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
        unary_f1<Op><<<blocks, kThreads, 0, s>>>(x0, x1, z0, z1, n);
    }
    return launch_status();
}

template <class Op>
int run_binary(const double* x0, const double* x1, const double* y0, const double* y1, double* z0, double* z1,
               int64_t n, void* stream) {
    if (n < 0 || n > kMaxN) return TF_ERR_SIZE;
    if (n == 0) return TF_OK;
    if (!x0 || !y0 || !z0 || !z1) return TF_ERR_NULL;
    if (!al(x0, 8) || !al(y0, 8) || !al(z0, 8) || !al(z1, 8) || (x1 && !al(x1, 8)) || (y1 && !al(y1, 8)))
        return TF_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool vec = al(x0, 16) && al(y0, 16) && al(z0, 16) && al(z1, 16) && (!x1 || al(x1, 16)) && (!y1 || al(y1, 16));
    if (vec) {
        int64_t threads = (n + 1) / 2;
        unsigned blocks = (unsigned)((threads + kThreads - 1) / kThreads);
        binary_v2<Op><<<blocks, kThreads, 0, s>>>(x0, x1, y0, y1, z0, z1, n);
    } else {
        unsigned blocks = (unsigned)((n + kThreads - 1) / kThreads);
        binary_v1<Op><<<blocks, kThreads, 0, s>>>(x0, x1, y0, y1, z0, z1, n);
    }
    return launch_status();
}

}  // namespace

extern "C" {

int tf_texp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpExp>(x0, x1, z0, z1, n, stream);
}
int tf_texpm1(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpExpm1>(x0, x1, z0, z1, n, stream);
}
int tf_tlog(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLog>(y0, y1, z0, z1, n, stream);
}
int tf_tlog1p(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLog1p>(y0, y1, z0, z1, n, stream);
}
int tf_pexp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpPExp>(x0, x1, z0, z1, n, stream);
}
int tf_pexpm1(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpPExpm1>(x0, x1, z0, z1, n, stream);
}
int tf_plog(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpPLog>(y0, y1, z0, z1, n, stream);
}
int tf_plog1p(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpPLog1p>(y0, y1, z0, z1, n, stream);
}
int tf_texpp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpExpP>(x0, x1, z0, z1, n, stream);
}
int tf_texpm1p(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpExpm1P>(x0, x1, z0, z1, n, stream);
}
int tf_tlogp(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLogP>(y0, y1, z0, z1, n, stream);
}
int tf_tlog1pp(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLog1pP>(y0, y1, z0, z1, n, stream);
}
int tf_texp_tables(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpExpTables>(x0, x1, z0, z1, n, stream);
}
int tf_tlog_newton_fp64(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLogN64>(y0, y1, z0, z1, n, stream);
}
int tf_tlog1p_newton_fp64(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream) {
    return run_unary<OpLog1pN64>(y0, y1, z0, z1, n, stream);
}
int tf_tadd(const double* x0, const double* x1, const double* y0, const double* y1, double* z0, double* z1,
            int64_t n, void* stream) {
    return run_binary<OpAdd>(x0, x1, y0, y1, z0, z1, n, stream);
}
int tf_tmul(const double* x0, const double* x1, const double* y0, const double* y1, double* z0, double* z1,
            int64_t n, void* stream) {
    return run_binary<OpMul>(x0, x1, y0, y1, z0, z1, n, stream);
}

int tf_texpf(const float* x0, const float* x1, float* z0, float* z1, int64_t n, void* stream) {
    return run_unary_f<OpExpF>(x0, x1, z0, z1, n, stream);
}
int tf_texpm1f(const float* x0, const float* x1, float* z0, float* z1, int64_t n, void* stream) {
    return run_unary_f<OpExpm1F>(x0, x1, z0, z1, n, stream);
}
int tf_tlogf(const float* y0, const float* y1, float* z0, float* z1, int64_t n, void* stream) {
    return run_unary_f<OpLogF>(y0, y1, z0, z1, n, stream);
}
int tf_tlog1pf(const float* y0, const float* y1, float* z0, float* z1, int64_t n, void* stream) {
    return run_unary_f<OpLog1pF>(y0, y1, z0, z1, n, stream);
}

const char* tf_strerror(int code) {
    switch (code) {
        case TF_OK: return "ok";
        case TF_ERR_NULL: return "a required pointer is NULL";
        case TF_ERR_SIZE: return "n is negative or too large";
        case TF_ERR_ALIGN: return "a pointer is not aligned to its element size";
        case TF_ERR_LAUNCH: return "kernel launch failed";
        case TF_ERR_NODEVICE: return "no usable CUDA device";
        case TF_ERR_ARG: return "invalid argument";
        default: return "unknown error code";
    }
}

int tf_version(void) { return (1 << 16) | 0; }

}  // extern "C"
