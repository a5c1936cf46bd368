// tf_chain.cu -- chains of twofold operations on sm_103a: one persistent fused
// launch per batch, and the per-operation step kernels of the baseline.
//
// A chain carries its twofold state s0 + s1 through a sequence of tadd, tmul,
// texp and tlog (the paper's on-the-fly error tracking, "Overview").  Each
// operation is the same device code as the elementwise entry points; only the
// warp votes are off in the fused kernel, whose lanes run different operations.
//
// Layout ("step major", see include/tf.h): chains are numbered longest first,
// so at step t the running chains are 0 .. active(t) - 1 and their operations
// are one contiguous block starting at step_base[t].  A warp that runs
// consecutive chains therefore loads each step's op codes and operands with
// coalesced accesses.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "tf.h"
#include "tf_core.cuh"

namespace {

// One operation on a chain's state; an unknown op code leaves it unchanged.
__device__ __forceinline__ void apply_op(int op, double a0, double a1, double& s0, double& s1) {
    double z0 = s0, z1 = s1;
    switch (op) {
        case TF_OP_ADD: tf::tadd1(s0, s1, a0, a1, z0, z1); break;
        case TF_OP_MUL: tf::tmul1(s0, s1, a0, a1, z0, z1); break;
        case TF_OP_EXP: tf::texp_impl<false, true>(s0, s1, z0, z1); break;
        case TF_OP_LOG: tf::tlog_impl<false>(s0, s1, z0, z1); break;
        default: break;
    }
    s0 = z0;
    s1 = z1;
}

// Chains per warp.  The lanes of a warp run different operations, so each
// step of a warp costs the union of the operations its lanes need: with the
// batched mix (tadd, tmul 30 % each, texp 17.5 %, tlog 22.4 %) about 1.8, 2.9,
// 4.0, 4.6 and 4.7 times one chain's step for 2, 4, 8, 16 and 32 chains.  The
// batch lasts as long as its slowest warp, so the longest chains get the
// fewest lanes.  Tier j gives kTierK[j] chains to a warp and takes the chains
// whose length exceeds max_len / kTierF[j + 1] but not max_len / kTierF[j]
// (kTierF[0] = 1): a chain of length L then finishes within about
// max_len one-chain steps.  group = k > 0 puts k chains in every warp instead.
constexpr int kTiers = 6;
__constant__ int kTierK[kTiers] = {1, 2, 4, 8, 16, 32};
__constant__ float kTierF[kTiers] = {1.78f, 2.87f, 3.97f, 4.58f, 4.7f, 1e30f};

// Number of chains longer than thr (len is non-increasing): a binary search.
__device__ __forceinline__ int64_t count_longer(const int32_t* __restrict__ len, int64_t n, int64_t thr) {
    int64_t lo = 0, hi = n;  // len[i] > thr for i < lo, <= thr for i >= hi
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(len + mid) > thr) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Persistent fused kernel.  Lane 0 of each warp takes the next task from the
// work queue (one atomicAdd, no waiting): a run of up to k consecutive chains
// of one tier, which the warp runs to the end before taking more, until the
// queue is empty.  Chains come longest first, so the long chains start early
// and the short ones fill in behind them.  The tiers partition the chains
// whatever their order; the order only decides how well they balance.
__global__ void chain_fused(const uint8_t* __restrict__ ops, const double* __restrict__ a0,
                            const double* __restrict__ a1, const int64_t* __restrict__ step_base,
                            const int32_t* __restrict__ len, double* s0, double* s1, int64_t n_chains,
                            int32_t max_len, int group, unsigned long long* queue) {
    const int lane = threadIdx.x & 31;
    // tier ends e[j] (chain index) and task counts: lane j < kTiers finds tier j's end
    int64_t e_mine = n_chains;
    if (group <= 0 && lane < kTiers - 1)
        e_mine = count_longer(len, n_chains, (int64_t)((float)max_len / kTierF[lane]));
    int64_t e[kTiers], first[kTiers + 1];
    int kk[kTiers];
    first[0] = 0;
    int64_t b = 0;
#pragma unroll
    for (int j = 0; j < kTiers; ++j) {
        int64_t ej = __shfl_sync(0xffffffffu, e_mine, j);
        ej = (group > 0) ? ((j == kTiers - 1) ? n_chains : 0) : max(ej, b);
        kk[j] = (group > 0) ? group : kTierK[j];
        e[j] = ej;
        first[j + 1] = first[j] + (ej - b + kk[j] - 1) / kk[j];
        b = ej;
    }
    while (true) {
        unsigned long long task = 0;
        if (lane == 0) task = atomicAdd(queue, 1ull);
        task = __shfl_sync(0xffffffffu, task, 0);
        if (task >= (unsigned long long)first[kTiers]) break;
        int64_t start = 0, end = 0;
        int k = 32;
#pragma unroll
        for (int j = 0; j < kTiers; ++j) {
            if ((int64_t)task >= first[j] && (int64_t)task < first[j + 1]) {
                int64_t b0 = (j == 0) ? 0 : e[j - 1];
                k = kk[j];
                start = b0 + ((int64_t)task - first[j]) * k;
                end = e[j];
            }
        }
        int64_t c = start + lane;
        bool in = (lane < k) && (c < end);
        int L = in ? len[c] : 0;
        double x0 = in ? s0[c] : 0.0, x1 = in ? s1[c] : 0.0;
        // software pipeline: the op code and operand of step t + 1 (and the block
        // base of step t + 2) are loaded before step t computes, so that a chain's
        // sequential steps do not wait on memory
        int op = 0;
        double b0 = 0.0, b1 = 0.0;
        int64_t sb1 = 0;
        if (L > 0) {
            int64_t k0 = __ldg(step_base) + c;
            op = __ldg(ops + k0);
            b0 = __ldg(a0 + k0);
            b1 = __ldg(a1 + k0);
            sb1 = (L > 1) ? __ldg(step_base + 1) : 0;
        }
        for (int t = 0; t < L; ++t) {
            int opn = 0;
            double b0n = 0.0, b1n = 0.0;
            int64_t sb2 = 0;
            if (t + 1 < L) {
                int64_t k1 = sb1 + c;
                opn = __ldg(ops + k1);
                b0n = __ldg(a0 + k1);
                b1n = __ldg(a1 + k1);
                sb2 = (t + 2 < L) ? __ldg(step_base + t + 2) : 0;
            }
            apply_op(op, b0, b1, x0, x1);
            op = opn;
            b0 = b0n;
            b1 = b1n;
            sb1 = sb2;
        }
        if (in) {
            s0[c] = x0;
            s1[c] = x1;
        }
    }
}

struct StepAdd {
    static constexpr double dummy = 0.0;
    __device__ static void eval(double x0, double x1, double y0, double y1, double& z0, double& z1) {
        tf::tadd1(x0, x1, y0, y1, z0, z1);
    }
};
struct StepMul {
    static constexpr double dummy = 0.0;
    __device__ static void eval(double x0, double x1, double y0, double y1, double& z0, double& z1) {
        tf::tmul1(x0, x1, y0, y1, z0, z1);
    }
};
struct StepExp {
    static constexpr double dummy = 0.0;
    __device__ static void eval(double x0, double x1, double, double, double& z0, double& z1) {
        tf::texp1(x0, x1, z0, z1);
    }
};
struct StepLog {
    static constexpr double dummy = 1.0;
    __device__ static void eval(double x0, double x1, double, double, double& z0, double& z1) {
        tf::tlog1(x0, x1, z0, z1);
    }
};

// One operation kind over the listed chains.  Every lane of a warp runs the
// operation (lanes past the end on a dummy state, storing nothing) so that the
// warp votes of texp/tlog see full warps.
template <class Op>
__global__ void __launch_bounds__(256) chain_step_kernel(const int32_t* __restrict__ idx, int64_t n,
                                                        int64_t sb, const double* __restrict__ a0,
                                                        const double* __restrict__ a1, double* s0, double* s1) {
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    bool in = i < n;
    int64_t c = in ? idx[i] : 0;
    double x0 = in ? s0[c] : Op::dummy, x1 = in ? s1[c] : 0.0;
    double y0 = in ? a0[sb + c] : 1.0, y1 = in ? a1[sb + c] : 0.0;
    double z0, z1;
    Op::eval(x0, x1, y0, y1, z0, z1);
    if (in) {
        s0[c] = z0;
        s1[c] = z1;
    }
}

int launch_status() {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return TF_OK;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return TF_ERR_NODEVICE;
    return TF_ERR_LAUNCH;
}

inline bool al8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

// Scratch of tf_chain_noalloc: the work-queue counter lives in this array,
// which every device that loads the library holds until the process exits.
// Host code must not pass the symbol itself to a kernel (on the host it only
// stands for the device array); each device's address is looked up once.
constexpr int kNoAllocScratchBytes = TF_CHAIN_NOALLOC_SCRATCH;
static __device__ __align__(256) unsigned char g_chain_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_chain_scratch on the current device, looked up with
// cudaGetSymbolAddress on the first call per device and cached.
int noalloc_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return launch_status() == TF_OK ? TF_ERR_NODEVICE : launch_status();
    if (dev < 0 || dev >= kMaxDevices) return TF_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_chain_scratch) != cudaSuccess || !p) {
            cudaGetLastError();  // do not leave the error for an unrelated later check
            return TF_ERR_LAUNCH;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return TF_OK;
}

}  // namespace

extern "C" {

int tf_chain(const uint8_t* ops, const double* a0, const double* a1, const int64_t* step_base,
             const int32_t* len, double* s0, double* s1, int64_t n_chains, int32_t max_len, void* workspace,
             int threads, int blocks, int group, void* stream) {
    if (n_chains < 0 || max_len < 0 || n_chains > ((int64_t)1 << 40)) return TF_ERR_SIZE;
    if (threads < 32 || threads > 1024 || (threads & 31)) return TF_ERR_ARG;
    if (group < 0 || group > 32) return TF_ERR_ARG;
    if (n_chains == 0 || max_len == 0) return TF_OK;
    if (!ops || !a0 || !a1 || !step_base || !len || !s0 || !s1 || !workspace) return TF_ERR_NULL;
    if (!al8(a0) || !al8(a1) || !al8(step_base) || !al8(s0) || !al8(s1) || !al8(workspace) ||
        (reinterpret_cast<uintptr_t>(len) & 3))
        return TF_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, chain_fused) != cudaSuccess) return launch_status() == TF_OK ? TF_ERR_LAUNCH : launch_status();
    if (threads > fa.maxThreadsPerBlock) return TF_ERR_ARG;  // the kernel's registers do not fit
    if (blocks <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_fused, threads, 0) != cudaSuccess)
            return launch_status() == TF_OK ? TF_ERR_LAUNCH : launch_status();
        blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    // more warps than tasks would idle (a task has at least one chain)
    int64_t need = (n_chains + threads / 32 - 1) / (threads / 32);
    if (blocks > need) blocks = (int)need;
    if (cudaMemsetAsync(workspace, 0, sizeof(unsigned long long), s) != cudaSuccess) return launch_status();
    chain_fused<<<blocks, threads, 0, s>>>(ops, a0, a1, step_base, len, s0, s1, n_chains, max_len, group,
                                           static_cast<unsigned long long*>(workspace));
    return launch_status();
}

int tf_chain_noalloc(const uint8_t* ops, const double* a0, const double* a1, const int64_t* step_base,
                     const int32_t* len, double* s0, double* s1, int64_t n_chains, int32_t max_len, int threads,
                     int blocks, int group, void* stream) {
    if (n_chains < 0 || max_len < 0 || n_chains > TF_CHAIN_NOALLOC_MAX_CHAINS) return TF_ERR_SIZE;
    if (threads < 32 || threads > 1024 || (threads & 31)) return TF_ERR_ARG;
    if (group < 0 || group > 32) return TF_ERR_ARG;
    if (n_chains == 0 || max_len == 0) return TF_OK;
    void* scratch = nullptr;
    int rc = noalloc_scratch(&scratch);
    if (rc != TF_OK) return rc;
    // the same launch as tf_chain with the static scratch as its workspace (tf_chain
    // clears the queue counter on `stream` before launching)
    return tf_chain(ops, a0, a1, step_base, len, s0, s1, n_chains, max_len, scratch, threads, blocks, group,
                    stream);
}

int tf_chain_step(int op, const int32_t* idx, int64_t n_idx, int64_t step_base_t, const double* a0,
                  const double* a1, double* s0, double* s1, void* stream) {
    if (op < TF_OP_ADD || op > TF_OP_LOG) return TF_ERR_ARG;
    if (n_idx < 0 || n_idx > ((int64_t)1 << 40) || step_base_t < 0) return TF_ERR_SIZE;
    if (n_idx == 0) return TF_OK;
    if (!idx || !a0 || !a1 || !s0 || !s1) return TF_ERR_NULL;
    if (!al8(a0) || !al8(a1) || !al8(s0) || !al8(s1) || (reinterpret_cast<uintptr_t>(idx) & 3)) return TF_ERR_ALIGN;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned grid = (unsigned)((n_idx + 255) / 256);
    switch (op) {
        case TF_OP_ADD: chain_step_kernel<StepAdd><<<grid, 256, 0, s>>>(idx, n_idx, step_base_t, a0, a1, s0, s1); break;
        case TF_OP_MUL: chain_step_kernel<StepMul><<<grid, 256, 0, s>>>(idx, n_idx, step_base_t, a0, a1, s0, s1); break;
        case TF_OP_EXP: chain_step_kernel<StepExp><<<grid, 256, 0, s>>>(idx, n_idx, step_base_t, a0, a1, s0, s1); break;
        default: chain_step_kernel<StepLog><<<grid, 256, 0, s>>>(idx, n_idx, step_base_t, a0, a1, s0, s1); break;
    }
    return launch_status();
}

}  // extern "C"
