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

// A cheap operation on a chain's state: tadd, tmul, or an unknown op code,
// which leaves it unchanged.
__device__ __forceinline__ void apply_cheap(int op, double a0, double a1, double& s0, double& s1) {
    double z0 = s0, z1 = s1;
    if (op == TF_OP_ADD) tf::tadd1(s0, s1, a0, a1, z0, z1);
    else if (op == TF_OP_MUL) tf::tmul1(s0, s1, a0, a1, z0, z1);
    s0 = z0;
    s1 = z1;
}

// Scheduling inside a warp.  The lanes of a warp run different chains, so a
// warp that ran every lane's next operation at once would pay, at each step,
// for every operation kind its lanes need (with the batched mix, texp and tlog
// both in most steps of a full warp).  A warp of several chains instead
// alternates two phases:
//  * cheap: every lane whose next operation is tadd, tmul (or an unknown code)
//    runs it, again until no lane has a cheap one next;
//  * costly: of texp and tlog, the warp runs the one whose waiting lanes hold
//    more remaining steps per unit cost (kCostExp : kCostLog, the ratio of
//    their instruction counts), for the lanes waiting on it; the other kind
//    waits a phase.
// Every lane still runs its own chain's operations in order, so the results
// are those of any other schedule; the choice only balances the lanes (the
// lanes with the most work left decide).  A warp of one chain runs its steps
// one after the other, without the phases' votes.
constexpr int kCostExp = 7, kCostLog = 10;
constexpr int kMaxWeight = 1 << 22;  // 32 lanes x 2^22 x 10 < 2^31

// Chains per warp.  A warp's lanes share its phases, so the longest lane of a
// warp of k chains takes about f(k) times as long as its chain alone would.
// Measured on GB300 with k chains of 800 steps per warp, one warp per SM
// sub-partition: f(2, 4, 8, 16, 32) = 1.38, 1.78, 2.27, 3.12, 3.77.  The
// batch lasts as long as its slowest warp, so the longest chains get the
// fewest lanes.  Tier j gives kTierK[j] chains to a warp and takes the chains
// with max_len / kTierF[j] < L <= max_len / kTierF[j - 1] (kTierF[-1] = 1),
// kTierF[j] ~ f(kTierK[j + 1]): a chain of length L then finishes within
// about max_len one-chain steps.  The table is f raised by about 7 % (a full
// GPU slows the shared warps a little more than an idle one); on the 65,536-
// chain batch it measured as fast as 1.15 times it and faster than 0.85 or
// 1.3 times it.  group = k > 0 puts k chains in every warp instead.
constexpr int kTiers = 6;
__constant__ int kTierK[kTiers] = {1, 2, 4, 8, 16, 32};
__constant__ float kTierF[kTiers] = {1.47f, 1.89f, 2.42f, 3.33f, 4.03f, 1e30f};

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

// A lane's position in its chain: the state, and the op codes and operands of
// steps t and t + 1 in registers.  Step t + 2's are loaded while step t runs,
// so that a chain's sequential steps do not wait on memory.
struct Cursor {
    int64_t c;
    int L, t;
    int op, opn;
    double b0, b1, b0n, b1n;
    int64_t sb2;  // step_base[t + 2]
    double x0, x1;
};

// Load step t + 2's op code and operand while step t runs, then advance.
__device__ __forceinline__ void load_next(Cursor& u, const uint8_t* __restrict__ ops, const double* __restrict__ a0,
                                          const double* __restrict__ a1, const int64_t* __restrict__ step_base,
                                          int& op2, double& b02, double& b12, int64_t& sb3) {
    op2 = 0;
    b02 = b12 = 0.0;
    sb3 = 0;
    if (u.t + 2 < u.L) {
        int64_t k2 = u.sb2 + u.c;
        op2 = __ldg(ops + k2);
        b02 = __ldg(a0 + k2);
        b12 = __ldg(a1 + k2);
        sb3 = (u.t + 3 < u.L) ? __ldg(step_base + u.t + 3) : 0;
    }
}

__device__ __forceinline__ void advance(Cursor& u, int op2, double b02, double b12, int64_t sb3) {
    u.op = u.opn;
    u.b0 = u.b0n;
    u.b1 = u.b1n;
    u.opn = op2;
    u.b0n = b02;
    u.b1n = b12;
    u.sb2 = sb3;
    ++u.t;
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
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // tier ends e[j] (chain index) and task counts: lane j < kTiers finds tier j's end
    int64_t e_mine = n_chains;
    if (group <= 0 && lane < kTiers - 1)
        e_mine = count_longer(len, n_chains, (int64_t)((float)max_len / kTierF[lane]));
    // A tier whose tasks, with those of the tiers before it, would not all fit
    // in the launch's warps at once doubles its chains per warp (up to 32): a
    // batch with many chains near max_len packs them rather than queueing
    // single-chain tasks behind each other.
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    int64_t e[kTiers], first[kTiers + 1];
    int kk[kTiers];
    first[0] = 0;
    int64_t b = 0;
#pragma unroll
    for (int j = 0; j < kTiers; ++j) {
        int64_t ej = __shfl_sync(kAll, e_mine, j);
        ej = (group > 0) ? ((j == kTiers - 1) ? n_chains : 0) : max(ej, b);
        int kj = (group > 0) ? group : kTierK[j];
        while (group <= 0 && kj < 32 && first[j] + (ej - b + kj - 1) / kj > warps) kj *= 2;
        kk[j] = kj;
        e[j] = ej;
        first[j + 1] = first[j] + (ej - b + kj - 1) / kj;
        b = ej;
    }
    while (true) {
        unsigned long long task = 0;
        if (lane == 0) task = atomicAdd(queue, 1ull);
        task = __shfl_sync(kAll, task, 0);
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
        Cursor u;
        u.c = start + lane;
        bool in = (lane < k) && (u.c < end);
        u.L = in ? len[u.c] : 0;
        u.t = 0;
        u.x0 = in ? s0[u.c] : 0.0;
        u.x1 = in ? s1[u.c] : 0.0;
        u.op = u.opn = 0;
        u.b0 = u.b1 = u.b0n = u.b1n = 0.0;
        u.sb2 = 0;
        if (u.L > 0) {
            int64_t k0 = __ldg(step_base) + u.c;
            u.op = __ldg(ops + k0);
            u.b0 = __ldg(a0 + k0);
            u.b1 = __ldg(a1 + k0);
            if (u.L > 1) {
                int64_t k1 = __ldg(step_base + 1) + u.c;
                u.opn = __ldg(ops + k1);
                u.b0n = __ldg(a0 + k1);
                u.b1n = __ldg(a1 + k1);
                u.sb2 = (u.L > 2) ? __ldg(step_base + 2) : 0;
            }
        }
        if (k == 1) {
            while (u.t < u.L) {
                int op2;
                double b02, b12;
                int64_t sb3;
                load_next(u, ops, a0, a1, step_base, op2, b02, b12, sb3);
                apply_op(u.op, u.b0, u.b1, u.x0, u.x1);
                advance(u, op2, b02, b12, sb3);
            }
        }
        while (k > 1 && __any_sync(kAll, u.t < u.L)) {
            // cheap phase
            while (true) {
                bool ch = (u.t < u.L) && u.op != TF_OP_EXP && u.op != TF_OP_LOG;
                if (!__any_sync(kAll, ch)) break;
                if (ch) {
                    int op2;
                    double b02, b12;
                    int64_t sb3;
                    load_next(u, ops, a0, a1, step_base, op2, b02, b12, sb3);
                    apply_cheap(u.op, u.b0, u.b1, u.x0, u.x1);
                    advance(u, op2, b02, b12, sb3);
                }
            }
            // costly phase: every running lane now waits on texp or tlog
            const bool run = u.t < u.L;
            const int w = run ? min(u.L - u.t, kMaxWeight) : 0;
            const int vote = __reduce_add_sync(kAll, u.op == TF_OP_EXP ? w * kCostLog : -w * kCostExp);
            const int X = vote >= 0 ? TF_OP_EXP : TF_OP_LOG;
            if (run && u.op == X) {
                int op2;
                double b02, b12;
                int64_t sb3;
                load_next(u, ops, a0, a1, step_base, op2, b02, b12, sb3);
                double z0 = u.x0, z1 = u.x1;
                if (X == TF_OP_EXP) tf::texp_impl<false, true>(u.x0, u.x1, z0, z1);
                else tf::tlog_impl<false>(u.x0, u.x1, z0, z1);
                u.x0 = z0;
                u.x1 = z1;
                advance(u, op2, b02, b12, sb3);
            }
        }
        if (in) {
            s0[u.c] = u.x0;
            s1[u.c] = u.x1;
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

// Error code of a failed (or successful) CUDA runtime call.  A failed call is
// never TF_OK.
int cuda_code(cudaError_t e) {
    if (e == cudaSuccess) return TF_OK;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return TF_ERR_NODEVICE;
    return TF_ERR_LAUNCH;
}

// Status after a launch: the launch's own error, read (and cleared) once.
int launch_status() { return cuda_code(cudaGetLastError()); }

// Status of a runtime call that returned e: its error code (the call's error
// is also cleared from the runtime's last-error slot, so that a later
// launch_status reports only that launch).
int call_status(cudaError_t e) {
    if (e != cudaSuccess) cudaGetLastError();
    return cuda_code(e);
}

inline bool al8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; }

// Scratch of tf_chain_noalloc: the work-queue counter lives in this array,
// which every device that loads the library holds until the process exits.
// Host code must not pass the symbol itself to a kernel (on the host it only
// stands for the device array); its device address is looked up instead.
constexpr int kNoAllocScratchBytes = TF_CHAIN_NOALLOC_SCRATCH;
static __device__ __align__(256) unsigned char g_chain_scratch[kNoAllocScratchBytes];

// The address is looked up once per CUDA context (with that context current)
// and cached under the context's id, which the driver never reuses within a
// process: a context that is destroyed and created again (cudaDeviceReset)
// loads the module again, possibly at another address, and gets a new id, so
// a stale address is never used.  The id comes from the driver's cuCtxGetId
// through the runtime's entry-point query (the library does not link the
// driver library itself).  Without that entry point every call looks the
// address up.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);
constexpr int kCacheSlots = 64;
std::mutex g_scratch_mu;
struct ScratchSlot {
    unsigned long long ctx_id;
    void* addr;
};
ScratchSlot g_scratch_cache[kCacheSlots] = {};
int g_scratch_next = 0;
bool g_entry_tried = false;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Id of the current context, or 0 if it cannot be had.
unsigned long long current_ctx_id() {
    if (!g_entry_tried) {
        g_entry_tried = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
        } else {
            cudaGetLastError();
        }
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_chain_scratch in the current device's context.
int noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return call_status(e);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    unsigned long long id = current_ctx_id();
    if (id != 0) {
        for (int k = 0; k < kCacheSlots; ++k) {
            if (g_scratch_cache[k].ctx_id == id) {
                *out = g_scratch_cache[k].addr;
                return TF_OK;
            }
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_chain_scratch);
    if (e != cudaSuccess) return call_status(e);
    if (!p) return TF_ERR_LAUNCH;
    if (id == 0) id = current_ctx_id();  // the lookup made the device's context current
    if (id != 0) {
        g_scratch_cache[g_scratch_next] = {id, p};
        g_scratch_next = (g_scratch_next + 1) % kCacheSlots;
    }
    *out = p;
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
    cudaError_t e = cudaFuncGetAttributes(&fa, chain_fused);
    if (e != cudaSuccess) return call_status(e);
    if (threads > fa.maxThreadsPerBlock) return TF_ERR_ARG;  // the kernel's registers do not fit
    if (blocks <= 0) {
        int dev = 0, sms = 0, per_sm = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chain_fused, threads, 0);
        if (e != cudaSuccess) return call_status(e);
        blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    // more warps than tasks would idle (a task has at least one chain)
    int64_t need = (n_chains + threads / 32 - 1) / (threads / 32);
    if (blocks > need) blocks = (int)need;
    e = cudaMemsetAsync(workspace, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return call_status(e);
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
