/*
 * tf.h -- C ABI of the GB300 twofold exp/log library (libtf.so).
 *
 * A twofold is a pair of floating-point numbers x0 + x1: the main part x0 is an
 * ordinary double and x1 assesses its deviation from the exact value (paper,
 * "Overview").  A twofold function z0 + z1 = f(x0 + x1) returns as main part z0
 * the correctly rounded f(x0) -- it depends on x0 only -- and as z1 a 1x-precise
 * estimate of the deviation f(x0 + x1) - z0, so that z0 + z1 is nearly
 * 2x-precise (paper, "Twofold exponent" > "Method summary").
 *
 * Common contract of the array entry points below:
 *   - Layout: structure of arrays.  Element i of the argument is x0[i] + x1[i];
 *     element i of the result is z0[i] + z1[i].  All arrays are contiguous
 *     doubles of length n.
 *   - Ownership: every pointer is a DEVICE pointer owned by the caller; the
 *     library allocates and frees nothing and keeps no pointer after the call.
 *     Pinned host memory (cudaHostAlloc / cudaHostRegister) is addressable from
 *     the device under unified addressing and may be passed as well: the
 *     kernel then reads and writes host memory over the GPU's host link.
 *   - x1 (and y1 for the binary operations) may be NULL: the argument is then
 *     "dotted", x1 = 0 (the paper's texp0/texpm10/tlog0/tlog1p0 variants).
 *     x0, z0 and z1 must not be NULL when n > 0.
 *   - Aliasing: z0 may be x0 and z1 may be x1 (in-place update); any other
 *     overlap of an output with an input or with the other output is undefined.
 *   - Alignment: pointers must be 8-byte aligned.  When every pointer is
 *     16-byte aligned the kernels use 128-bit loads and stores; otherwise a
 *     scalar kernel runs (same results, bit for bit).
 *   - Stream: the work is enqueued on `stream` (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream) and the call returns without
 *     waiting.  Errors of the execution itself surface at the caller's next
 *     synchronisation with that stream.
 *   - n == 0 is a no-op that returns TF_OK; n < 0 returns TF_ERR_SIZE.
 *   - Return value: TF_OK or one of the TF_ERR_* codes; nothing is printed,
 *     nothing is launched when an argument check fails.
 *   - Numerics: all arithmetic is IEEE binary64, round to nearest even, no
 *     flush of subnormals.  Special values: NaN in x0 gives z0 = z1 = NaN;
 *     NaN in x1 with a numeric z0 gives z1 = NaN; when z0 is +-Inf, or 0 by
 *     underflow, z1 = 0 (the paper's "avoid NaN" remark after the texp
 *     algorithm and its "domain errors" remark after tlog).
 */
#ifndef TF_H
#define TF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TF_OK = 0,
    TF_ERR_NULL = 1,     /* a required pointer is NULL */
    TF_ERR_SIZE = 2,     /* n < 0, or n beyond the supported range */
    TF_ERR_ALIGN = 3,    /* a pointer is not aligned to its element size */
    TF_ERR_LAUNCH = 4,   /* the kernel launch was rejected (cudaGetLastError) */
    TF_ERR_NODEVICE = 5, /* no usable CUDA device */
    TF_ERR_ARG = 6       /* another invalid argument (e.g. an unknown variant) */
};

/* Twofold exponent z0 + z1 = e^(x0 + x1).
 * Paper: "Twofold exponent" > "Algorithm summary", algorithms texp and texp0.
 * The 2x-precise e^x0 (the paper's pexp0) is computed here by a reduction
 * x0 = k ln2 + j ln2/65536 + r (N = 65536 k + j and the exact leading part of
 * r in binary64), a 2^(j/65536) table and the Taylor polynomial of
 * (e^r - 1)/r, the table product and the Taylor/Horner evaluation in exact
 * 128-bit integer fixed point (not in twofold arithmetic), then the 2^k
 * rescale in binary64.  z0 = RN(e^x0): +Inf for x0 >= 709.782712893384,
 * subnormal below x0 = -708.396..., 0 at or below x0 = -745.1332191019412. */
int tf_texp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);

/* Twofold z0 + z1 = e^(x0 + x1) - 1.
 * Paper: "Twofold exponent" > "Algorithm summary", texpm1 / texpm10 (with
 * pexpm10).  z0 = RN(e^x0 - 1); z0 = -1 for x0 below about -37.43. */
int tf_texpm1(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);

/* Twofold logarithm z0 + z1 = log(y0 + y1).
 * Paper: "Twofold logarithm" > "Newton inversion" and "Algorithm summary"
 * (tlog, plog, tlog0): y0 = 2^n z, log z = -log c_i - log c2_j + log1p(t)
 * with two reciprocal tables c_i, c2_j, and one Newton step on e^x seeded by a
 * 1x-precise log1p of the reduced argument t (the reduction, seed, Newton step
 * and final sum in exact 128-bit integer fixed point).
 * z0 = RN(log y0); y0 < 0 or NaN gives NaN, y0 = +-0 gives -Inf (z1 = 0).
 * y1 may be any double: a twofold that is not renormalised takes a slower
 * path in its warp. */
int tf_tlog(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);

/* Twofold z0 + z1 = log(1 + y0 + y1).
 * Paper: "Twofold logarithm" > "Newton inversion" and "Algorithm summary"
 * (tlog1p, plog1p, tlog1p0): Newton step on e^x - 1.  z0 = RN(log1p y0);
 * y0 < -1 gives NaN, y0 = -1 gives -Inf (z1 = 0). */
int tf_tlog1p(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);

/* Coupled results.  Paper: "Twofold exponent" > "Algorithm summary" (pexp,
 * pexpm1: "coupled exponent of coupled argument") and "Twofold logarithm" >
 * "Algorithm summary" (plog, plog1p).  z0 + z1 is the same 2x-precise value as
 * the twofold function's, renormalised: z0 = RN(z0 + z1) (so z0 is the
 * correctly rounded f(x0 + x1) unless that lies within about 2^-106 relative
 * of a rounding midpoint) and z1 the exact remainder.  x1 = NULL gives pexp0,
 * pexpm10, plog0, plog1p0.  Special results (z0 or z1 not finite) and z1 = 0
 * are returned as the twofold function returns them.  Same contract as tf_texp. */
int tf_pexp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);
int tf_pexpm1(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);
int tf_plog(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);
int tf_plog1p(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);

/* Twofold results of coupled arguments.  Paper: texpp, texpm1p ("twofold
 * exponent of coupled argument"), tlogp, tlog1pp ("coupled argument,
 * |y1| << |y0|").  As tf_texp, tf_texpm1, tf_tlog, tf_tlog1p, except that the
 * argument is taken as coupled (|x1| at most about 2^-30 |x0|; 2^-20 for
 * tlog1pp relative to 1 + y0): the renormalising path for a loose x1 is not
 * taken, so for a loose argument z1 is only first-order accurate.  Non-finite
 * x1 keep the twofold functions' rules. */
int tf_texpp(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);
int tf_texpm1p(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);
int tf_tlogp(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);
int tf_tlog1pp(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);

/* tf_texp computed with the paper's own argument reduction instead (an A/B
 * variant).  Paper: "Function pexp0()": x = 2^L m + 2^-K n + y with y exact and
 * e^x = E C e^y, E = e^(2^L m) and C = e^(n/2^K) from tables; here K = 8 and
 * L = 1 (|y| <= 2^-9, so the Taylor part is the same as tf_texp's), the tables
 * e^(2m) and e^(n/256) in 128-bit fixed point.  Same results contract as
 * tf_texp (z0 = RN(e^x0), z0 + z1 within the same bound; z1 may differ from
 * tf_texp's in its last bits). */
int tf_texp_tables(const double* x0, const double* x1, double* z0, double* z1, int64_t n, void* stream);

/* tf_tlog and tf_tlog1p with the Newton step taken in binary64 (A/B variants).
 * Paper: "Twofold logarithm" > "Newton inversion": after the 1x seed R of
 * log1p(t), one Newton step on e^x gives u = (1 + t) e^-R - 1 and log1p(t) = R +
 * log1p(u).  tf_tlog/tf_tlog1p take u in exact 128-bit integer fixed point;
 * these take e^-R - 1 = S and t as pairs of doubles and u = t + S + t S with
 * binary64 operations (FMA-based exact product, exact sums where the terms
 * cancel), the paper's own arithmetic for that step.  Same results contract as
 * tf_tlog/tf_tlog1p (z0 = RN(log y0) resp. RN(log1p y0), z0 + z1 within the
 * same bound; z1 may differ in its last bits). */
int tf_tlog_newton_fp64(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);
int tf_tlog1p_newton_fp64(const double* y0, const double* y1, double* z0, double* z1, int64_t n, void* stream);

/* Float twofolds: the same four functions over pairs of floats, with the
 * paper's "f"-suffixed float variants in mind ("Twofold exponent" and
 * "Twofold logarithm" give each algorithm for float and double).  Every
 * pointer is a device float array of n elements; alignment 4 bytes (16 for
 * the 128-bit vector kernel); otherwise the contract of the double entry
 * points applies.  All arithmetic is float-float on the FP32 pipes, IEEE
 * binary32 round to nearest, no flush of subnormals.  z0 = RN_float(f(x0));
 * texpf overflows at x0 >= 88.72284 and underflows to 0 at x0 <= -103.97208;
 * tlogf/tlog1pf as tlog/tlog1p. */
int tf_texpf(const float* x0, const float* x1, float* z0, float* z1, int64_t n, void* stream);
int tf_texpm1f(const float* x0, const float* x1, float* z0, float* z1, int64_t n, void* stream);
int tf_tlogf(const float* y0, const float* y1, float* z0, float* z1, int64_t n, void* stream);
int tf_tlog1pf(const float* y0, const float* y1, float* z0, float* z1, int64_t n, void* stream);

/* Twofold sum z0 + z1 = (x0 + x1) + (y0 + y1).
 * Paper: "Overview" (z0 = x0 (+) y0, the ordinary double sum) and
 * "Twofolds update" > "Twofold bugs", Algorithm 2.2 (the exact rounding error
 * of x0 (+) y0); z1 = that error + (x1 + y1).  z0 is NOT renormalised. */
int tf_tadd(const double* x0, const double* x1, const double* y0, const double* y1,
            double* z0, double* z1, int64_t n, void* stream);

/* Twofold product z0 + z1 = (x0 + x1)(y0 + y1).
 * Paper: "Overview" (z0 = x0 (*) y0) and "Twofold exponent" > "Method summary"
 * (FMA-based exact product, 2 MUL + 1 FMA + 1 ADD per twofold-by-dotted step):
 * z1 = x0 y1 + x1 y0 + fma(x0, y0, -z0) (two FMAs); the x1 y1 term is dropped. */
int tf_tmul(const double* x0, const double* x1, const double* y0, const double* y1,
            double* z0, double* z1, int64_t n, void* stream);

/* ------------------------------------------------------------------------
 * Chains of twofold operations (the paper's on-the-fly error tracking: a
 * twofold carries its deviation z1 through a whole computation, "Overview";
 * here many independent computations run at once).
 *
 * A batch holds n_chains independent chains.  Chain c starts from the twofold
 * state s = s0[c] + s1[c] and applies len[c] operations in order; operation t
 * of chain c is ops[k] with operand a = a0[k] + a1[k], k = step_base[t] + c:
 *   TF_OP_ADD  s <- tadd(s, a)      TF_OP_MUL  s <- tmul(s, a)
 *   TF_OP_EXP  s <- texp(s)         TF_OP_LOG  s <- tlog(s)   (a unused)
 * each exactly as the elementwise entry points compute it.  Layout ("step
 * major"): the chains are numbered by non-increasing length, so the chains
 * still running at step t are 0 .. active(t) - 1, and step t's operations are
 * the contiguous block ops/a0/a1[step_base[t] .. step_base[t] + active(t)),
 * with step_base[0] = 0 and step_base[t + 1] = step_base[t] + active(t).
 * step_base has max_len + 1 entries (the last is the total number of
 * operations).  s0/s1 are updated in place and hold the final states on
 * return.  All pointers are device pointers owned by the caller.  An unknown
 * op code leaves the state unchanged.
 * ------------------------------------------------------------------------ */
enum { TF_OP_ADD = 0, TF_OP_MUL = 1, TF_OP_EXP = 2, TF_OP_LOG = 3 };

/* Bytes of device workspace tf_chain needs (the work-queue counter). */
#define TF_CHAIN_WORKSPACE 256

/* All chains in one persistent launch: each warp takes the next task (a run
 * of consecutive chains) from an atomic work queue (a counter in `workspace`,
 * reset by this call with an asynchronous memset on `stream`) and runs its
 * chains to the end, so short and long chains balance across the GPU; no
 * thread ever waits on another.
 * group: chains per task.  1 .. 32 puts that many chains in every task (one
 * per lane; lanes beyond it idle).  A warp of several chains alternates a
 * phase that runs every lane's pending tadd/tmul with one that runs texp or
 * tlog for the lanes waiting on it, so its chains share its time.  0 picks
 * the group by length: the longest chains (above max_len / 1.47) run one per
 * warp, then 2, 4, 8, 16 per warp down to max_len / 4.03, and the rest 32 per
 * warp; a tier whose tasks, with the longer tiers', outnumber the launch's
 * warps packs more chains per warp (up to 32), so that batches with many
 * chains near max_len are not queued one chain per task.  The tiers are found
 * by a binary search of len, which must then be non-increasing (the
 * step-major layout above already requires it).  Results
 * do not depend on group, threads or blocks: every chain runs the same
 * operations in the same order.
 * threads: block size, a multiple of 32 in [32, 1024] that the kernel's register
 * use allows (TF_ERR_ARG otherwise; 512 always fits); blocks: grid size, <= 0
 * for one wave of resident blocks (capped at what n_chains can use).
 * workspace: TF_CHAIN_WORKSPACE bytes of device memory, 8-byte aligned,
 * owned by the caller and used by no other call in flight (concurrent calls
 * need separate workspaces).  len must be 4-byte aligned, the double and
 * int64 arrays 8-byte aligned.  Returns TF_ERR_ARG for a bad block size or
 * group, TF_ERR_NULL / TF_ERR_SIZE / TF_ERR_ALIGN as the other calls. */
int tf_chain(const uint8_t* ops, const double* a0, const double* a1, const int64_t* step_base,
             const int32_t* len, double* s0, double* s1, int64_t n_chains, int32_t max_len,
             void* workspace, int threads, int blocks, int group, void* stream);

/* tf_chain without the caller's workspace, for callers that cannot allocate
 * device memory themselves: code that runs where a host framework owns all of
 * the device's memory through its own pool or a hard cap, and code on a
 * latency-critical path that cannot afford cudaMalloc, which may synchronize
 * the whole device.  The paper has no counterpart; it is a deployment variant
 * of tf_chain.
 *
 * The work-queue counter lives in a static device array of
 * TF_CHAIN_NOALLOC_SCRATCH bytes inside the library, which every GPU that
 * loads the library holds until the process exits.  This call allocates
 * nothing: the first call in each CUDA context (normally once per device, in
 * its primary context) looks up that context's address of the array
 * (cudaGetSymbolAddress, with the device current) and caches it under the
 * context's id, so make that first call before any stream capture.  After a
 * cudaDeviceReset the device's new context gets a new id and the address is
 * looked up again (the array starts over at another address).  Every call clears the
 * counter on `stream` and then uses it; all calls share the one array, so
 * calls whose work overlaps on the GPU (on different streams, or from
 * different host threads) race on it and give wrong results: keep them
 * ordered.  Arguments and results as tf_chain; n_chains above
 * TF_CHAIN_NOALLOC_MAX_CHAINS returns TF_ERR_SIZE. */
#define TF_CHAIN_NOALLOC_SCRATCH 256
#define TF_CHAIN_NOALLOC_MAX_CHAINS (1LL << 40)
int tf_chain_noalloc(const uint8_t* ops, const double* a0, const double* a1, const int64_t* step_base,
                     const int32_t* len, double* s0, double* s1, int64_t n_chains, int32_t max_len,
                     int threads, int blocks, int group, void* stream);

/* One operation kind at one step, for the chains listed in idx[0 .. n_idx)
 * (the per-op baseline: one launch per step and operation kind): for each
 * listed chain c, s[c] <- op(s[c], a[step_base_t + c]).  op is one of TF_OP_*. */
int tf_chain_step(int op, const int32_t* idx, int64_t n_idx, int64_t step_base_t, const double* a0,
                  const double* a1, double* s0, double* s1, void* stream);

/* Human-readable name of an error code (static storage, never NULL). */
const char* tf_strerror(int code);

/* Version of this ABI: (major << 16) | minor. */
int tf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TF_H */
