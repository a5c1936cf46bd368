// tf_core_f.cuh -- per-element twofold exp/log over float (device functions).
//
// The float twofold z0 + z1 (two floats) of the same four functions as the
// double path (paper: the float variants of texp, texpm1, tlog, tlog1p, "f"
// suffix), with all the Taylor, table and Newton arithmetic in float-float
// on the FP32 pipes (paper, "Method summary": twofold partial sums with
// 1x-precise coefficients; TwoSum / FMA-based TwoProduct in float):
//
//   exp core   x = N ln2/512 + r, N = 512 k + j, r = rh + rl (ln2/512 in three
//              floats, the first of 7 bits so that N C0 is exact);
//              e^r - 1 = rh + rh^2/2 + rh^3 q(rh) + rl (1 + rh), the first two
//              terms in float-float, the dotted tail q in float (|r| < 2^-10.5,
//              so the tail's rounding stays below 2^-55 and e^x - 1 keeps
//              2^-45 relative where E_j + T_j P cancels);
//              e^x = 2^k T_j (1 + P),  e^x - 1 = 2^k (E_j + T_j P) + 2^k - 1
//   log        y = 2^n z, z in [sqrt(1/2), sqrt(2)), d = z - 1 exact; a
//              reciprocal table reduces z to t = z c_i - 1 (exact pair,
//              |t| < 2^-11.4); seed R ~ log1p(t) (1x float); one Newton step
//              on e^x: u = t + S + t S, S = e^-R - 1 (a short float-float
//              series); log y = n ln2 - log c_i + R + u (paper, "Newton
//              inversion")
//
// z0 = RN_float(f(x0)) from the float-float value (2^-46 or better), so it is
// correctly rounded unless f(x0) lies that close to a rounding midpoint; the
// special-value rules are those of the double path.
#pragma once

#include "tf_core.cuh"

namespace tff {

using tf::warp_any;

struct ff {
    float hi, lo;
};

__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ uint32_t bits(float a) { return (uint32_t)__float_as_int(a); }
__device__ __forceinline__ float from_bits(uint32_t b) { return __int_as_float((int)b); }
__device__ __forceinline__ uint32_t absbits(float a) {  // kept on the integer ALU (see tf_eft.cuh)
    uint32_t r;
    asm("and.b32 %0, %1, 0x7fffffff;" : "=r"(r) : "r"(bits(a)));
    return r;
}

constexpr uint32_t kExpMask = 0x7f800000u;
constexpr uint32_t kSignMask = 0x80000000u;
constexpr uint32_t kMantMask = 0x007fffffu;
constexpr float kInf = __builtin_huge_valf();

__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    float s = add(a, b);
    return {s, sub(b, sub(s, a))};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
    float s = add(a, b);
    float bp = sub(s, a);
    float ap = sub(s, bp);
    return {s, add(sub(a, ap), sub(b, bp))};
}
__device__ __forceinline__ ff sorted_two_sum(float a, float b) {
    bool sw = absbits(b) > absbits(a);
    return fast_two_sum(sw ? b : a, sw ? a : b);
}
__device__ __forceinline__ ff two_prod(float a, float b) {
    float p = mul(a, b);
    return {p, fma_rn(a, b, -p)};
}

// 2^k as a float for any int k: 0 below 2^-149, +Inf above 2^127.
__device__ __forceinline__ float pow2f(int k) {
    uint32_t normal = (uint32_t)(k + 127) << 23;
    uint32_t subn = (k >= -149) ? (1u << ((k + 149) & 31)) : 0u;
    uint32_t b = (k >= -126) ? normal : subn;
    b = (k > 127) ? kExpMask : b;
    return from_bits(b);
}

__device__ __forceinline__ ff tab(const float (*t)[2], int j) {
    float2 v = __ldg(reinterpret_cast<const float2*>(t) + (j + TF_F_TAB_HALF));
    return {v.x, v.y};
}

// ---------------------------------------------------------------------------
// exp core.  r = rh + rl to ~2^-57 absolute for |N| <= 256 (2^-48 at the
// largest N); P = e^r - 1 as Ph + Pl to ~2^-57 (|r| < 2^-10.5: the cubic tail
// rh^3 q, rounded in float, stays below 2^-34).
// ---------------------------------------------------------------------------
struct RedF {
    float rh, rl;
    int N;
};

__device__ __forceinline__ RedF reduce_f(float x) {
    const float kShift = 0x1.8p23f;
    float t = fma_rn(x, TF_F_INV_C, kShift);  // |x 512/ln2| < 2^22: N in the low bits
    int N = (int)(bits(t) - bits(kShift));
    float Nf = sub(t, kShift);
    float r0 = fma_rn(-Nf, TF_F_C0, x);  // exact: N C0 has at most 24 bits (|N| < 2^17)
    ff p1 = two_prod(Nf, TF_F_C1);
    ff r = two_sum(r0, -p1.hi);
    float rl = fma_rn(-Nf, TF_F_C2, sub(r.lo, p1.lo));
    ff rr = fast_two_sum(r.hi, rl);
    return {rr.hi, rr.lo, N};
}

__device__ __forceinline__ ff expm1_reduced_f(float rh, float rl) {
    float q = fma_rn(fma_rn(TF_F_R5, rh, TF_F_R4), rh, TF_F_R3);  // 1/6 + rh/24 + rh^2/120
    ff s2 = two_prod(rh, rh);
    float r3 = mul(s2.hi, rh);
    ff P = fast_two_sum(rh, mul(0.5f, s2.hi));  // |rh| > rh^2/2
    P.lo = add(P.lo, add(mul(0.5f, s2.lo), fma_rn(r3, q, fma_rn(rl, rh, rl))));
    return P;
}

// T P as m.hi + m.lo (T.lo P.lo dropped).
__device__ __forceinline__ ff tab_times_f(ff T, ff P) {
    ff m = two_prod(T.hi, P.hi);
    m.lo = fma_rn(T.hi, P.lo, fma_rn(T.lo, P.hi, m.lo));
    return m;
}

struct ExpCoreF {
    float zA, eA;  // zA + eA = e^x / 2^k, zA = RN of it, in [0.70, 1.42]
    int k;
};

__device__ __forceinline__ ExpCoreF exp_core_f(float x) {
    RedF R = reduce_f(x);
    int k = (R.N + TF_F_TAB_HALF) >> 9;
    int j = R.N - (k << 9);
    ff P = expm1_reduced_f(R.rh, R.rl);
    ff T = tab(TF_FT_TABLE, j);
    ff m = tab_times_f(T, P);
    ff s = fast_two_sum(T.hi, m.hi);
    float lo = add(s.lo, add(T.lo, m.lo));
    ff z = fast_two_sum(s.hi, lo);
    return {z.hi, z.lo, k};
}

// e^x - 1 for |x| <= 0.3466 (k = 0, j = N in [-256, 256]) as a renormalised pair:
// E_j + T_j P (|E_j| >= 0.00135 > |T_j P|), or P itself for N = 0 (r = x exactly,
// so the relative precision holds down to tiny x).
__device__ __forceinline__ ff expm1_small_f(float x) {
    RedF R = reduce_f(x);
    ff P = expm1_reduced_f(R.rh, R.rl);
    ff T = tab(TF_FT_TABLE, R.N);
    ff E = tab(TF_FE_TABLE, R.N);
    ff m = tab_times_f(T, P);
    ff s = fast_two_sum(E.hi, m.hi);
    ff W = fast_two_sum(s.hi, add(s.lo, add(E.lo, m.lo)));
    return (R.N == 0) ? fast_two_sum(P.hi, P.lo) : W;
}

// Clamp into [-104, 89] with integer compares (NaN goes to one end).
__device__ __forceinline__ float clamp_exp_arg(float x) {
    uint32_t b = bits(x);
    uint32_t ab = b & ~kSignMask;
    bool neg = (b & kSignMask) != 0;
    x = (!neg && ab > bits(89.0f)) ? 89.0f : x;
    x = (neg && ab > bits(104.0f)) ? -104.0f : x;
    return x;
}

// (z + e)(x1 + x1^2/2) + c for e^x0 = z + e (z its leading float, e the rest)
// and a small x1 (|x1| < 2^-15: the x1^3/6 term is below 2^-47.6 e^x0): t = z
// x1/2 + e, then t x1 + c, then z x1 + that, the large term rounded once.
__device__ __forceinline__ float add_pert(float z, float e, float x1, float c) {
    float t = fma_rn(z, mul(0.5f, x1), e);
    return fma_rn(z, x1, fma_rn(t, x1, c));
}
__device__ __forceinline__ bool pert_is_large(float x1) { return absbits(x1) >= 0x38000000u; }  // 2^-15
__device__ __forceinline__ bool pert_is_loose(float x1) { return absbits(x1) > 0x3eae0000u; }   // 0.33984

static __device__ __noinline__ ff expm1_pair_f(float x1) {
    if (absbits(x1) <= 0x3eae0000u) return expm1_small_f(x1);
    return {expm1f(x1), 0.0f};
}

// kPair: the 2x-precise e^x1 - 1 for every finite x1 (texpm1f, whose result
// may be as small as x1 itself).
template <bool kPair = false>
__device__ __forceinline__ float pert_term(float eh, float el, float x1, float c) {
    if (!kPair && !pert_is_large(x1)) return fma_rn(eh, x1, fma_rn(el, x1, fma_rn(eh, mul(mul(0.5f, x1), x1), c)));
    if (absbits(x1) >= kExpMask) return (x1 > 0.0f) ? x1 : sub(sub(c, el), eh);
    ff t = expm1_pair_f(x1);
    return fma_rn(eh, t.hi, fma_rn(el, t.hi, fma_rn(eh, t.lo, c)));
}

// Round 2^k (zA + eA) to the float grid when the result may be subnormal.
__device__ __forceinline__ float round_subnormal_inl(float zA, float eA, int k) {
    float sc = pow2f(k + 149);  // k + 149 in [-3, 24]
    float u = mul(zA, sc);      // exact
    float g = mul(eA, sc);
    float m = rintf(u);
    float f = sub(u, m);
    m = (f == 0.5f && g > 0.0f) ? add(m, 1.0f) : m;
    m = (f == -0.5f && g < 0.0f) ? sub(m, 1.0f) : m;
    return mul(m, 0x1p-149f);
}

// The same out of line, for the rare paths.
static __device__ __noinline__ float round_subnormal_f(float zA, float eA, int k) {
    return round_subnormal_inl(zA, eA, k);
}

template <bool kVote, bool kTop = kVote>
__device__ __forceinline__ void texpf_impl(float x0, float x1, float& z0, float& z1);
template <bool kVote, bool kTop = kVote>
__device__ __forceinline__ void texpm1f_impl(float x0, float x1, float& z0, float& z1);

// A loose twofold: f at the renormalised sum, z1 = (w0 - z0) + w1.
template <bool kExpm1>
static __device__ __noinline__ float loose_deviation_f(float x0, float x1, float z0) {
    if (absbits(x1) >= kExpMask) {
        if (x1 > 0.0f) return x1;
        return kExpm1 ? sub(-1.0f, z0) : -z0;
    }
    ff s = two_sum(x0, x1);
    if (absbits(s.hi) >= kExpMask) return (s.hi > 0.0f) ? s.hi : (kExpm1 ? sub(-1.0f, z0) : -z0);
    float slo = (absbits(s.hi) >= bits(256.0f)) ? 0.0f : s.lo;
    float w0, w1;
    if constexpr (kExpm1) texpm1f_impl<false, false>(s.hi, slo, w0, w1);
    else texpf_impl<false, false>(s.hi, slo, w0, w1);
    if (absbits(w0) == kExpMask) return w0;
    ff d = two_sum(w0, -z0);  // w0 - z0 exactly
    return add(d.hi, add(d.lo, w1));
}

// ---------------------------------------------------------------------------
// texp over float
// ---------------------------------------------------------------------------
template <bool kTop>
static __device__ __noinline__ void texpf_rare(float x0, float x1, float zA, float eA, int k, float& z0, float& z1) {
    float e;
    if (k > 127) {
        float sh = pow2f(k - 64);
        z0 = mul(mul(zA, sh), 0x1p64f);
        e = mul(mul(eA, sh), 0x1p64f);
    } else if (k < -125) {
        z0 = round_subnormal_f(zA, eA, k);
        e = 0.0f;
    } else {
        float sk = pow2f(k);
        z0 = mul(zA, sk);
        e = mul(eA, sk);
    }
    if constexpr (kTop) {
        if (pert_is_loose(x1)) {
            z1 = loose_deviation_f<false>(x0, x1, z0);
            return;
        }
    }
    z1 = pert_term(z0, e, x1, e);  // e^x0 = z0 + e
}

template <bool kVote, bool kTop>
__device__ __forceinline__ void texpf_impl(float x0, float x1, float& z0, float& z1) {
    if constexpr (kVote) {
        // |x0| <= 88 and a finite x1 everywhere in the warp (one vote): no
        // clamp, k <= 127, a finite nonzero result, no special values.  A
        // separate path rather than selects on a warp-uniform flag: predicated
        // instructions still take issue slots, and this kernel is issue-bound.
        // The subnormal results (x0 below -87.3, k <= -126) are rounded inline
        // under their own vote, the lanes with a large x1 go to the rare path.
        const bool special = !(fabsf(x0) <= 88.0f) | !(fabsf(x1) < kInf);
        if (!warp_any<kVote>(special)) {
            ExpCoreF c = exp_core_f(x0);
            float sk = from_bits((uint32_t)(c.k + 127) << 23);
            z0 = mul(c.zA, sk);
            z1 = mul(add_pert(c.zA, c.eA, x1, c.eA), sk);
            bool rare = fabsf(x1) >= 0x1p-15f;  // pert_is_large for a finite x1
            bool sub = (c.k < -125) & !rare;
            if (warp_any<kVote>(sub)) {
                if (sub) {
                    z0 = round_subnormal_inl(c.zA, c.eA, c.k);
                    z1 = pert_term(z0, 0.0f, x1, 0.0f);
                }
            }
            if (warp_any<kVote>(rare)) {
                if (rare) texpf_rare<kTop>(x0, x1, c.zA, c.eA, c.k, z0, z1);
            }
            return;
        }
    }
    ExpCoreF c = exp_core_f(clamp_exp_arg(x0));
    float sk = from_bits((uint32_t)(c.k + 127) << 23);  // 2^k for -126 <= k <= 127; other k are rare
    z0 = mul(c.zA, sk);
    z1 = mul(add_pert(c.zA, c.eA, x1, c.eA), sk);  // one rounding into a subnormal z1
    bool rare = (c.k < -125) | (c.k > 127) | pert_is_large(x1);
    if (warp_any<kVote>(rare)) {
        if (rare) texpf_rare<kTop>(x0, x1, c.zA, c.eA, c.k, z0, z1);
    }
    uint32_t a0 = absbits(z0);
    z1 = (a0 == 0 || a0 == kExpMask) ? 0.0f : z1;
    z1 = (absbits(x1) > kExpMask) ? x1 : z1;
    bool nan0 = absbits(x0) > kExpMask;
    z0 = nan0 ? x0 : z0;
    z1 = nan0 ? x0 : z1;
}

// kN elements of a thread in one call: one vote on special inputs for all of
// them; a warp without any runs the kN main paths in straight-line code, then
// one vote on subnormal results and one on rare lanes; any other warp runs
// texpf_impl for each.  Results are those of texpf_impl, bit for bit.  The
// float kernel calls it twice with kN = 2 for its four elements per thread:
// 2.8 % faster at 2^28 than four per-element calls; kN = 4 spilled at 32
// registers and was 2 % slower.
template <int kN>
__device__ __forceinline__ void texpf_multi(const float* x0, const float* x1, float* z0, float* z1) {
    bool special = false;
#pragma unroll
    for (int q = 0; q < kN; ++q) special |= !(fabsf(x0[q]) <= 88.0f) | !(fabsf(x1[q]) < kInf);
    if (__any_sync(0xffffffffu, special)) {
#pragma unroll
        for (int q = 0; q < kN; ++q) texpf_impl<true>(x0[q], x1[q], z0[q], z1[q]);
        return;
    }
    ExpCoreF c[kN];
    bool rare[kN], sub[kN], anysub = false, anyrare = false;
#pragma unroll
    for (int q = 0; q < kN; ++q) {
        c[q] = exp_core_f(x0[q]);
        float sk = from_bits((uint32_t)(c[q].k + 127) << 23);
        z0[q] = mul(c[q].zA, sk);
        z1[q] = mul(add_pert(c[q].zA, c[q].eA, x1[q], c[q].eA), sk);
        rare[q] = fabsf(x1[q]) >= 0x1p-15f;
        sub[q] = (c[q].k < -125) & !rare[q];
        anysub |= sub[q];
        anyrare |= rare[q];
    }
    if (__any_sync(0xffffffffu, anysub)) {
#pragma unroll
        for (int q = 0; q < kN; ++q) {
            if (sub[q]) {
                z0[q] = round_subnormal_inl(c[q].zA, c[q].eA, c[q].k);
                z1[q] = pert_term(z0[q], 0.0f, x1[q], 0.0f);
            }
        }
    }
    if (__any_sync(0xffffffffu, anyrare)) {
#pragma unroll
        for (int q = 0; q < kN; ++q)
            if (rare[q]) texpf_rare<true>(x0[q], x1[q], c[q].zA, c[q].eA, c[q].k, z0[q], z1[q]);
    }
}

// ---------------------------------------------------------------------------
// texpm1 over float.  k = 0: E_j + T_j P (or P); k >= 1: 2^k (V - 2^-k);
// k <= -1: V 2^k - 1, V = e^x / 2^k (for k <= -25 this is -1 + e^x exactly as
// a pair).
// ---------------------------------------------------------------------------
template <bool kTop>
static __device__ __noinline__ void texpm1f_rare(float x0, float x1, float vh, float vl, float zl, int k, float& z0,
                                                 float& z1) {
    float exh, exl, e;
    if (k > 127) {
        float sh = pow2f(k - 64);
        z0 = mul(mul(vh, sh), 0x1p64f);
        e = mul(mul(vl, sh), 0x1p64f);
        exh = z0;
        exl = e;
    } else {
        ff s = two_sum(1.0f, z0);
        exh = s.hi;
        exl = add(s.lo, zl);
        e = zl;
    }
    if constexpr (kTop) {
        if (pert_is_loose(x1)) {
            z1 = loose_deviation_f<true>(x0, x1, z0);
            return;
        }
    }
    z1 = pert_term<true>(exh, exl, x1, e);
}

// |x1| >= 2^-16 min(1, |x0|) (exponent fields): texpm1f's second-order term
// could then miss 2^-44 of the result, and the lane takes the rare path.
__device__ __forceinline__ bool pert_is_large_m1(float x0, float x1) {
    uint32_t a = min(absbits(x0), 0x3f800000u);
    uint32_t thr = (a > (16u << 23)) ? ((a & kExpMask) - (16u << 23)) : 0u;
    return absbits(x1) > thr;
}

// e^x - 1 = z0 + zl (z0 its leading float) and V = e^x / 2^k for an x in
// [-104, 89].
struct Expm1F {
    float z0, zl;
    ff V;
    int k;
};

__device__ __forceinline__ Expm1F expm1_core_f(float x) {
    RedF R = reduce_f(x);
    int k = (R.N + TF_F_TAB_HALF) >> 9;
    k = (R.N == TF_F_TAB_HALF) ? 0 : k;
    int j = R.N - (k << 9);
    ff P = expm1_reduced_f(R.rh, R.rl);
    ff T = tab(TF_FT_TABLE, j);
    ff E = tab(TF_FE_TABLE, j);
    ff m = tab_times_f(T, P);
    // V = T (1 + P) = e^x / 2^k
    ff s = fast_two_sum(T.hi, m.hi);
    ff V = fast_two_sum(s.hi, add(s.lo, add(T.lo, m.lo)));
    // k = 0
    ff se = fast_two_sum(E.hi, m.hi);
    ff W0 = fast_two_sum(se.hi, add(se.lo, add(E.lo, m.lo)));
    W0 = (R.N == 0) ? fast_two_sum(P.hi, P.lo) : W0;
    // k != 0: A + B + C with A + B exact by TwoSum
    bool kpos = k >= 1;
    float sk = pow2f(k);
    float A = kpos ? V.hi : -1.0f;
    float B = kpos ? -pow2f(-k) : mul(V.hi, sk);
    float C = kpos ? V.lo : mul(V.lo, sk);
    ff ab = two_sum(A, B);
    ff W1 = fast_two_sum(ab.hi, add(ab.lo, C));
    ff W = (k == 0) ? W0 : W1;
    float sc = kpos ? sk : 1.0f;
    return {mul(W.hi, sc), mul(W.lo, sc), V, k};
}

template <bool kVote, bool kTop>
__device__ __forceinline__ void texpm1f_impl(float x0, float x1, float& z0, float& z1) {
    if constexpr (kVote) {
        // |x0| <= 88, x0 != 0 and a finite x1 everywhere in the warp (one
        // vote): no clamp, k <= 127, no special values
        const bool special = !(fabsf(x0) <= 88.0f) | !(fabsf(x1) < kInf) | (x0 == 0.0f);
        if (!warp_any<kVote>(special)) {
            Expm1F c = expm1_core_f(x0);
            z0 = c.z0;
            ff ex = sorted_two_sum(1.0f, z0);  // e^x0 = ex.hi + ex.lo + zl
            z1 = add_pert(ex.hi, add(ex.lo, c.zl), x1, c.zl);
            bool rare = pert_is_large_m1(x0, x1);
            if (warp_any<kVote>(rare)) {
                if (rare) texpm1f_rare<kTop>(x0, x1, c.V.hi, c.V.lo, c.zl, c.k, z0, z1);
            }
            return;
        }
    }
    Expm1F c = expm1_core_f(clamp_exp_arg(x0));
    z0 = c.z0;
    ff ex = sorted_two_sum(1.0f, z0);  // e^x0 = ex.hi + ex.lo + zl
    z1 = add_pert(ex.hi, add(ex.lo, c.zl), x1, c.zl);
    bool rare = (c.k > 127) | pert_is_large_m1(x0, x1);
    if (warp_any<kVote>(rare)) {
        if (rare) texpm1f_rare<kTop>(x0, x1, c.V.hi, c.V.lo, c.zl, c.k, z0, z1);
    }
    uint32_t b0 = bits(x0);
    z0 = ((b0 & ~kSignMask) == 0) ? x0 : z0;  // expm1(-0) = -0
    bool neginf = b0 == (kSignMask | kExpMask);
    z1 = (absbits(z0) == kExpMask || neginf) ? 0.0f : z1;
    z1 = (absbits(x1) > kExpMask) ? x1 : z1;
    bool nan0 = absbits(x0) > kExpMask;
    z0 = nan0 ? x0 : z0;
    z1 = nan0 ? x0 : z1;
}

// ---------------------------------------------------------------------------
// Logarithm over float (paper, "Newton inversion"), after a reciprocal-table
// reduction as in the double path.  z = 1 + d in [sqrt(1/2), sqrt(2)),
// i = round(2048 z), c = c_i from TF_FLOGT (the float nearest 2048/i):
//   log z = -log c + log1p(t),   t = (c - 1) + d c = th + tl exactly
// (d c split by an FMA; (c - 1) plus its high part cancels exactly by the
// Sterbenz lemma, or c = 1), |t| < 2^-11.4.  Seed R = t - t^2/2 + t^3/3 in
// float (within about 2^-24 |t|); one Newton step on e^x:
//   S = e^-R - 1 = -R + R^2/2 - R^3/6 + R^4/24 - R^5/120 as a float pair,
//   u = (1 + t)(1 + S) - 1 = t + S + t S   (t + S and t S cancel exactly),
//   log1p(t) = R + u (u^2/2 is below 2^-48 |t|).
// Then n ln2 (a float pair from a table) - log c (a float pair) + R + u, the
// leading parts by Fast2Sum: |n ln2| >= 0.69 > |log c| unless n = 0, and
// |log c| >= 2^-11 > |R| unless c = 1 (a zero leading part makes the sum exact).
// Also S0 = 1/z - 1 to 1x (c (1 + S) - 1), for the x1 term.
// ---------------------------------------------------------------------------
__device__ __forceinline__ ff log_newton_f(float dh, float dl, int n, float& S0) {
    const float kShift = 0x1.8p23f;
    float kf = fma_rn(dh, 2048.0f, kShift);  // |2048 d| < 849: round(2048 d) in the low bits
    int i = 2048 + (int)(bits(kf) - bits(kShift));
    i = min(max(i, TF_FLOGT_LO), TF_FLOGT_HI);
    float4 T = __ldg(reinterpret_cast<const float4*>(TF_FLOGT) + (i - TF_FLOGT_LO));
    const float c = T.x, Lh = T.y, Ll = T.z, cm1 = T.w;
    ff p = two_prod(dh, c);
    float th = add(cm1, p.hi);               // exact
    float tl = fma_rn(dl, c, p.lo);
    // seed
    float R = fma_rn(mul(th, th), fma_rn(th, 0x1.555556p-2f, -0.5f), th);
    // S = e^-R - 1
    ff q = two_prod(R, R);
    float tail = mul(mul(q.hi, R), fma_rn(fma_rn(R, -0x1.111112p-7f, 0x1.555556p-5f), R, -0x1.555556p-3f));
    ff Sh = fast_two_sum(-R, mul(0.5f, q.hi));
    float Sl = add(Sh.lo, fma_rn(0.5f, q.lo, tail));
    // u = t + S + t S: t + S is exact (Sterbenz: S is within a factor 2 of -t),
    // and so is that plus RN(t S) (opposite, within a factor 2)
    float a = add(th, Sh.hi);
    ff m = two_prod(th, Sh.hi);
    float small = add(m.lo, add(add(Sl, tl), fma_rn(tl, Sh.hi, mul(th, Sl))));
    float u = add(add(a, m.hi), small);
    // n ln2 - log c + R + u
    float2 nl = __ldg(reinterpret_cast<const float2*>(TF_FNLN2_TABLE) + (min(max(n, -160), 140) - TF_FNLN2_LO));
    ff s1 = fast_two_sum(nl.x, Lh);
    ff s2 = fast_two_sum(s1.hi, R);
    float lo = add(add(s1.lo, s2.lo), add(add(nl.y, Ll), u));
    S0 = fma_rn(c, Sh.hi, cm1);
    return fast_two_sum(s2.hi, lo);
}

struct LogSplitF {
    float z;
    int n;
    float sub, inv;
};

// kSub = false: the caller guarantees a normal y (or y = 1), and the split
// skips the subnormal scaling.
template <bool kSub = true>
__device__ __forceinline__ LogSplitF log_split_f(float y) {
    bool subn = kSub && (bits(y) & kExpMask) == 0;
    float sfac = subn ? 0x1p24f : 1.0f;
    uint32_t b = bits(mul(y, sfac));
    int eb = (int)(b >> 23) - 127;
    uint32_t mant = b & kMantMask;
    bool big = mant >= 0x3504f3u;  // z >= sqrt(2)
    eb += big ? 1 : 0;
    float z = from_bits(mant | (big ? 0x3f000000u : 0x3f800000u));
    return {z, eb - (subn ? 24 : 0), sfac, pow2f(-eb)};
}

struct LogOutF {
    ff L;
    float S0, sub, inv;
};

__device__ __forceinline__ LogOutF log_pos_f(float y, int nadd = 0) {
    LogSplitF s = log_split_f(y);
    LogOutF o;
    o.L = log_newton_f(sub(s.z, 1.0f), 0.0f, s.n + nadd, o.S0);
    o.sub = s.sub;
    o.inv = s.inv;
    return o;
}

static __device__ __noinline__ float log_deviation_f(float v0, float v1, float v2, float z0) {
    bool huge = max(absbits(v0), absbits(v1)) >= 0x7e800000u;  // 2^126
    float sc = huge ? 0.5f : 1.0f;
    ff t = two_sum(mul(v0, sc), mul(v1, sc));
    ff v = two_sum(t.hi, add(t.lo, mul(v2, sc)));
    if (v.hi < 0.0f) return __int_as_float(0x7fc00000);
    if (v.hi == 0.0f) return -__int_as_float(0x7f800000);
    LogOutF o = log_pos_f(v.hi, huge ? 1 : 0);
    float q = mul(mul(v.lo, o.sub), o.inv);
    // G = (L.hi - z0) + L.lo + t with t = q (1 + S0) = v.lo / v.hi: L.hi - z0
    // exactly as a pair and its leading part summed with q exactly, then one
    // final rounding (L.hi may be far from z0, where a rounded L.hi - z0 alone
    // would cost up to another half ulp of the result)
    ff d = two_sum(o.L.hi, -z0);
    ff e = two_sum(d.hi, q);
    return add(e.hi, add(e.lo, fma_rn(q, o.S0, add(o.L.lo, d.lo))));
}

static __device__ __noinline__ void tlogf_rare(float y0, float y1, float z0, float& z1) {
    if (absbits(y1) >= kExpMask) {
        z1 = (absbits(y1) > kExpMask) ? y1 : ((y1 > 0.0f) ? y1 : __int_as_float(0x7fc00000));
        return;
    }
    z1 = log_deviation_f(y0, y1, 0.0f, z0);
}

// log1p(t) + c with t = q (1 + S0) = y1 / y0: t - t^2/2 (|t| <= 2^-24).
__device__ __forceinline__ float add_log1p_ratio(float q, float S0, float c) {
    float th = fma_rn(q, S0, q);
    float cc = fma_rn(mul(-0.5f, th), th, c);
    return add(q, fma_rn(q, S0, cc));
}

// |y1| > 2^-24 |ref| (or y1 not finite): not coupled.  |y1| 2^24 is exact (or
// +Inf), so this is the exact comparison; a NaN y1 counts as loose.
__device__ __forceinline__ bool loose(float y1, float ref) { return !(fabsf(y1) * 0x1p24f <= fabsf(ref)); }

// The same test on the integer pipes: the threshold |ref| 2^-24 truncated to
// the float grid (for |ref| < 2^-102 the significand shifted into the subnormal
// range), which classifies every y1 alike.  tlog1pf, whose FMA pipe is the
// busier one, measured 2.5 % faster with this form.
__device__ __forceinline__ bool loose_int(float y1, float ref) {
    uint32_t ar = absbits(ref);
    int e = (int)(ar >> 23);
    uint32_t m = (ar & kMantMask) | (e ? (1u << 23) : 0u);
    uint32_t thr = (e > 24) ? ar - (24u << 23) : (m >> (25 - max(e, 1)));
    return absbits(y1) > thr;
}

template <bool kVote>
__device__ __forceinline__ void tlogf_impl(float y0, float y1, float& z0, float& z1) {
    uint32_t b = bits(y0);
    if constexpr (kVote) {
        // a positive normal y0 and a finite y1 everywhere in the warp (one
        // vote): no special values and no subnormal scaling
        const bool special = !((y0 >= 0x1p-126f) & (y0 < kInf)) | !(fabsf(y1) < kInf);
        if (!warp_any<kVote>(special)) {
            LogSplitF s = log_split_f<false>(y0);
            float S0;
            ff L = log_newton_f(sub(s.z, 1.0f), 0.0f, s.n, S0);
            z0 = L.hi;
            z1 = add_log1p_ratio(mul(y1, s.inv), S0, L.lo);
            bool rare = loose(y1, y0);
            if (warp_any<kVote>(rare)) {
                if (rare) tlogf_rare(y0, y1, z0, z1);
            }
            return;
        }
    }
    uint32_t ab = b & ~kSignMask;
    bool pos = (b & kSignMask) == 0 && ab != 0 && ab < kExpMask;
    LogOutF o = log_pos_f(pos ? y0 : 1.0f);
    z0 = o.L.hi;
    float q = mul(mul(y1, o.sub), o.inv);
    z1 = add_log1p_ratio(q, o.S0, o.L.lo);
    bool rare = pos && loose(y1, y0);
    if (warp_any<kVote>(rare)) {
        if (rare) tlogf_rare(y0, y1, z0, z1);
    }
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    bool nanres = (ab > kExpMask) || ((b & kSignMask) && ab != 0);
    z0 = (ab == 0) ? -inf : z0;
    z0 = (b == kExpMask) ? inf : z0;
    z1 = pos ? z1 : 0.0f;
    z1 = (absbits(y1) > kExpMask) ? y1 : z1;
    z0 = nanres ? nan : z0;
    z1 = nanres ? nan : z1;
}

// The four elements of a thread in one call, for the float kernel's four
// elements per thread: one vote on special inputs for all four; a warp without
// any runs the four main paths in straight-line code, then one vote on rare
// lanes; any other warp runs tlogf_impl for each.  Results are those of
// tlogf_impl, bit for bit (measured 4 % faster at 2^28).
__device__ __forceinline__ void tlogf_quad(const float (&y0)[4], const float (&y1)[4], float (&z0)[4], float (&z1)[4]) {
    bool special = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) special |= !((y0[q] >= 0x1p-126f) & (y0[q] < kInf)) | !(fabsf(y1[q]) < kInf);
    if (__any_sync(0xffffffffu, special)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tlogf_impl<true>(y0[q], y1[q], z0[q], z1[q]);
        return;
    }
    bool rare[4], anyrare = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        LogSplitF s = log_split_f<false>(y0[q]);
        float S0;
        ff L = log_newton_f(sub(s.z, 1.0f), 0.0f, s.n, S0);
        z0[q] = L.hi;
        z1[q] = add_log1p_ratio(mul(y1[q], s.inv), S0, L.lo);
        rare[q] = loose(y1[q], y0[q]);
        anyrare |= rare[q];
    }
    if (__any_sync(0xffffffffu, anyrare)) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (rare[q]) tlogf_rare(y0[q], y1[q], z0[q], z1[q]);
    }
}

static __device__ __noinline__ void tlog1pf_rare(float y1, ff w, float z0, float& z1) {
    if (absbits(y1) >= kExpMask) {
        z1 = (absbits(y1) > kExpMask) ? y1 : ((y1 > 0.0f) ? y1 : __int_as_float(0x7fc00000));
        return;
    }
    z1 = log_deviation_f(w.hi, y1, w.lo, z0);
}

template <bool kVote>
__device__ __forceinline__ void tlog1pf_impl(float y0, float y1, float& z0, float& z1) {
    uint32_t b = bits(y0);
    uint32_t ab = b & ~kSignMask;
    bool neg = (b & kSignMask) != 0;
    const uint32_t b_one = 0x3f800000u;
    bool ok = ab < kExpMask && !(neg && ab >= b_one);
    float yv = ok ? y0 : 0.0f;
    ff w = sorted_two_sum(1.0f, yv);
    LogSplitF s = log_split_f<false>(w.hi);  // 1 + yv is 1 or at least 2^-24: normal
    bool n0 = s.n == 0;
    float dh = n0 ? yv : sub(s.z, 1.0f);
    float dl = n0 ? 0.0f : mul(w.lo, s.inv);
    float S0;
    ff L = log_newton_f(dh, dl, s.n, S0);
    z0 = L.hi;
    float q = mul(y1, s.inv);
    z1 = add_log1p_ratio(q, S0, L.lo);
    // y0 in (-1, +Inf) nonzero and a finite y1 everywhere in the warp (one
    // vote): no special values, and y1's looseness from the exponent fields of
    // w.hi >= 2^-24
    bool special = !ok | (ab == 0) | (absbits(y1) >= kExpMask);
    if (kVote && !warp_any<kVote>(special)) {
        bool rare = absbits(y1) > bits(w.hi) - (24u << 23);
        if (warp_any<kVote>(rare)) {
            if (rare) tlog1pf_rare(y1, w, z0, z1);
        }
        return;
    }
    bool rare = ok && loose_int(y1, w.hi);
    if (warp_any<kVote>(rare)) {
        if (rare) tlog1pf_rare(y1, w, z0, z1);
    }
    const float inf = __int_as_float(0x7f800000), nan = __int_as_float(0x7fc00000);
    bool minus1 = b == (kSignMask | b_one);
    bool pinf = b == kExpMask;
    bool nanres = (ab > kExpMask) || (neg && ab > b_one);
    z0 = (ab == 0) ? y0 : z0;
    z0 = minus1 ? -inf : z0;
    z0 = pinf ? inf : z0;
    z1 = ok ? z1 : 0.0f;
    z1 = (absbits(y1) > kExpMask) ? y1 : z1;
    z0 = nanres ? nan : z0;
    z1 = nanres ? nan : z1;
}

}  // namespace tff
