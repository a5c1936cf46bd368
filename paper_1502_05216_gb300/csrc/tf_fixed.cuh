// tf_fixed.cuh -- 128-bit fixed-point arithmetic on the integer pipes.
//
// On a GB300 the FP64 pipe issues 2 thread-instructions per SM per cycle while
// the integer multiply-add (IMAD.WIDE.U32, 32 x 32 -> 64 bits) issues ~64, so
// the long Taylor evaluation of the exp core (paper, "Twofold exponent" >
// "Method summary": a Horner scheme carried to 2x precision) runs here in
// unsigned 128-bit fixed point, and only the argument reduction, the 2^k
// rescale and the twofold corrections stay in FP64.
//
// Every routine is exact integer arithmetic; truncations are stated where they
// happen.  A value v held "in units 2^-u" is the integer round_down(v 2^u).
#pragma once

#include <cstdint>

namespace tf {

struct u128 {
    uint64_t lo, hi;
};

// The arithmetic goes through the compiler's unsigned __int128, which keeps the
// carry chains of 128-bit sums in fused three-input integer adds (measured:
// 11-14 % faster kernels than explicit add.cc/addc pairs, identical results).
typedef unsigned __int128 v128;
__device__ __forceinline__ v128 V(u128 a) { return ((v128)a.hi << 64) | a.lo; }
__device__ __forceinline__ u128 U(v128 v) { return {(uint64_t)v, (uint64_t)(v >> 64)}; }

// Full 64 x 64 -> 128-bit product.
__device__ __forceinline__ u128 mul_full(uint64_t a, uint64_t b) { return U((v128)a * b); }

__device__ __forceinline__ uint64_t mul_hi(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

__device__ __forceinline__ u128 add128(u128 a, u128 b) { return U(V(a) + V(b)); }

__device__ __forceinline__ u128 sub128(u128 a, u128 b) { return U(V(a) - V(b)); }

// Two's complement negation.
__device__ __forceinline__ u128 neg128(u128 a) { return U(0 - V(a)); }

__device__ __forceinline__ bool is_neg128(u128 a) { return (int64_t)a.hi < 0; }

// c + t or c - t by the sign flag.
__device__ __forceinline__ u128 addsub128(u128 c, u128 t, bool minus) {
    return minus ? sub128(c, t) : add128(c, t);
}

// Logical shift right by a compile-time 0 <= s < 64.
template <int s>
__device__ __forceinline__ u128 shr128(u128 a) {
    if constexpr (s == 0) {
        return a;
    } else {
        return U(V(a) >> s);
    }
}

// Logical shift left by a compile-time 0 < s < 64.
template <int s>
__device__ __forceinline__ u128 shl128(u128 a) {
    return U(V(a) << s);
}

// Logical shift right by a run-time 0 <= s < 64.
__device__ __forceinline__ u128 shr128_var(u128 a, int s) {
    uint64_t carry = (a.hi << 1) << (63 - s);  // a.hi << (64 - s), 0 for s == 0
    return {(a.lo >> s) | carry, a.hi >> s};
}

// Logical shift left by a run-time 0 <= s <= 127.
__device__ __forceinline__ u128 shl128_var(u128 a, int s) {
    if (s >= 64) return {0ull, a.lo << (s - 64)};
    uint64_t carry = (a.lo >> 1) >> (63 - s);  // a.lo >> (64 - s), 0 for s == 0
    return {a.lo << s, (a.hi << s) | carry};
}

// Logical shift right by any run-time s >= 0 (0 from s >= 128).
__device__ __forceinline__ u128 shr128_any(u128 a, int s) {
    int s1 = min(s, 63);
    int s2 = min(max(s - 64, 0), 63);
    uint64_t lo = (s < 64) ? ((a.lo >> s1) | ((a.hi << 1) << (63 - s1))) : ((s < 128) ? (a.hi >> s2) : 0ull);
    uint64_t hi = (s < 64) ? (a.hi >> s1) : 0ull;
    return {lo, hi};
}

// Arithmetic (sign-extending) shift right of a two's complement value by a
// compile-time 0 < s < 64.
template <int s>
__device__ __forceinline__ u128 sar128(u128 a) {
    return U((v128)((__int128)V(a) >> s));
}

// a * b for a < 2^64 and a 32-bit b.
__device__ __forceinline__ u128 mul_u64_u32(uint64_t a, uint32_t b) { return U((v128)a * b); }

// A 53-bit (or shorter) integer m shifted by s bits, left for s >= 0 and right
// (truncating) for s < 0; s <= 74 keeps the result below 2^127.
__device__ __forceinline__ u128 place53(uint64_t m, int s) {
    uint64_t lo = (s >= 0) ? ((s < 64) ? (m << s) : 0ull) : ((s > -64) ? (m >> -s) : 0ull);
    uint64_t hi = (s >= 64) ? (m << (s - 64)) : ((s > 0) ? ((m >> 1) >> (63 - s)) : 0ull);
    return {lo, hi};
}

// (a * b) >> (128 + s) for a, b < 2^128, 0 <= s < 64, from the three leading
// partial products: the dropped low product a.lo * b.lo and the low halves of
// the cross products make the result at most 3 units too small.  The caller
// keeps a.hi * b.hi below 2^127 so that the sum cannot overflow.
template <int s>
__device__ __forceinline__ u128 mulshift(u128 a, u128 b) {
    v128 p = (v128)a.hi * b.hi;
    p += __umul64hi(a.hi, b.lo);
    p += __umul64hi(a.lo, b.hi);
    return U(p >> s);
}

// a * n for a < 2^128 and a 32-bit n whose product stays below 2^128.
__device__ __forceinline__ u128 mul128_u32(u128 a, uint32_t n) { return U(V(a) * n); }

// (a * n) >> s for a < 2^128, a 32-bit n and 0 < s < 64, from the full
// 160-bit product; the caller keeps the result below 2^128.
template <int s>
__device__ __forceinline__ u128 mul128_u32_shr(u128 a, uint32_t n) {
    // (a.lo n + a.hi n 2^64) >> s = (a.lo n >> s) + a.hi n 2^(64 - s), modulo 2^128
    return U((((v128)a.lo * n) >> s) + (((v128)a.hi * n) << (64 - s)));
}

// High 64 bits of the signed product of a signed a and a non-negative b < 2^63
// (one sign correction: for a < 0 the unsigned product is a b + 2^64 b).
__device__ __forceinline__ int64_t mul_hi_su(int64_t a, uint64_t b) {
    return (int64_t)(__umul64hi((uint64_t)a, b) - ((a < 0) ? b : 0ull));
}

// The top 128 bits of the 181-bit product m * b (m < 2^53): (m b) >> 64.
__device__ __forceinline__ u128 mul53_top(uint64_t m, u128 b) {
    return U((v128)m * b.hi + __umul64hi(m, b.lo));
}

// ---------------------------------------------------------------------------
// Fixed point -> twofold.  hi + lo = (-1)^neg M 2^E with hi = RN(M 2^E) (ties
// to even) and lo = RN of the remainder, which is kept to 64 bits: |hi + lo -
// M 2^E| <= 2^-115 |hi|.  M == 0 gives (+-0, 0).  The caller guarantees that
// both parts are normal doubles (2^-960 <= M 2^E < 2^1023).
// ---------------------------------------------------------------------------
template <bool kHi = false>
__device__ __forceinline__ void to_pair(u128 M, int E, bool neg, double& hi, double& lo) {
    const uint64_t sgn = neg ? 0x8000000000000000ull : 0ull;
    bool zero = (M.hi | M.lo) == 0;
    int lz;
    u128 Mn;
    if constexpr (kHi) {  // the caller guarantees M.hi != 0: a one-word count and shift
        lz = min(__clzll((long long)M.hi), 63);
        Mn = {M.lo << lz, (M.hi << lz) | ((M.lo >> 1) >> (63 - lz))};
    } else {
        lz = (M.hi != 0) ? __clzll((long long)M.hi) : 64 + __clzll((long long)(M.lo | 1ull));
        Mn = shl128_var(M, lz);  // bit 127 set
    }
    int L = 127 - lz;              // position of the leading bit of M
    uint64_t m53 = Mn.hi >> 11;
    bool rb = (Mn.hi >> 10) & 1;
    bool st = ((Mn.hi & 0x3ffull) | Mn.lo) != 0;
    bool up = rb && (st || (m53 & 1));
    int be = E + L + 1023;  // biased exponent of the leading bit
    uint64_t hib = ((uint64_t)(int64_t)(be - 1) << 52) + m53 + (up ? 1ull : 0ull);
    // remainder: bits 74 .. 11 of Mn, weight of bit 11 = 2^(E + L - 116); rounding
    // up leaves W - 2^64 (W >= 2^63 then), which is -(2^64 - W)
    uint64_t W = (Mn.hi << 53) | (Mn.lo >> 11);
    uint64_t mag = up ? (0ull - W) : W;
    uint64_t lsg = up ? (sgn ^ 0x8000000000000000ull) : sgn;
    int lz2 = __clzll((long long)(mag | 1ull));
    uint64_t mn = mag << lz2;
    uint64_t lm53 = mn >> 11;
    bool lrb = (mn >> 10) & 1;
    bool lst = (mn & 0x3ffull) != 0;
    bool lup = lrb && (lst || (lm53 & 1));
    int lbe = E + L - 116 + (63 - lz2) + 1023;
    uint64_t lob = ((uint64_t)(int64_t)(lbe - 1) << 52) + lm53 + (lup ? 1ull : 0ull);
    hi = __longlong_as_double((long long)((zero ? 0ull : hib) | sgn));
    lo = __longlong_as_double((long long)((mag == 0 || zero) ? 0ull : (lob | lsg)));
}

}  // namespace tf
