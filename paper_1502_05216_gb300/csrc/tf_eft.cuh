// tf_eft.cuh -- error-free transforms in binary64 for the twofold kernels.
//
// Every operation goes through an explicit round-to-nearest intrinsic
// (__dadd_rn, __dmul_rn, __fma_rn) so that no compiler contraction or
// reassociation can change the rounding the transforms rely on (the paper's
// "Compiler flags" section asks for the same protection on the CPU).
#pragma once

#include <cstdint>

namespace tf {

struct tf2 {
    double hi, lo;
};

__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ uint64_t bits(double a) { return (uint64_t)__double_as_longlong(a); }
__device__ __forceinline__ double from_bits(uint64_t b) { return __longlong_as_double((long long)b); }
// Magnitude bits of a double.  The inline PTX keeps comparisons of these bits
// on the integer ALU: the compiler may otherwise turn a compare of two
// magnitude bit patterns into an FP64 compare, which occupies the FP64 pipe
// (tadd, FP64-bound, ran at half speed that way).
__device__ __forceinline__ uint64_t absbits(double a) {
    uint64_t r;
    asm("and.b64 %0, %1, 0x7fffffffffffffff;" : "=l"(r) : "l"(bits(a)));
    return r;
}
// The plain form, which leaves the choice of compare to the compiler (used
// where the integer ALU, not the FP64 pipe, is the busier unit).
__device__ __forceinline__ uint64_t absbits_any(double a) { return bits(a) & 0x7fffffffffffffffull; }

// Fast2Sum (Dekker): s + e == a + b exactly when a == 0 or exponent(a) >= exponent(b).
// Three additions; the paper uses it for the "fast renormalization" (Twofold
// exponent > Algorithm summary) and whenever the larger operand is known.
__device__ __forceinline__ tf2 fast_two_sum(double a, double b) {
    double s = add(a, b);
    return {s, sub(b, sub(s, a))};
}

// TwoSum for arbitrary a, b (the paper's corrected Algorithm 2.2, "Twofolds
// update" > "Twofold bugs", written for a sum): six additions.
__device__ __forceinline__ tf2 two_sum(double a, double b) {
    double s = add(a, b);
    double bp = sub(s, a);
    double ap = sub(s, bp);
    return {s, add(sub(a, ap), sub(b, bp))};
}

// Fast2Sum after ordering the operands by magnitude with integer compares and
// selects: three FP64 additions, the ordering costs no FP64 instruction.
__device__ __forceinline__ tf2 sorted_two_sum(double a, double b) {
    bool sw = absbits(b) > absbits(a);
    double big = sw ? b : a;
    double sml = sw ? a : b;
    return fast_two_sum(big, sml);
}

// 2^k as a double for any int k: 0 below 2^-1074, +Inf above 2^1023, built from bits.
__device__ __forceinline__ double pow2i(int k) {
    uint64_t normal = (uint64_t)(int64_t)(k + 1023) << 52;
    uint64_t subn = (k >= -1074) ? (1ull << ((k + 1074) & 63)) : 0ull;
    uint64_t b = (k >= -1022) ? normal : subn;
    b = (k > 1023) ? 0x7ff0000000000000ull : b;
    return from_bits(b);
}

}  // namespace tf
