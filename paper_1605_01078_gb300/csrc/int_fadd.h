// IEEE 754 binary64 addition with round-to-nearest-even computed with integer
// operations only.
//
// On GB300 the FP64 pipe delivers about 2 lanes per clock per SM while the integer
// pipes are tens of times wider, so the operand sums of the Strassen staging (one
// addition per source tile element) are formed here instead of with DADD: the FP64
// pipe is left to the product's fused multiply-adds.  The result is bit-identical to
// the hardware addition for every pair of finite or infinite inputs (NaN inputs give
// a quiet NaN).  The algorithm is the textbook one: align the significands with three
// extra bits (guard, round, sticky), add or subtract the magnitudes, normalise, round to
// nearest even, and handle subnormal and overflowing results.
#pragma once

#include <stdint.h>

namespace sgb {

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ int ifa_clz64(uint64_t x) { return __clzll((long long)x); }
__device__ __forceinline__ uint64_t ifa_bits(double x) { return (uint64_t)__double_as_longlong(x); }
__device__ __forceinline__ double ifa_double(uint64_t b) { return __longlong_as_double((long long)b); }
#else
inline int ifa_clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }
inline uint64_t ifa_bits(double x) {
  uint64_t b;
  __builtin_memcpy(&b, &x, 8);
  return b;
}
inline double ifa_double(uint64_t b) {
  double x;
  __builtin_memcpy(&x, &b, 8);
  return x;
}
#endif

// Shift right by n (0 <= n), OR-ing every bit shifted out into bit 0 ("jamming").
__host__ __device__ __forceinline__ uint64_t ifa_shr_jam(uint64_t x, int n) {
  if (n == 0) return x;
  if (n >= 64) return x != 0 ? 1 : 0;
  return (x >> n) | ((x << (64 - n)) != 0 ? 1 : 0);
}

// Round s (value s * 2^(e - 1078): three extra low bits; the leading one at bit 55 for a
// normal result, below it only when e == 1, i.e. a subnormal result) to nearest even
// and pack it with `sign`.
__host__ __device__ __forceinline__ uint64_t ifa_round_pack(uint64_t sign, int e, uint64_t s) {
  const uint64_t low = s & 7;
  uint64_t sig = s >> 3;
  if (low > 4 || (low == 4 && (sig & 1))) sig += 1;
  if (sig >> 53) {  // rounding carried into a new binade
    sig >>= 1;
    e += 1;
  }
  if (e >= 2047) return sign | 0x7ff0000000000000ULL;  // overflow to infinity
  if (sig < (1ULL << 52)) return sign | sig;             // subnormal: exponent field 0
  return sign | ((uint64_t)e << 52) | (sig & ((1ULL << 52) - 1));
}

// The bits of a + b (b's sign bit already flipped for a subtraction), rounded to
// nearest even; operands and result are binary64 bit patterns, so no value of floating
// type (and no floating-point instruction) appears in the computation.
__host__ __device__ __forceinline__ uint64_t int_fadd_bits(uint64_t ua, uint64_t ub) {
  const uint64_t kExpMask = 0x7ff0000000000000ULL, kMag = 0x7fffffffffffffffULL;
  // Infinities and NaNs: rare; follow the definition of IEEE addition.
  if ((ua & kExpMask) == kExpMask || (ub & kExpMask) == kExpMask) {
    const bool nan_a = (ua & kMag) > kExpMask, nan_b = (ub & kMag) > kExpMask;
    if (nan_a || nan_b) return 0x7ff8000000000000ULL;
    const bool inf_a = (ua & kMag) == kExpMask, inf_b = (ub & kMag) == kExpMask;
    if (inf_a && inf_b) return ((ua ^ ub) >> 63) ? 0x7ff8000000000000ULL : ua;
    return inf_a ? ua : ub;
  }
  // Zeros: x + 0 = x; (+0) + (-0) = +0 and (-0) + (-0) = -0 under round to nearest.
  if ((ub & kMag) == 0) return (ua & kMag) == 0 ? (ua & ub) : ua;
  if ((ua & kMag) == 0) return ub;
  // Order by magnitude: |a| >= |b|.
  if ((ub & kMag) > (ua & kMag)) {
    const uint64_t t = ua;
    ua = ub;
    ub = t;
  }
  const uint64_t sign = ua & 0x8000000000000000ULL;
  int ea = (int)((ua >> 52) & 0x7ff), eb = (int)((ub >> 52) & 0x7ff);
  uint64_t ma = ua & ((1ULL << 52) - 1), mb = ub & ((1ULL << 52) - 1);
  if (ea) ma |= 1ULL << 52; else ea = 1;  // subnormals: no hidden bit, exponent 1
  if (eb) mb |= 1ULL << 52; else eb = 1;
  ma <<= 3;  // guard, round and sticky bits
  mb = ifa_shr_jam(mb << 3, ea - eb);
  uint64_t s;
  int e = ea;
  if (((ua ^ ub) >> 63) == 0) {
    s = ma + mb;
    if (s >> 56) {  // carry out of the 53 + 3 bit field
      s = ifa_shr_jam(s, 1);
      e += 1;
    }
  } else {
    s = ma - mb;                       // >= 0 since |a| >= |b|
    if (s == 0) return 0;  // exact cancellation gives +0
    const int lz = ifa_clz64(s) - 8;   // the leading one belongs at bit 55
    if (lz > 0) {
      const int shift = lz < e - 1 ? lz : e - 1;  // never below the subnormal exponent
      s <<= shift;
      e -= shift;
    }
  }
  return ifa_round_pack(sign, e, s);
}

// a + b, or a - b when `negate_b`, rounded to nearest even.
__host__ __device__ __forceinline__ double int_fadd(double a, double b, bool negate_b) {
  return ifa_double(int_fadd_bits(ifa_bits(a), ifa_bits(b) ^ (negate_b ? 0x8000000000000000ULL : 0)));
}

}  // namespace sgb
