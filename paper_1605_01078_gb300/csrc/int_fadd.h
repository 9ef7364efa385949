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

// The bits of a + b (b's sign bit already flipped for a subtraction), rounded to
// nearest even; operands and result are binary64 bit patterns, so no value of floating
// type (and no floating-point instruction) appears in the computation.  Written without
// data-dependent branches (the add and subtract cases, the alignment shift, the
// normalisation and the special operands are all selects), so the lanes of a warp stay
// converged and the compiler can interleave independent additions.
__host__ __device__ __forceinline__ uint64_t int_fadd_bits(uint64_t ua, uint64_t ub) {
  const uint64_t kExpMask = 0x7ff0000000000000ULL, kMag = 0x7fffffffffffffffULL;
  const uint64_t kFrac = (1ULL << 52) - 1, kHidden = 1ULL << 52, kQNaN = 0x7ff8000000000000ULL;
  const uint64_t am = ua & kMag, bm = ub & kMag;
  const bool sub = ((ua ^ ub) >> 63) != 0;
  // x: the operand of larger magnitude (it gives the sign), y: the other.
  const bool swap = bm > am;
  const uint64_t x = swap ? ub : ua;
  const uint64_t xm = swap ? bm : am, ym = swap ? am : bm;
  const int ex_f = (int)(xm >> 52), ey_f = (int)(ym >> 52);
  // Significands with the hidden bit (none for subnormals and zeros, whose exponent
  // reads as 1), scaled by 8 for the guard, round and sticky bits.
  const uint64_t mx = ((xm & kFrac) | (ex_f ? kHidden : 0)) << 3;
  uint64_t my = ((ym & kFrac) | (ey_f ? kHidden : 0)) << 3;
  const int ex = ex_f + (ex_f == 0), ey = ey_f + (ey_f == 0);
  // Align y to x's exponent, OR-ing every bit shifted out into bit 0 (my < 2^56, so
  // any shift of 63 or more leaves only the sticky bit).
  const int d = (ex - ey) < 63 ? (ex - ey) : 63;
  my = (my >> d) | ((my & ((1ULL << d) - 1)) != 0 ? 1 : 0);
  uint64_t s = sub ? mx - my : mx + my;  // >= 0 since |x| >= |y|
  const bool zero = s == 0;
  // Normalise so the leading one sits at bit 55: one right shift (with sticky) after a
  // carry out of an addition, else a left shift after cancellation, never below the
  // subnormal exponent 1.
  const bool carry = (s >> 56) != 0;
  const int lz = ifa_clz64(s) - 8;
  const int sh = carry ? 0 : (lz < ex - 1 ? lz : ex - 1);
  s = carry ? ((s >> 1) | (s & 1)) : (s << sh);
  const int e = carry ? ex + 1 : ex - sh;
  // Round to nearest even on the three extra bits.
  const uint64_t low = s & 7;
  uint64_t sig = s >> 3;
  sig += (low > 4 || (low == 4 && (sig & 1))) ? 1 : 0;
  // Pack: (e - 1) << 52 plus the significand with its hidden bit gives the exponent
  // field e for a normal result, 0 for a subnormal (no hidden bit, e == 1), and carries
  // a rounding overflow (sig == 2^53) into the next binade.  Anything at or above the
  // infinity pattern overflowed.
  uint64_t r = ((uint64_t)(e - 1) << 52) + sig;
  r = (x & 0x8000000000000000ULL) | (r >= kExpMask ? kExpMask : r);
  // A zero sum: +0 from exact cancellation, or (+-0) + (+-0) = +0 unless both are -0.
  r = zero ? (xm == 0 ? (ua & ub) : 0) : r;
  // Infinities and NaNs (IEEE addition): NaN in -> quiet NaN; inf + (-inf) -> NaN;
  // otherwise the infinity.
  const bool nan_in = am > kExpMask || bm > kExpMask;
  const bool inf_a = am == kExpMask, inf_b = bm == kExpMask;
  const uint64_t special = (nan_in || (inf_a && inf_b && sub)) ? kQNaN : (inf_a ? ua : ub);
  return (am >= kExpMask || bm >= kExpMask) ? special : r;
}

// a + b, or a - b when `negate_b`, rounded to nearest even.
__host__ __device__ __forceinline__ double int_fadd(double a, double b, bool negate_b) {
  return ifa_double(int_fadd_bits(ifa_bits(a), ifa_bits(b) ^ (negate_b ? 0x8000000000000000ULL : 0)));
}

}  // namespace sgb
