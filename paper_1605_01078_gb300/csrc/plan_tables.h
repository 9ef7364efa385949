// Coefficient tables of the general operation (Eq. 1, Eq. 3, Eq. 4), built at compile
// time so that host code and device constant memory hold the same table.
//
// One level is Figure 1 (Section 3.1).  L levels is its L-th Kronecker power
// (Sections 3.5-3.6): product r = 7a + b of level L applies product a of level L - 1
// (outer) to product b of Figure 1 (inner); along each dimension the block index is
// 2 * outer + inner and signs multiply.  Figure 2 prints the two-level table with the
// C-update signs; its operand signs are printed as "+" throughout and are not used.
// Level 0 is the single classical product C00 += A00 B00.  Three levels (343 products
// with up to 8 terms per operand and 8 C targets) is the deepest table built.
#pragma once

#include <stdint.h>

namespace sgb {

// One term of a product: block (bi, bj) of the 2^L x 2^L partition with a sign.
// Encoded in one byte: bits 0-2 block column, bits 3-5 block row, bit 7 negative.
__host__ __device__ constexpr uint8_t term_code(int bi, int bj, int neg) {
  return (uint8_t)((bj & 7) | ((bi & 7) << 3) | (neg ? 0x80 : 0));
}
__host__ __device__ constexpr int term_bj(uint8_t c) { return c & 7; }
__host__ __device__ constexpr int term_bi(uint8_t c) { return (c >> 3) & 7; }
__host__ __device__ constexpr int term_neg(uint8_t c) { return (c >> 7) & 1; }

constexpr int kMaxLevels = 3;
constexpr int kMaxTerms = 1 << kMaxLevels;
constexpr int kTableRows = 1 + 7 + 49 + 343;
constexpr int kPlanOffset[kMaxLevels + 1] = {0, 1, 8, 57};
constexpr int kPlanCount[kMaxLevels + 1] = {1, 7, 49, 343};

struct PlanTables {
  uint8_t na[kTableRows], nb[kTableRows], nc[kTableRows];
  uint8_t ta[kTableRows][kMaxTerms], tb[kTableRows][kMaxTerms], tc[kTableRows][kMaxTerms];
};

namespace detail {

struct T1 { int bi, bj, s; };
struct Row1 { int na; T1 a[2]; int nb; T1 b[2]; int nc; T1 c[2]; };

// Figure 1:
//   M0 = (A00 + A11)(B00 + B11);  C00 += M0;  C11 += M0
//   M1 = (A10 + A11) B00;         C10 += M1;  C11 -= M1
//   M2 = A00 (B01 - B11);         C01 += M2;  C11 += M2
//   M3 = A11 (B10 - B00);         C00 += M3;  C10 += M3
//   M4 = (A00 + A01) B11;         C01 += M4;  C00 -= M4
//   M5 = (A10 - A00)(B00 + B01);  C11 += M5
//   M6 = (A01 - A11)(B10 + B11);  C00 += M6
constexpr Row1 kOneLevel[7] = {
    {2, {{0, 0, 1}, {1, 1, 1}}, 2, {{0, 0, 1}, {1, 1, 1}}, 2, {{0, 0, 1}, {1, 1, 1}}},
    {2, {{1, 0, 1}, {1, 1, 1}}, 1, {{0, 0, 1}, {0, 0, 0}}, 2, {{1, 0, 1}, {1, 1, -1}}},
    {1, {{0, 0, 1}, {0, 0, 0}}, 2, {{0, 1, 1}, {1, 1, -1}}, 2, {{0, 1, 1}, {1, 1, 1}}},
    {1, {{1, 1, 1}, {0, 0, 0}}, 2, {{1, 0, 1}, {0, 0, -1}}, 2, {{0, 0, 1}, {1, 0, 1}}},
    {2, {{0, 0, 1}, {0, 1, 1}}, 1, {{1, 1, 1}, {0, 0, 0}}, 2, {{0, 1, 1}, {0, 0, -1}}},
    {2, {{1, 0, 1}, {0, 0, -1}}, 2, {{0, 0, 1}, {0, 1, 1}}, 1, {{1, 1, 1}, {0, 0, 0}}},
    {2, {{0, 1, 1}, {1, 1, -1}}, 2, {{1, 0, 1}, {1, 1, 1}}, 1, {{0, 0, 1}, {0, 0, 0}}},
};

// Kronecker product of an outer term list with an inner one (block 2*outer + inner).
constexpr int kron(const uint8_t* outer, int no, const T1* inner, int ni, uint8_t* out) {
  int n = 0;
  for (int i = 0; i < no; ++i)
    for (int j = 0; j < ni; ++j) {
      const int bi = 2 * term_bi(outer[i]) + inner[j].bi;
      const int bj = 2 * term_bj(outer[i]) + inner[j].bj;
      const int neg = term_neg(outer[i]) ^ (inner[j].s < 0 ? 1 : 0);
      out[n++] = term_code(bi, bj, neg);
    }
  return n;
}

constexpr PlanTables build_tables() {
  PlanTables t{};
  t.na[0] = t.nb[0] = t.nc[0] = 1;
  t.ta[0][0] = t.tb[0][0] = t.tc[0][0] = term_code(0, 0, 0);
  for (int L = 1; L <= kMaxLevels; ++L) {
    const int po = kPlanOffset[L - 1], pc = kPlanCount[L - 1], off = kPlanOffset[L];
    for (int a = 0; a < pc; ++a)
      for (int b = 0; b < 7; ++b) {
        const int r = off + 7 * a + b;
        const Row1& in = kOneLevel[b];
        t.na[r] = (uint8_t)kron(t.ta[po + a], t.na[po + a], in.a, in.na, t.ta[r]);
        t.nb[r] = (uint8_t)kron(t.tb[po + a], t.nb[po + a], in.b, in.nb, t.tb[r]);
        t.nc[r] = (uint8_t)kron(t.tc[po + a], t.nc[po + a], in.c, in.nc, t.tc[r]);
      }
  }
  return t;
}

}  // namespace detail

constexpr PlanTables kPlanTables = detail::build_tables();

}  // namespace sgb
