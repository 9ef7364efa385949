// Coefficient tables of the general operation (Eq. 1, Eq. 3, Eq. 4).
//
// One level is Figure 1 (Section 3.1).  Two levels is its Kronecker square (Section
// 3.5): product r = 7a + b applies outer product a to inner product b; along each
// dimension the block index is 2 * outer + inner and signs multiply.  Figure 2 prints
// this table with the C-update signs; its operand signs are printed as "+" throughout
// and are not used.  Level 0 is the single classical product C00 += A00 B00.
#include <cstring>

#include "internal.h"

namespace sgb {
namespace {

struct T { int bi, bj, s; };
struct Row { int na; T a[2]; int nb; T b[2]; int nc; T c[2]; };

// Figure 1:
//   M0 = (A00 + A11)(B00 + B11);  C00 += M0;  C11 += M0
//   M1 = (A10 + A11) B00;         C10 += M1;  C11 -= M1
//   M2 = A00 (B01 - B11);         C01 += M2;  C11 += M2
//   M3 = A11 (B10 - B00);         C00 += M3;  C10 += M3
//   M4 = (A00 + A01) B11;         C01 += M4;  C00 -= M4
//   M5 = (A10 - A00)(B00 + B01);  C11 += M5
//   M6 = (A01 - A11)(B10 + B11);  C00 += M6
const Row kOneLevel[7] = {
    {2, {{0, 0, 1}, {1, 1, 1}}, 2, {{0, 0, 1}, {1, 1, 1}}, 2, {{0, 0, 1}, {1, 1, 1}}},
    {2, {{1, 0, 1}, {1, 1, 1}}, 1, {{0, 0, 1}, {0, 0, 0}}, 2, {{1, 0, 1}, {1, 1, -1}}},
    {1, {{0, 0, 1}, {0, 0, 0}}, 2, {{0, 1, 1}, {1, 1, -1}}, 2, {{0, 1, 1}, {1, 1, 1}}},
    {1, {{1, 1, 1}, {0, 0, 0}}, 2, {{1, 0, 1}, {0, 0, -1}}, 2, {{0, 0, 1}, {1, 0, 1}}},
    {2, {{0, 0, 1}, {0, 1, 1}}, 1, {{1, 1, 1}, {0, 0, 0}}, 2, {{0, 1, 1}, {0, 0, -1}}},
    {2, {{1, 0, 1}, {0, 0, -1}}, 2, {{0, 0, 1}, {0, 1, 1}}, 1, {{1, 1, 1}, {0, 0, 0}}},
    {2, {{0, 1, 1}, {1, 1, -1}}, 2, {{1, 0, 1}, {1, 1, 1}}, 1, {{0, 0, 1}, {0, 0, 0}}},
};

// Kronecker product of two term lists: (outer, inner) -> block 2*outer + inner.
int kron(const uint8_t* outer, int no, const T* inner, int ni, uint8_t* out) {
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

}  // namespace

bool make_plan(int levels, Plan* p) {
  if (levels < 0 || levels > 2 || !p) return false;
  std::memset(p, 0, sizeof(*p));
  p->levels = levels;
  // Level 0: C00 += A00 B00.
  p->nprod = 1;
  p->na[0] = p->nb[0] = p->nc[0] = 1;
  p->ta[0][0] = p->tb[0][0] = p->tc[0][0] = term_code(0, 0, 0);
  for (int l = 0; l < levels; ++l) {
    Plan q;
    std::memset(&q, 0, sizeof(q));
    q.levels = l + 1;
    q.nprod = p->nprod * 7;
    for (int a = 0; a < p->nprod; ++a)
      for (int b = 0; b < 7; ++b) {
        const int r = 7 * a + b;
        const Row& in = kOneLevel[b];
        q.na[r] = (uint8_t)kron(p->ta[a], p->na[a], in.a, in.na, q.ta[r]);
        q.nb[r] = (uint8_t)kron(p->tb[a], p->nb[a], in.b, in.nb, q.tb[r]);
        q.nc[r] = (uint8_t)kron(p->tc[a], p->nc[a], in.c, in.nc, q.tc[r]);
      }
    *p = q;
  }
  return true;
}

}  // namespace sgb
