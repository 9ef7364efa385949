// Host copies of the coefficient tables (built at compile time in plan_tables.h).
#include <cstring>

#include "internal.h"

namespace sgb {

bool make_plan(int levels, Plan* p) {
  if (levels < 0 || levels > kMaxLevels || !p) return false;
  std::memset(p, 0, sizeof(*p));
  p->levels = levels;
  p->nprod = kPlanCount[levels];
  const int off = kPlanOffset[levels];
  for (int r = 0; r < p->nprod; ++r) {
    p->na[r] = kPlanTables.na[off + r];
    p->nb[r] = kPlanTables.nb[off + r];
    p->nc[r] = kPlanTables.nc[off + r];
    for (int t = 0; t < kMaxTerms; ++t) {
      p->ta[r][t] = kPlanTables.ta[off + r][t];
      p->tb[r][t] = kPlanTables.tb[off + r][t];
      p->tc[r][t] = kPlanTables.tc[off + r][t];
    }
  }
  return true;
}

Fp64Launch make_launch(int64_t m, int64_t n, int64_t k, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, int levels) {
  Fp64Launch L;
  std::memset(&L, 0, sizeof(L));
  L.A = A; L.B = B; L.C = C;
  L.lda = lda; L.ldb = ldb; L.ldc = ldc;
  L.a_rows = m; L.a_cols = k;
  L.b_rows = k; L.b_cols = n;
  L.c_rows = m; L.c_cols = n;
  L.hm = block_edge(m, levels); L.hn = block_edge(n, levels); L.hk = block_edge(k, levels);
  L.levels = levels;
  L.prod_begin = 0;
  L.nprod = -1;
  L.m_target = 0;
  L.epi = kEpiAtomicAdd;
  L.sched = kSchedStreamK;
  L.tile = -1;  // chosen by choose_fp64_schedule / launch_fp64
  L.trans_a = 0;
  L.trans_b = 0;
  L.alpha = 1.0;
  return L;
}

}  // namespace sgb
