/* A plain C client of include/strassen.h: compiles as C99 against the header and links
 * the library.  Without a GPU it exercises the calls that do no device work: the
 * coefficient tables, status strings, argument checks, workspace sizes, the analytic
 * model and the selector's model choice.  Prints "abi client ok" on success. */
#include <stdio.h>
#include <string.h>

#include "strassen.h"

static int fail(const char* what) {
  printf("FAIL %s\n", what);
  return 1;
}

int main(void) {
  static int na[343], nb[343], nc[343];
  static int ta[343 * STRASSEN_MAX_TERMS], tb[343 * STRASSEN_MAX_TERMS], tc[343 * STRASSEN_MAX_TERMS];
  int levels, total_c;
  for (levels = 0; levels <= STRASSEN_MAX_LEVELS; ++levels) {
    int r, expect = 1, i;
    for (i = 0; i < levels; ++i) expect *= 7;
    if (strassen_plan_table(levels, 343, na, nb, nc, ta, tb, tc) != expect) return fail("plan table size");
    total_c = 0;
    for (r = 0; r < expect; ++r) total_c += nc[r];
    /* C updates: 1, 12, 144, 1728 (12^L) */
    {
      int e12 = 1;
      for (i = 0; i < levels; ++i) e12 *= 12;
      if (total_c != e12) return fail("C update count");
    }
  }
  if (strassen_plan_table(STRASSEN_MAX_LEVELS + 1, 343, na, nb, nc, ta, tb, tc) != STRASSEN_ERR_LEVELS)
    return fail("levels check");
  if (strcmp(strassen_status_string(STRASSEN_OK), "ok") != 0) return fail("status string");
  /* argument checks fail before any device work */
  if (strassen_gemm(-1, 4, 4, (const double*)0x1000, 4, (const double*)0x2000, 4, (double*)0x3000, 4, 1,
                    STRASSEN_ABC, STRASSEN_F64, 0) != STRASSEN_ERR_DIM)
    return fail("dim check");
  if (strassen_dgemm(1, 0, 8, 4, 4, 1.0, (const double*)0x1000, 4, (const double*)0x2000, 4, 1.0,
                     (double*)0x3000, 4, 1, STRASSEN_ABC, STRASSEN_F64, 0) != STRASSEN_ERR_LD)
    return fail("dgemm ld check");
  if (strassen_dgemm_ex(0, 0, 4, 4, 4, 1.0, (const double*)0x1000, 4, (const double*)0x2000, 4, 1.0,
                        (double*)0x3000, 4, 1, STRASSEN_ABC, STRASSEN_F64, 4u, 0) != STRASSEN_ERR_ARG)
    return fail("dgemm_ex flags check");
  if (strassen_workspace_size(4096, 4096, 4096, 1, STRASSEN_AB, STRASSEN_F64) != 8LL * 2048 * 2048)
    return fail("AB workspace");
  if (strassen_workspace_size(4096, 4096, 4096, 2, STRASSEN_ABC, STRASSEN_F64) != 0) return fail("ABC workspace");
  if (!(strassen_model_seconds(8192, 8192, 8192, 2, STRASSEN_ABC) < strassen_model_seconds(8192, 8192, 8192, 0,
                                                                                          STRASSEN_ABC)))
    return fail("model");
  {
    int lv = -1, tile = -1;
    strassen_variant v = STRASSEN_AUTO;
    if (strassen_select(8192, 8192, 8192, STRASSEN_F64, &lv, &v, &tile) != STRASSEN_OK) return fail("select");
    if (lv < 1 || lv > STRASSEN_MAX_LEVELS || tile < 0) return fail("select result");
  }
  printf("abi client ok\n");
  return 0;
}
