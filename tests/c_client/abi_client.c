/* A plain C99 client of libg3gemm: it includes only g3gemm.h, links only the
 * shared library and exercises the calls that need no device (argument
 * validation, status strings, the generated family, the planner).  Exit
 * status 0 when every check holds; otherwise the first failed check is
 * printed and the status is 1. */
#include <stdio.h>
#include <string.h>

#include "g3gemm.h"

#define CHECK(cond)                                                \
  do {                                                             \
    if (!(cond)) {                                                 \
      fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
      return 1;                                                    \
    }                                                              \
  } while (0)

int main(void) {
  /* any non-null "device" address: validation fails before any use */
  void* p = (void*)(size_t)16;
  char buf[256];
  int cfg = 0, sk = 0, rs = 0, i;
  g3_gemm_args a;

  /* positional argument errors of g3_gemm, in the order of its signature */
  CHECK(g3_gemm(-1, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, G3_F32) == -101);
  CHECK(g3_gemm(4, -1, 4, 1.0, p, 4, p, 4, 0.0, p, 4, G3_F32) == -102);
  CHECK(g3_gemm(4, 4, -1, 1.0, p, 4, p, 4, 0.0, p, 4, G3_F32) == -103);
  CHECK(g3_gemm(4, 4, 8, 1.0, NULL, 8, p, 4, 0.0, p, 4, G3_F32) == -105);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 7, p, 4, 0.0, p, 4, G3_F32) == -106);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 8, NULL, 4, 0.0, p, 4, G3_F32) == -107);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 8, p, 3, 0.0, p, 4, G3_F32) == -108);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, NULL, 4, G3_F32) == -110);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, p, 3, G3_F32) == -111);
  CHECK(g3_gemm(4, 4, 8, 1.0, p, 8, p, 4, 0.0, p, 4, (g3_dtype)42) == -112);
  /* m == 0 is a no-op that touches nothing */
  CHECK(g3_gemm(0, 4, 8, 1.0, NULL, 8, NULL, 4, 0.0, NULL, 4, G3_BF16) == G3_OK);

  /* extended arguments: defaults, then a transposed operand's rule */
  g3_gemm_args_init(&a);
  CHECK(a.config == -1 && a.split_k == 0 && a.trans_a == 0 && a.workspace == NULL);
  a.m = 6; a.n = 4; a.k = 8; a.alpha = 1.0; a.A = p; a.B = p; a.C = p;
  a.lda = 5; a.ldb = 4; a.ldc = 4; a.trans_a = 1;
  {
    size_t bytes = 0;
    CHECK(g3_gemm_workspace_size(&a, &bytes) == -106);
  }

  /* every status has a description */
  for (i = G3_ERR_NOT_INIT; i <= G3_OK; ++i) CHECK(g3_status_string(i) && strlen(g3_status_string(i)) > 0);

  /* the generated family and the planner */
  CHECK(g3_family_size() > 0);
  CHECK(g3_family_describe(0, buf, sizeof buf) == G3_OK && strncmp(buf, "mode=", 5) == 0);
  CHECK(g3_plan_query(16384, 16384, 16384, G3_F32_3XBF16, &cfg, &sk, &rs) == G3_OK);
  CHECK(cfg >= 0 && cfg < g3_family_size() && sk >= 1 && rs >= 1);
  CHECK(g3_family_describe(cfg, buf, sizeof buf) == G3_OK && strstr(buf, "mode=3xbf16") != NULL);
  CHECK(g3_plan_query(512, 512, 512, G3_F32, &cfg, &sk, &rs) == G3_OK && cfg == -1 && sk >= 1);
  CHECK(g3_plan_query(-1, 4, 4, G3_BF16, &cfg, &sk, &rs) == -101);

  printf("abi client ok: %d family members, planner member %d for FP32-accurate 16384^3\n", g3_family_size(),
         cfg);
  return 0;
}
