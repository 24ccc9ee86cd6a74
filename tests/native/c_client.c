/* A plain C client of the library: every call below must return an error
 * code (never abort) on a machine without a usable GPU, and the size queries
 * and error strings must behave as include/dt.h states.  Built and run by
 * tests/test_c_client.py with the host C compiler. */
#include <stdio.h>
#include <string.h>

#include "dt.h"

#define CHECK(x)                                                  \
  do {                                                            \
    if (!(x)) {                                                   \
      printf("check failed at line %d: %s\n", __LINE__, #x);      \
      return 1;                                                   \
    }                                                             \
  } while (0)

int main(void) {
  dt_config cfg;
  CHECK(dt_config_default(&cfg) == DT_OK);
  CHECK(cfg.divide == DT_DIVIDE_SAMPLE && cfg.primitive == DT_PRIM_GRID && cfg.recursive == 0);
  dt_ctx* ctx = NULL;
  int rc = dt_create(&ctx, 0, NULL, &cfg);
  if (rc == DT_OK) {            /* a GPU is present: one tiny triangulation through the C ABI */
    double pts[5 * 2] = {0, 0, 1, 0, 0, 1, 1, 1, 0.25, 0.6};
    int64_t count = 0;
    CHECK(dt_triangulate(ctx, pts, 5, 2, 1, 0.0) == DT_OK);
    CHECK(dt_get_simplices(ctx, NULL, 0, &count) == DT_OK && count == 4);
    int32_t out[4 * 3];
    CHECK(dt_get_simplices(ctx, out, 1, &count) == DT_E_ARG);   /* capacity too small */
    CHECK(dt_get_simplices(ctx, out, 4, &count) == DT_OK);
    dt_destroy(ctx);
    printf("ok gpu\n");
    return 0;
  }
  CHECK(rc < 0 && ctx == NULL);
  CHECK(dt_triangulate(NULL, NULL, 0, 2, 1, 0.0) == DT_E_ARG);
  CHECK(strcmp(dt_last_error(NULL), "null context") == 0);
  int done = 0;
  uint64_t job = 0;
  CHECK(dt_submit(NULL, NULL, 0, 2, 1, 0.0, &job) == DT_E_ARG);
  CHECK(dt_poll(NULL, 1, &done) == DT_E_ARG);
  CHECK(dt_release_job(NULL, 1) == DT_E_ARG);
  dt_destroy(NULL);
  printf("ok\n");
  return 0;
}
