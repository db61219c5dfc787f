/* A plain C99 caller of the C ABI: include/hp.h must compile as C, and the
 * host-only entry points must work without a GPU.  Built and run by
 * tests/test_c_abi.py; exits 0 on success. */
#include <stdio.h>

#include "hp.h"

int main(void) {
  /* Sec. 3.3's example: sync() reserve(barrier) over sync(barrier) -> GRID over CLUSTER */
  hp_level_req req[2] = {{0u, (uint32_t)HP_PROP_BARRIER, 0}, {(uint32_t)HP_PROP_BARRIER, 0u, 0}};
  hp_level_map map[2];
  uint32_t props = 0;
  int64_t num = 0;
  hp_nest *n = NULL;
  int64_t ext[2] = {16, 4096};
  char buf[4096];
  double bound = -1.0;
  if (hp_level_select(2, req, map) != HP_OK) { printf("select: %s\n", hp_last_error()); return 1; }
  if (map[0].hw != HP_HW_GRID || map[1].hw != HP_HW_CLUSTER) { printf("unexpected map\n"); return 2; }
  if (hp_level_check(2, req, map) != HP_OK) { printf("check: %s\n", hp_last_error()); return 3; }
  if (hp_level_properties(HP_HW_WARP, &props, &num) != HP_OK || !(props & HP_PROP_SHUFFLE) || num != 32) return 4;
  /* planning is host-only: create, describe and destroy a nest without a GPU */
  if (hp_nest_create(2, ext, NULL, 0, NULL, HP_RED_SUM, 1, HP_F32_COMP, HP_BODY_LOAD, NULL, &n) != HP_OK) {
    printf("create: %s\n", hp_last_error());
    return 5;
  }
  if (hp_nest_describe(n, buf, sizeof buf) != HP_OK || buf[0] != '{') return 6;
  if (hp_nest_error_bound(n, &bound) != HP_OK || !(bound > 0.0 && bound < 1e-5)) return 7;
  hp_nest_destroy(n);
  /* errors are status codes with a message, never an abort */
  if (hp_nest_create(0, ext, NULL, 0, NULL, HP_RED_SUM, 1, HP_F32, HP_BODY_LOAD, NULL, &n) != HP_EINVAL) return 8;
  if (hp_last_error()[0] == '\0') return 9;
  printf("ok %d\n", hp_version());
  return 0;
}
