/* A plain C99 client of the library's C-ABI: includes the public header,
 * links the shared library and calls the host-only entry points (no device
 * is needed).  Built and run by tests/test_c_abi.py. */
#include <stdio.h>
#include <string.h>

#include "lift.h"

int main(void) {
  int op, total = 0;
  for (op = 0; op < LIFT_NUM_OPS; ++op) {
    const int cnt = lift_variant_count(op);
    lift_variant_info info;
    if (cnt <= 0 || lift_variant_describe(op, 0, &info) != LIFT_OK || info.op != op) return 1;
    total += cnt;
  }
  printf("variants %d\n", total);
  {
    lift_variant_info info;
    int v = -1;
    if (lift_pick(LIFT_OP_DOT, (int64_t)1 << 26, 0, 0, &v) != LIFT_OK) return 2;
    if (lift_variant_describe(LIFT_OP_DOT, v, &info) != LIFT_OK) return 3;
    printf("fixed dot pick %s\n", info.name);
  }
  {
    float f[LIFT_NUM_FEATURES];
    if (lift_features(LIFT_OP_GEMV, 0, 4096, 1024, f) != LIFT_OK) return 4;
    printf("gemv features %.3f %.0f %.0f\n", f[4], f[10], f[11]);
  }
  printf("status %s\n", lift_status_string(LIFT_ERR_TIMEOUT));
  /* arguments are checked before anything touches a device */
  if (lift_asum(NULL, 10, NULL, NULL) != LIFT_ERR_INVALID_ARG) return 5;
  printf("ok\n");
  return 0;
}
