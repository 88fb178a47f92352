/* A plain C client of the library: includes the public header with a C
 * compiler, links against the shared library and calls the host-only entry
 * points (workspace sizing and error strings), so no GPU is needed. */
#include <stdio.h>
#include <string.h>

#include "ccladder.h"

int main(void) {
  cc_ladder_system s;
  memset(&s, 0, sizeof(s));
  s.o = 4;
  s.v = 20;
  s.nj = 60;
  s.L_vv = (const double*)0x1000; /* sizing never dereferences */
  s.t2 = (const double*)0x2000;
  size_t step = cc_ladder_workspace_size(&s, 1, CC_PREC_MIXED, CC_WS_STEP);
  size_t res = cc_ladder_workspace_size(&s, 1, CC_PREC_MIXED, CC_WS_RESIDUAL);
  size_t f16 = cc_ladder_workspace_size(&s, 1, CC_PREC_FP16X2, CC_WS_STEP);
  size_t bad = cc_ladder_workspace_size(&s, 1, (cc_precision)7, CC_WS_STEP);
  const char* msg = cc_ladder_strerror(CC_ERR_WORKSPACE);
  size_t drv = cc_ladder_mp2_driver_workspace_size(4, 20, 60, CC_PREC_FP64);
  printf("%zu %zu %zu %zu %zu %s\n", step, res, f16, bad, drv, msg);
  return (step >= res && res > 0 && f16 > 0 && f16 < step && bad == 0 && drv > 0 && msg && *msg) ? 0 : 1;
}
