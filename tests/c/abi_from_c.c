/* The C ABI used from plain C99: include/hfx.h must compile as C, and the calls that
 * answer on the host (defaults, argument checks) must work without a GPU.  Built and run
 * by tests/test_abi_cpu.py; exits 0 on success, otherwise the number of the failed check. */
#include <stdio.h>
#include <string.h>

#include "hfx.h"

int main(void) {
  hfx_options o;
  hfx_default_options(&o);
  if (o.omega != 0.11 || o.schwarz_tau != 1e-10 || o.precision != HFX_FP64 || o.schedule != HFX_SCHED_DYNAMIC)
    return 1;
  if (o.fp32_class_mask != HFX_FP32_CLASSES_DEFAULT || o.density_tau != 0.0) return 2;

  hfx_server_options so;
  hfx_server_default_options(&so);
  if (so.hbm_budget_gb != 120.0 || so.max_inflight != 4 || so.max_batch != 16) return 3;

  /* argument checks come before any device work */
  hfx_ctx* ctx = NULL;
  if (hfx_init_basis(NULL, 1, NULL, 1, NULL, NULL, NULL, NULL, NULL, NULL, NULL) != HFX_ERR_ARG) return 4;
  if (hfx_init_basis(&ctx, 0, NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL, NULL) != HFX_ERR_ARG) return 5;
  if (ctx != NULL) return 6;
  const char* msg = hfx_last_error(NULL);
  if (!msg || strlen(msg) == 0) return 7;
  if (hfx_build_K(NULL, NULL, NULL, 0) != HFX_ERR_ARG) return 8;
  if (hfx_build_pairs(NULL) != HFX_ERR_ARG) return 9;
  int64_t q0 = -1, q1 = -1;
  if (hfx_part_range(10, 1, 3, &q0, &q1) != HFX_OK || q0 != 3 || q1 != 6) return 10;
  if (hfx_serve_poll(NULL, 1, NULL) != HFX_ERR_ARG) return 11;
  if (hfx_energy_noalloc(NULL, NULL, 4, 4, NULL, NULL) != HFX_ERR_ARG) return 12;
  printf("C ABI ok\n");
  return 0;
}
