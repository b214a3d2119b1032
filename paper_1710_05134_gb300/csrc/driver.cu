// Three-stage k-th eigenpair driver (Algorithm 4).
#include "kep_ctx.h"

void kep_ctx::driver_release() {}

extern "C" kep_status kep_kth_eigenpair(kep_ctx* ctx, int64_t k, const kep_params* params, double* lambda,
                                        double* x, kep_report* report) {
  (void)ctx; (void)k; (void)params; (void)lambda; (void)x; (void)report;
  return KEP_ERR_INVALID;
}
