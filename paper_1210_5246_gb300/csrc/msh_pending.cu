// msh_pending.cu -- entry points whose kernels are not in this build yet.
#include <string>

#include "../../include/msh.h"

extern "C" {
msh_status msh_adjoint_run(msh_grid *, const void *, int64_t, const double *, int32_t, const void *, void *,
                           int32_t, int32_t) {
  return MSH_E_STATE;
}
msh_status msh_batch_init(msh_batch **, int32_t, const int32_t *, const double *, const double *, const double *,
                          int32_t, double, void *) {
  return MSH_E_STATE;
}
msh_status msh_batch_reset(msh_batch *) { return MSH_E_STATE; }
msh_status msh_batch_run(msh_batch *, int32_t, int64_t) { return MSH_E_STATE; }
msh_status msh_batch_run_per_tube(msh_batch *, const int32_t *, int32_t, int64_t) { return MSH_E_STATE; }
msh_status msh_batch_get_state(msh_batch *, void *, int32_t, int32_t) { return MSH_E_STATE; }
msh_status msh_batch_info(msh_batch *, int64_t *, double *, int64_t *) { return MSH_E_STATE; }
msh_status msh_batch_destroy(msh_batch *) { return MSH_E_STATE; }
}
