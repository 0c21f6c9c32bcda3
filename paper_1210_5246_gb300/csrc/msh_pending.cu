// msh_pending.cu -- entry points whose kernels are not in this build yet.
#include <string>

#include "../../include/msh.h"

extern "C" {
msh_status msh_adjoint_run(msh_grid *, const void *, int64_t, const double *, int32_t, const void *, void *,
                           int32_t, int32_t) {
  return MSH_E_STATE;
}
}
