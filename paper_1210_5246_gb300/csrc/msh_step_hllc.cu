// msh_step_hllc.cu -- launchers of the characteristic step with the HLLC flux (the step
// kernels of msh_step_kernels.cuh with SCH = 4, compiled apart in parallel).
#include "msh_step_kernels.cuh"

namespace msh {

template <typename T>
cudaError_t launch_step_hllc(const StepArgs<T> &a, int ndim, int rows, bool retry, cudaStream_t s, int *nblocks_out) {
  if (nblocks_out) *nblocks_out = step_blocks<T>(ndim, rows, a.nx, a.ny, a.nz, a.zchunk);
  return retry ? launch_step_mode<T, 4, true>(a, ndim, rows, s) : launch_step_mode<T, 4, false>(a, ndim, rows, s);
}

template cudaError_t launch_step_hllc<float>(const StepArgs<float> &, int, int, bool, cudaStream_t, int *);
template cudaError_t launch_step_hllc<double>(const StepArgs<double> &, int, int, bool, cudaStream_t, int *);

}  // namespace msh
