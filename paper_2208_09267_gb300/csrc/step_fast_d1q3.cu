// step_fast_d1q3.cu -- D1Q3 instantiations of the fused FP32/FP16 step (one
// cell per thread; a one-dimensional lattice has no rows to stage).
#include "step_fast.cuh"

namespace lbm {

template <class ST>
static cudaError_t launch_d1q3_st(const LatticeDev *L_dev, bool odd, int red, int k, const StepLaunch &ls,
                                  cudaStream_t s) {
  if (odd) {
    if (red) step_fast_kernel<D1Q3, ST, true, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    else step_fast_kernel<D1Q3, ST, true, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
  } else {
    if (red) step_fast_kernel<D1Q3, ST, false, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    else step_fast_kernel<D1Q3, ST, false, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_fast_d1q3(const LatticeDev *L_dev, int storage, bool odd, int red, int k,
                                  const StepLaunch &ls, cudaStream_t s) {
  if (storage == 1) return launch_d1q3_st<float>(L_dev, odd, red, k, ls, s);
  if (storage == 2) return launch_d1q3_st<__half>(L_dev, odd, red, k, ls, s);
  return cudaErrorInvalidValue;
}

}  // namespace lbm
