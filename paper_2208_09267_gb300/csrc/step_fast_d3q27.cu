// step_fast_d3q27.cu -- D3Q27 instantiations of the fused FP32/FP16 step.
#include "step_fast.cuh"

namespace lbm {

cudaError_t launch_step_fast_d3q27(const LatticeDev *L_dev, int storage, bool odd, int red, int k,
                                   const StepLaunch &ls, cudaStream_t s) {
  if (storage == 1) {
    if (odd) {
      if (red) step_fast_kernel<D3Q27, float, true, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
      else step_fast_kernel<D3Q27, float, true, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    } else {
      if (red) step_fast_kernel<D3Q27, float, false, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
      else step_fast_kernel<D3Q27, float, false, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    }
  } else if (storage == 2) {
    if (odd) {
      if (red) step_fast_kernel<D3Q27, __half, true, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
      else step_fast_kernel<D3Q27, __half, true, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    } else {
      if (red) step_fast_kernel<D3Q27, __half, false, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
      else step_fast_kernel<D3Q27, __half, false, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    }
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm

#include "step_row.cuh"

#ifndef LBM_ROW_MINB_D3Q27
#define LBM_ROW_MINB_D3Q27 1
#endif

namespace lbm {

cudaError_t launch_step_row_d3q27(const LatticeDev *L_dev, int storage, bool odd, int red, int k,
                                  const StepLaunch &ls, cudaStream_t s) {
  if (storage == 1) return launch_row_t<D3Q27, float, LBM_ROW_MINB_D3Q27>(L_dev, odd, red, k, ls, s);
  if (storage == 2) return launch_row_t<D3Q27, __half, LBM_ROW_MINB_D3Q27>(L_dev, odd, red, k, ls, s);
  return cudaErrorInvalidValue;
}

int plan_row_d3q27(int storage, int nx, int nxp, int ny, int nz, unsigned walls, StepLaunch &ls) {
  if (storage == 1) return plan_row_t<D3Q27, float, LBM_ROW_MINB_D3Q27>(nx, nxp, ny, nz, walls, ls);
  if (storage == 2) return plan_row_t<D3Q27, __half, LBM_ROW_MINB_D3Q27>(nx, nxp, ny, nz, walls, ls);
  return 0;
}

}  // namespace lbm
