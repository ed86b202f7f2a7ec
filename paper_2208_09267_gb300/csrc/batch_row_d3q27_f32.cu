// batch_row_d3q27_f32.cu -- D3Q27 instantiations of the batched row kernel,
// FP32 storage (one file per lattice and storage, compiled in parallel).
#include "batch_row.cuh"

namespace lbm {

// shape class: bits 0-1 row pitch (2: 256, 3: 512); bit 2 walls on y/z;
// odd: the step parity of the launched part; redc: a check replay; first:
// the replay's first step
cudaError_t launch_batch_row_d3q27_f32(int shape, int odd, int redc, int first, const BatchMember *members,
                                     const int *item_member, const int *item_begin, const int2 *cls,
                                     double *member_sums, int *status, int k, int kmax, int check, int grid,
                                     cudaStream_t s) {
#define LBM_BR(P, W)                                                                                       \
  return launch_batch_row_t<D3Q27, float, P, W>(odd != 0, redc != 0, first != 0, members, item_member, item_begin, \
                                             cls, member_sums, status, k, kmax, check, grid, s)
  switch (shape) {
    case 2: LBM_BR(256, false);
    case 3: LBM_BR(512, false);
    case 6: LBM_BR(256, true);
    case 7: LBM_BR(512, true);
  }
#undef LBM_BR
  return cudaErrorInvalidValue;
}

int configure_batch_row_d3q27_f32(int shape) {
  switch (shape) {
    case 2: return configure_batch_row_t<D3Q27, float, 256, false>();
    case 3: return configure_batch_row_t<D3Q27, float, 512, false>();
    case 6: return configure_batch_row_t<D3Q27, float, 256, true>();
    case 7: return configure_batch_row_t<D3Q27, float, 512, true>();
  }
  return 0;
}

}  // namespace lbm
