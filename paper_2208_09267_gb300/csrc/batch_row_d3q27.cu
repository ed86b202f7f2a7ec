// batch_row_d3q27.cu -- D3Q27 instantiations of the batched row kernel.
#include "batch_row.cuh"

namespace lbm {

// pclass: row pitch 64, 128, 256, 512 for 0..3
cudaError_t launch_batch_row_d3q27(int storage, int pclass, const BatchMember *members, const int *row_member,
                                  const int *row_begin, const int2 *cls, double *member_sums, int *status,
                                  int k, int kmax, int check, int grid, cudaStream_t s) {
#define LBM_BR(ST, P) \
  return launch_batch_row_t<D3Q27, ST, P>(members, row_member, row_begin, cls, member_sums, status, k, kmax, check, grid, s)
  if (storage == 1) {
    switch (pclass) {
      case 0: LBM_BR(float, 64);
      case 1: LBM_BR(float, 128);
      case 2: LBM_BR(float, 256);
      case 3: LBM_BR(float, 512);
    }
  } else if (storage == 2) {
    switch (pclass) {
      case 0: LBM_BR(__half, 64);
      case 1: LBM_BR(__half, 128);
      case 2: LBM_BR(__half, 256);
      case 3: LBM_BR(__half, 512);
    }
  }
#undef LBM_BR
  return cudaErrorInvalidValue;
}

int configure_batch_row_d3q27(int storage, int pclass) {
  if (storage == 1) {
    switch (pclass) {
      case 0: return configure_batch_row_t<D3Q27, float, 64>();
      case 1: return configure_batch_row_t<D3Q27, float, 128>();
      case 2: return configure_batch_row_t<D3Q27, float, 256>();
      case 3: return configure_batch_row_t<D3Q27, float, 512>();
    }
  } else if (storage == 2) {
    switch (pclass) {
      case 0: return configure_batch_row_t<D3Q27, __half, 64>();
      case 1: return configure_batch_row_t<D3Q27, __half, 128>();
      case 2: return configure_batch_row_t<D3Q27, __half, 256>();
      case 3: return configure_batch_row_t<D3Q27, __half, 512>();
    }
  }
  return 0;
}

}  // namespace lbm
