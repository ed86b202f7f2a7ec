// batch_row_d2q9.cu -- D2Q9 instantiations of the batched row kernel.
#include "batch_row.cuh"

namespace lbm {

// shape class: bits 0-1 row pitch 64, 128, 256, 512; bit 2 walls on y/z;
// odd: the step parity of the launched part; redc: a check replay
cudaError_t launch_batch_row_d2q9(int storage, int shape, int odd, int redc, const BatchMember *members, const int *row_member,
                                  const int *row_begin, const int2 *cls, double *member_sums, int *status,
                                  int k, int kmax, int check, int grid, cudaStream_t s) {
#define LBM_BR(ST, P, W) \
  return launch_batch_row_t<D2Q9, ST, P, W>(odd != 0, redc != 0, members, row_member, row_begin, cls, member_sums, status, k, kmax, check, grid, s)
#define LBM_BR_SHAPES(ST)           \
  switch (shape) {                 \
    case 0: LBM_BR(ST, 64, false);  \
    case 1: LBM_BR(ST, 128, false); \
    case 2: LBM_BR(ST, 256, false); \
    case 3: LBM_BR(ST, 512, false); \
    case 4: LBM_BR(ST, 64, true);   \
    case 5: LBM_BR(ST, 128, true);  \
    case 6: LBM_BR(ST, 256, true);  \
    case 7: LBM_BR(ST, 512, true);  \
  }
  if (storage == 1) LBM_BR_SHAPES(float)
  else if (storage == 2) LBM_BR_SHAPES(__half)
#undef LBM_BR_SHAPES
#undef LBM_BR
  return cudaErrorInvalidValue;
}

int configure_batch_row_d2q9(int storage, int shape) {
#define LBM_CF(ST, P, W) return configure_batch_row_t<D2Q9, ST, P, W>()
#define LBM_CF_SHAPES(ST)           \
  switch (shape) {                 \
    case 0: LBM_CF(ST, 64, false);  \
    case 1: LBM_CF(ST, 128, false); \
    case 2: LBM_CF(ST, 256, false); \
    case 3: LBM_CF(ST, 512, false); \
    case 4: LBM_CF(ST, 64, true);   \
    case 5: LBM_CF(ST, 128, true);  \
    case 6: LBM_CF(ST, 256, true);  \
    case 7: LBM_CF(ST, 512, true);  \
  }
  if (storage == 1) LBM_CF_SHAPES(float)
  else if (storage == 2) LBM_CF_SHAPES(__half)
#undef LBM_CF_SHAPES
#undef LBM_CF
  return 0;
}

}  // namespace lbm
