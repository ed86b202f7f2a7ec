// internal.h -- device-side lattice descriptor and internal launchers.
//
// Everything a step kernel needs that can change between calls lives in a
// small struct in device memory (LatticeDev), not in kernel arguments: the
// time counter, the phi and force fields and the shift pointers.  A captured
// CUDA graph of step kernels therefore stays valid when the caller refreshes
// phi (set_epsilon) or the force, and when the time counter advances.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

struct LatticeDev {
  // geometry: cell (x, y, z) is stored at index (z*ny + y)*nxp + x, rows
  // padded to a pitch of nxp >= nx elements (16-byte aligned rows for the
  // bulk copies); population slot i of a cell lives at pop[i*plane + cell].
  // Caller-facing fields are dense (x fastest, pitch nx).
  int nx, ny, nz;
  int lattice;             // 0 D2Q9, 1 D3Q19, 2 D3Q27
  long long ncell;         // nxp * ny * nz: stored cells, padding included
  long long plane;         // elements between population planes (>= ncell)
  int nxp;                 // row pitch
  int pad0;
  unsigned walls;          // axis bits of solid first/last layers
  unsigned quad_axes;      // axis bits entering eq. (quad)
  int storage;             // 0 FP64, 1 FP32, 2 FP16
  int has_deps;            // phi has a time derivative field
  int has_force;           // per-cell force field present
  int has_dforce;          // ... and its time derivative
  void *pop;
  const void *eps;         // phi_ref (double for FP64, float otherwise)
  const void *deps;        // d_t phi or null
  const __half *sig_rd;    // shift sigma the stored populations are encoded with
  const __half *sig_wr;    // shift the next write encodes with (from phi_ref)
  const void *force;       // 3*ncell, component-major, or null
  const void *dforce;
  double g[3];             // uniform force density
  long long n;             // time counter: state is f(., n)
  long long n_eps, n_force;
  double omega;            // 1/tau
  double cf;               // 1 - 1/(2 tau)
  double rho0;
  double qw0, qw1;         // Table "weights" row of quad_dim
  float scale, inv_scale;  // 2^k, 2^-k (FP16); 1, 1 otherwise
  // the parameters above rounded to float once on the host, so the FP32
  // kernels convert nothing per cell (double conversions run on the narrow
  // FP64 pipe): rho0, omega, 3 cf, 9 cf, qw0, qw1, g, cf
  float rho0f, omegaf, cf3f, cf9f, qw0f, qw1f, gf[3], cff;
  // reductions of a check step
  double *partials;        // per-block partial sums, kRedWidth each
  float *u_prev;           // 3*ncell velocity of the previous check, or null
  int have_prev;           // u_prev holds a previous check
  int pad1;
  int *status;             // device flag: nonzero after a bounded wait gave up
  unsigned wait_limit;     // iteration limit of the row kernel's stage waits
  int withhold_copies;     // test only: the row kernel issues no copies
  int fp16_nearest;        // FP16 stores: 0 stochastic rounding, 1 nearest
  int pad3;
  // phase-interaction drag (Ergun-type, implicit in eq. (velocity)) and the
  // Smagorinsky closure; both zero = the plain scheme.  Doubles as given by
  // the caller (the FP64 kernels follow the reference's operation order),
  // floats premultiplied for the FP32 kernels.
  int drag_model;          // 0 none, 1 Ergun-type
  int les;                 // Smagorinsky closure on
  double drag_c1, drag_c2, drag_d;  // viscous / inertial coefficients, particle diameter
  double tau0;             // the laminar relaxation time tau
  double les_cs;           // Smagorinsky constant C
  float drag_linf;         // c1 nu / d^2
  float drag_qf;           // c2 / d
  float les_cf;            // 18 sqrt(2) C^2
  float tau0f;
};

constexpr int kRedWidth = 12;  // M0, mom x/y/z, |du|^2, |u|^2, nan, F x/y/z, spare x2

struct StepLaunch {
  dim3 grid, block;
  int block_threads;
  // row-staged kernel (step_row.cuh): used when row != 0
  int row;
  int row_grid;
  int row_smem_even, row_smem_odd;
  // row kernel shape: consumer warps and input stages per block (0 = the
  // compiled default; the planner writes back what it chose)
  int row_consumers, row_stages;
};

// Plan the row-staged kernel for a lattice: fills ls.row* and returns 1 when
// the lattice qualifies (storage FP32/FP16, rows 16-byte aligned, nx <= 512,
// no x walls, shared memory fits), else 0.
int plan_row_kernel(int lattice, int storage, int nx, int nxp, int ny, int nz, unsigned walls, StepLaunch &ls);

// Default/chosen block shape -> launch geometry for a lattice.
StepLaunch make_launch(int nx, int ny, int nz, int bx, int by);

// Launch one fused step (parity from n_host) of a single lattice, reading
// the descriptor at L_dev.  `k` is added to the device-side time counter
// (steps inside a captured chunk).  red = 1 makes it a check step.
cudaError_t launch_step(const LatticeDev &host_mirror, const LatticeDev *L_dev, long long n_host,
                        int k, int red, const StepLaunch &ls, cudaStream_t s);

// Advance the device-side time counter by k.
cudaError_t launch_advance(LatticeDev *L_dev, int k, cudaStream_t s);

// Sum per-block partials into out[kRedWidth] in a fixed order.
cudaError_t launch_finalize(const double *partials, int nblocks, double *out, cudaStream_t s);

// Moments at the device-side time n into double or float outputs (device
// pointers, any may be null).
cudaError_t launch_moments(const LatticeDev &host_mirror, const LatticeDev *L_dev, long long n_host,
                           double *rho, double *p, double *u, float *rho_f, float *p_f,
                           float *u_f, cudaStream_t s);

// Equilibrium initialisation at time n (mode bits as lbm_vanse_init_equilibrium);
// p0 and u0 are device double arrays or null.
cudaError_t launch_init(const LatticeDev &host_mirror, const LatticeDev *L_dev, long long n_host,
                        const double *p0, const double *u0, int mode, cudaStream_t s);

// Decoded populations f[cell*Q + i] (double, natural order) into a device buffer.
cudaError_t launch_get_populations(const LatticeDev &host_mirror, const LatticeDev *L_dev,
                                   long long n_host, double *f, cudaStream_t s);

// Shift of the reduced-precision storages from phi_ref (float, N values):
// sigma(x) = int phi dV by eq. (quad) on the lattice's quadrature axes,
// rounded to half.
cudaError_t launch_shift(const LatticeDev &host_mirror, const float *eps, __half *sig, cudaStream_t s);

// Scan n values (float or double) on the device: sets *first_bad to the
// smallest index whose value is not finite or, with unit != 0, not in (0, 1].
// *first_bad must hold a value >= n beforehand.
cudaError_t launch_validate(const void *data, long long n, int is_f64, int unit, long long *first_bad,
                            cudaStream_t s);

// OR into *mask the axes (bit a = axis a < dims) along which the pitched
// field f (float or double, nx*ny*nz values at row pitch nxp) varies.
cudaError_t launch_variation(const void *f, int is_f64, int nx, int nxp, int ny, int nz, int dims,
                             unsigned *mask, cudaStream_t s);

// Float -> double / double -> float conversions for field uploads.
cudaError_t launch_convert_f2d(const float *in, double *out, long long n, cudaStream_t s);
cudaError_t launch_convert_d2f(const double *in, float *out, long long n, cudaStream_t s);

// Dense (row length nx) device array of `rows` rows -> pitched array (row
// pitch nxp), converting float <-> double as needed.
cudaError_t launch_pitch_convert(const void *in, int in_f64, void *out, int out_f64, int nx, int nxp,
                                 long long rows, cudaStream_t s);

// ---- batched stepping ---------------------------------------------------

struct BatchTile {
  int member;        // index into the member descriptor table
  int z, y0, ny;     // rows [y0, y0+ny) of plane z
  int x0, nxt;       // columns [x0, x0 + nxt)
};

struct BatchMember {
  LatticeDev *L;       // device descriptor of the member lattice
  long long budget;    // steps left at the start of the replay
  int tile_begin, tile_end;
  int lattice, storage;
  int row;             // 1: stepped by the batched row kernel (sums in the member sums)
  int pad;
};

cudaError_t launch_batch_step(int lattice, int storage, const BatchMember *members,
                              const BatchTile *tiles, const int *ntiles_dev, int max_tiles,
                              int k, int red, int grid, int block, cudaStream_t s);
cudaError_t launch_batch_advance(BatchMember *members, const int *nmembers_dev, int max_members,
                                 int k, cudaStream_t s);
cudaError_t launch_batch_finalize(const BatchMember *members, const int *nmembers_dev,
                                  int max_members, const double *tile_partials, double *out,
                                  cudaStream_t s);

int sm_count();

// Process-wide count of launched kernels (see lbm_vanse_launch_count).
void count_launches(long long n);

}  // namespace lbm
