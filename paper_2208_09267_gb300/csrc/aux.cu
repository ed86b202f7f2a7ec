// aux.cu -- launch geometry, step dispatch and small helper kernels.
#include <atomic>

#include <cuda_runtime.h>

#include "../../include/lbm_vanse.h"
#include "internal.h"

namespace lbm {

cudaError_t launch_step_fast_d1q3(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_fast_d2q9(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_fast_d3q19(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_fast_d3q27(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_exact(int lattice, const LatticeDev *L_dev, bool odd, int red, int k,
                              const StepLaunch &ls, cudaStream_t s);
cudaError_t launch_step_row_d2q9(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_row_d3q19(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
cudaError_t launch_step_row_d3q27(const LatticeDev *, int, bool, int, int, const StepLaunch &, cudaStream_t);
int plan_row_d2q9(int, int, int, int, int, unsigned, StepLaunch &);
int plan_row_d3q19(int, int, int, int, int, unsigned, StepLaunch &);
int plan_row_d3q27(int, int, int, int, int, unsigned, StepLaunch &);

int plan_row_kernel(int lattice, int storage, int nx, int nxp, int ny, int nz, unsigned walls,
                    StepLaunch &ls) {
  ls.row = 0;
  if (storage == 0) return 0;
  switch (lattice) {
    case 0: return plan_row_d2q9(storage, nx, nxp, ny, nz, walls, ls);
    case 1: return plan_row_d3q19(storage, nx, nxp, ny, nz, walls, ls);
    case 2: return plan_row_d3q27(storage, nx, nxp, ny, nz, walls, ls);
  }
  return 0;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

StepLaunch make_launch(int nx, int ny, int nz, int bx, int by) {
  StepLaunch ls;
  if (bx <= 0 || by <= 0) {
    bx = round_up(nx, 32);
    if (bx > 256) bx = 256;
    by = 256 / bx;
    if (by > ny) by = ny;
    if (by < 1) by = 1;
  }
  ls.block = dim3(bx, by, 1);
  ls.grid = dim3((nx + bx - 1) / bx, (ny + by - 1) / by, nz);
  ls.block_threads = bx * by;
  ls.row = 0;
  ls.row_grid = 0;
  ls.row_smem_even = ls.row_smem_odd = 0;
  ls.row_consumers = ls.row_stages = 0;
  return ls;
}

cudaError_t launch_step(const LatticeDev &h, const LatticeDev *L_dev, long long n_host, int k, int red,
                        const StepLaunch &ls, cudaStream_t s) {
  const bool odd = ((n_host + k) & 1) != 0;
  if (h.storage == 0) return launch_step_exact(h.lattice, L_dev, odd, red, k, ls, s);
  if (ls.row) {
    // bit 1: this step decodes with the previous phi's shift (set_epsilon
    // since the last step); the row kernel is instantiated for both cases
    // bit 2: phi has no time derivative (a stage layout without d_t phi)
    const int rr = (red ? 1 : 0) | (h.sig_rd != h.sig_wr ? 2 : 0) | (h.has_deps ? 0 : 4);
    switch (h.lattice) {
      case 0: return launch_step_row_d2q9(L_dev, h.storage, odd, rr, k, ls, s);
      case 1: return launch_step_row_d3q19(L_dev, h.storage, odd, rr, k, ls, s);
      case 2: return launch_step_row_d3q27(L_dev, h.storage, odd, rr, k, ls, s);
    }
    return cudaErrorInvalidValue;
  }
  switch (h.lattice) {
    case 0: return launch_step_fast_d2q9(L_dev, h.storage, odd, red, k, ls, s);
    case 1: return launch_step_fast_d3q19(L_dev, h.storage, odd, red, k, ls, s);
    case 2: return launch_step_fast_d3q27(L_dev, h.storage, odd, red, k, ls, s);
    case 3: return launch_step_fast_d1q3(L_dev, h.storage, odd, red, k, ls, s);
  }
  return cudaErrorInvalidValue;
}

// After a chunk of k steps: advance the time counter and commit a pending
// change of shift (the first step of the chunk re-encoded every slot).
__global__ void advance_kernel(LatticeDev *L, int k) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    L->n += k;
    L->sig_rd = L->sig_wr;
  }
}

cudaError_t launch_advance(LatticeDev *L_dev, int k, cudaStream_t s) {
  advance_kernel<<<1, 32, 0, s>>>(L_dev, k);
  return cudaGetLastError();
}

// Deterministic sum of per-block partials: thread t adds blocks t, t+T, ...
// in order, then a fixed tree over the threads.
__global__ void finalize_kernel(const double *partials, int nblocks, double *out) {
  __shared__ double sm[256][kRedWidth];
  const int t = threadIdx.x;
  double acc[kRedWidth];
  for (int j = 0; j < kRedWidth; ++j) acc[j] = 0.0;
  for (int b = t; b < nblocks; b += blockDim.x)
    for (int j = 0; j < kRedWidth; ++j) acc[j] += partials[(long long)b * kRedWidth + j];
  for (int j = 0; j < kRedWidth; ++j) sm[t][j] = acc[j];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int j = 0; j < kRedWidth; ++j) sm[t][j] += sm[t + w][j];
    __syncthreads();
  }
  if (t < kRedWidth) out[t] = sm[0][t];
}

cudaError_t launch_finalize(const double *partials, int nblocks, double *out, cudaStream_t s) {
  finalize_kernel<<<1, 256, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// Threads along x; each thread walks a segment of y at fixed (x, z) with
// the rows y-1, y, y+1 of phi in registers, so phi is read about three
// times per cell (own row, z-1, z+1) instead of seven; x neighbours come
// from the row the warp has just read (L1).  Same sum order as eq. (quad)
// is written everywhere: x pair, y pair, z pair.
constexpr int kShiftSeg = 32;  // rows of y per thread

__global__ void shift_kernel(const float *eps, __half *sig, int nx, int nxp, int ny, int nz, unsigned qa,
                             float w0, float w1) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= nxp) return;
  const int nseg = (ny + kShiftSeg - 1) / kShiftSeg;
  const long long plane = (long long)ny * nxp;
  for (long long t = blockIdx.y; t < (long long)nz * nseg; t += gridDim.y) {
    const int z = (int)(t / nseg), y0 = (int)(t % nseg) * kShiftSeg;
    const int y1 = y0 + kShiftSeg < ny ? y0 + kShiftSeg : ny;
    const long long pz = (long long)z * plane;
    if (x >= nx) {  // row padding: a valid value that nothing decodes
      for (int y = y0; y < y1; ++y) sig[pz + (long long)y * nxp + x] = __float2half_rn(1.0f);
      continue;
    }
    const long long pzm = (long long)(z == 0 ? nz - 1 : z - 1) * plane;
    const long long pzp = (long long)(z == nz - 1 ? 0 : z + 1) * plane;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    float e_ym = eps[pz + (long long)(y0 == 0 ? ny - 1 : y0 - 1) * nxp + x];
    float e_c = eps[pz + (long long)y0 * nxp + x];
    for (int y = y0; y < y1; ++y) {
      const long long row = pz + (long long)y * nxp;
      const float e_yp = eps[pz + (long long)(y == ny - 1 ? 0 : y + 1) * nxp + x];
      float nb = 0.f;
      if (qa & 1u) nb += eps[row + xp] + eps[row + xm];
      if (qa & 2u) nb += e_yp + e_ym;
      if (qa & 4u) nb += eps[pzp + (long long)y * nxp + x] + eps[pzm + (long long)y * nxp + x];
      sig[row + x] = __float2half_rn(fmaf(w0, e_c, w1 * nb));
      e_ym = e_c;
      e_c = e_yp;
    }
  }
}

cudaError_t launch_shift(const LatticeDev &h, const float *eps, __half *sig, cudaStream_t s) {
  const int block = h.nxp >= 256 ? 256 : (h.nxp >= 128 ? 128 : 64);
  const long long work = (long long)h.nz * ((h.ny + kShiftSeg - 1) / kShiftSeg);
  const dim3 grid((unsigned)((h.nxp + block - 1) / block), (unsigned)(work < 65535 ? work : 65535));
  shift_kernel<<<grid, block, 0, s>>>(eps, sig, h.nx, h.nxp, h.ny, h.nz, h.quad_axes, (float)h.qw0,
                                      (float)h.qw1);
  return cudaGetLastError();
}

// Axes along which a pitched field varies: bit a of *mask is set when some
// cell's value differs from that of its +e_a neighbour (periodic), compared
// exactly.  One warp vote per axis, one atomicOr per warp that saw a change.
template <class T>
__global__ void variation_kernel(const T *f, int nx, int nxp, int ny, int nz, int dims, unsigned *mask) {
  const long long n = (long long)nx * ny * nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i - threadIdx.x < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned bits = 0;
    if (i < n) {
      const int x = (int)(i % nx);
      const long long r = i / nx;
      const int y = (int)(r % ny), z = (int)(r / ny);
      const long long row = ((long long)z * ny + y) * nxp;
      const T v = f[row + x];
      if (f[row + (x + 1 == nx ? 0 : x + 1)] != v) bits |= 1u;
      if (dims > 1 && f[((long long)z * ny + (y + 1 == ny ? 0 : y + 1)) * nxp + x] != v) bits |= 2u;
      if (dims > 2 && f[((long long)(z + 1 == nz ? 0 : z + 1) * ny + y) * nxp + x] != v) bits |= 4u;
    }
    const unsigned any = __reduce_or_sync(0xffffffffu, bits);
    if ((threadIdx.x & 31) == 0 && any) atomicOr(mask, any);
  }
}

cudaError_t launch_variation(const void *f, int is_f64, int nx, int nxp, int ny, int nz, int dims,
                             unsigned *mask, cudaStream_t s) {
  const long long n = (long long)nx * ny * nz;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (is_f64)
    variation_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double *>(f), nx, nxp, ny, nz,
                                                              dims, mask);
  else
    variation_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float *>(f), nx, nxp, ny, nz,
                                                             dims, mask);
  return cudaGetLastError();
}

__global__ void pitch_convert_kernel(const void *in, int in_f64, void *out, int out_f64, int nx, int nxp,
                                     long long rows) {
  const long long n = (long long)nx * rows;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nx, x = i % nx;
    const double v = in_f64 ? static_cast<const double *>(in)[i] : (double)static_cast<const float *>(in)[i];
    const long long o = r * nxp + x;
    if (out_f64)
      static_cast<double *>(out)[o] = v;
    else
      static_cast<float *>(out)[o] = (float)v;
  }
}

cudaError_t launch_pitch_convert(const void *in, int in_f64, void *out, int out_f64, int nx, int nxp,
                                 long long rows, cudaStream_t s) {
  const long long n = (long long)nx * rows;
  if (n <= 0) return cudaSuccess;
  long long g = (n + 255) / 256;
  if (g > 152LL * 32) g = 152LL * 32;
  pitch_convert_kernel<<<(int)g, 256, 0, s>>>(in, in_f64, out, out_f64, nx, nxp, rows);
  return cudaGetLastError();
}

template <class T>
__global__ void validate_kernel(const T *data, long long n, int unit, long long *first_bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = data[i];  // checked in its own type (no conversion on the FP64 pipe)
    const bool bad = !isfinite(v) || (unit && !(v > T(0) && v <= T(1)));
    if (bad) atomicMin((unsigned long long *)first_bad, (unsigned long long)i);
  }
}

cudaError_t launch_validate(const void *data, long long n, int is_f64, int unit, long long *first_bad,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  long long g = (n + 255) / 256;
  if (g > 152LL * 16) g = 152LL * 16;
  if (is_f64)
    validate_kernel<double><<<(int)g, 256, 0, s>>>(static_cast<const double *>(data), n, unit, first_bad);
  else
    validate_kernel<float><<<(int)g, 256, 0, s>>>(static_cast<const float *>(data), n, unit, first_bad);
  return cudaGetLastError();
}

__global__ void f2d_kernel(const float *in, double *out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (double)in[i];
}

__global__ void d2f_kernel(const double *in, float *out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

static int grid_for(long long n) {
  long long g = (n + 255) / 256;
  const long long cap = 152LL * 32;
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

cudaError_t launch_convert_f2d(const float *in, double *out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  f2d_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_convert_d2f(const double *in, float *out, long long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  d2f_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

static std::atomic<long long> g_launches{0};

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace lbm

extern "C" long long lbm_vanse_launch_count(void) { return lbm::g_launches.load(); }
