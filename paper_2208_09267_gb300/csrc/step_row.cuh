// step_row.cuh -- persistent row kernel: the fused step of step_fast.cuh with
// its inputs staged in shared memory by TMA bulk copies.
//
// Work item: one fluid x-row (y, z) of the lattice, all nx cells.  A block
// keeps NSTAGE rows in flight: while the threads update row j, the bulk
// copies of row j + NSTAGE - 1 are landing.  Per row and step the block
// stages
//   - the Q population rows it reads: at even n plane i of its own row; at
//     odd n plane opp(i) of row (y - c_iy, z - c_iz) (the x shift of -c_ix
//     is a modular index into the staged row), or plane i of its own row when
//     that neighbour row is a wall layer (halfway bounce-back);
//   - phi_ref on the rows (y + dy, z + dz), dy, dz in {-1, 0, 1} (odd steps;
//     these also give the shift sigma of every neighbour) or the 5-point
//     cross (even steps), and d_t phi on the 5-point cross when phi varies;
// each as one contiguous cp.async.bulk of nx elements, completing on one
// mbarrier per stage.  Updated populations are written straight to global
// memory (coalesced, in place, AA pattern).
//
// Requirements (checked by the host before choosing this kernel): nx *
// sizeof(storage) and nx * 4 are multiples of 16 bytes, nx <= 512, walls
// only on y and/or z.  Every wait is bounded: a block that waits too long
// records the failure in L.status, drains its copies (again bounded) and
// leaves; the host reports LBM_ETIMEOUT.
#pragma once

#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"
#include "step_fast.cuh"

namespace lbm {

constexpr int kRowThreads = 256;
constexpr unsigned kWaitSpins = 1u << 22;  // bounded mbarrier wait

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes,
                                         unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for a phase with an iteration limit; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned limit = kWaitSpins) {
  for (unsigned i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Shared-memory layout of one stage (bytes), given the lattice.
struct RowLayout {
  int nx;
  int pop_bytes;   // one population row
  int eps_rows;    // phi_ref rows staged (9 odd / 5 even in 3D; 3 in 2D)
  int deps_rows;   // d_t phi rows staged (5 in 3D, 3 in 2D; 0 if static)
  int stage_bytes;
};

template <class LAT, class ST, bool ODD>
__host__ __device__ inline RowLayout row_layout(int nx, bool tv) {
  RowLayout r;
  r.nx = nx;
  r.pop_bytes = nx * (int)sizeof(ST);
  r.eps_rows = LAT::D == 2 ? 3 : (ODD ? 9 : 5);
  r.deps_rows = tv ? (LAT::D == 2 ? 3 : 5) : 0;
  r.stage_bytes = LAT::Q * r.pop_bytes + (r.eps_rows + r.deps_rows) * nx * 4;
  return r;
}

// Index of the phi_ref row (dy, dz) inside a stage.
template <class LAT, bool ODD>
__device__ __forceinline__ int eps_row_index(int dy, int dz) {
  if (LAT::D == 2) return dy + 1;
  if (ODD) return (dz + 1) * 3 + (dy + 1);
  // 5-point cross: 0 centre, 1 y-1, 2 y+1, 3 z-1, 4 z+1
  return dz == 0 ? (dy == 0 ? 0 : (dy < 0 ? 1 : 2)) : (dz < 0 ? 3 : 4);
}

// Index of the d_t phi row (dy, dz) (5-point cross; 2D: dy only).
template <class LAT>
__device__ __forceinline__ int deps_row_index(int dy, int dz) {
  if (LAT::D == 2) return dy + 1;
  return dz == 0 ? (dy == 0 ? 0 : (dy < 0 ? 1 : 2)) : (dz < 0 ? 3 : 4);
}

struct RowGeom {
  int y0, nyf, z0, nzf;  // fluid rows: y in [y0, y0+nyf), z in [z0, z0+nzf)
};

__device__ __forceinline__ RowGeom row_geom(const LatticeDev &L) {
  RowGeom g;
  const bool wy = (L.walls & 2u) != 0, wz = (L.walls & 4u) != 0;
  g.y0 = wy ? 1 : 0;
  g.nyf = wy ? L.ny - 2 : L.ny;
  g.z0 = wz ? 1 : 0;
  g.nzf = wz ? L.nz - 2 : L.nz;
  return g;
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

__device__ __forceinline__ bool row_solid(const LatticeDev &L, int y, int z) {
  return ((L.walls & 2u) && (y <= 0 || y >= L.ny - 1)) || ((L.walls & 4u) && (z <= 0 || z >= L.nz - 1));
}

// Thread 0: issue every bulk copy of row (y, z) into `stage`.
template <class LAT, class ST, bool ODD>
__device__ __forceinline__ void issue_row(const LatticeDev &L, const RowLayout &lay, unsigned char *stage,
                                          unsigned long long *bar, int y, int z) {
  const bool tv = L.has_deps != 0;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const unsigned total = (unsigned)lay.stage_bytes;
  mbar_arrive_expect_tx(bar, total);
  const ST *pop = static_cast<const ST *>(L.pop);
  const long long plane = L.plane;
  for (int i = 0; i < LAT::Q; ++i) {
    int plane_i = i, yy = y, zz = z;
    if (ODD && i != 0) {
      const int cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      const int ys = wrapi(y - cy, ny), zs = LAT::D == 3 ? wrapi(z - cz, nz) : z;
      if (!row_solid(L, ys, zs)) {
        plane_i = opp_of(i);
        yy = ys;
        zz = zs;
      }
    }
    const ST *src = pop + (long long)plane_i * plane + ((long long)zz * ny + yy) * nx;
    bulk_g2s(stage + i * lay.pop_bytes, src, (unsigned)lay.pop_bytes, bar);
  }
  const float *eps = static_cast<const float *>(L.eps);
  unsigned char *erow = stage + LAT::Q * lay.pop_bytes;
  const unsigned rb = (unsigned)nx * 4u;
  if (LAT::D == 2) {
    for (int dy = -1; dy <= 1; ++dy)
      bulk_g2s(erow + (dy + 1) * rb, eps + (long long)wrapi(y + dy, ny) * nx, rb, bar);
  } else if (ODD) {
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        bulk_g2s(erow + ((dz + 1) * 3 + (dy + 1)) * rb,
                 eps + ((long long)wrapi(z + dz, nz) * ny + wrapi(y + dy, ny)) * nx, rb, bar);
  } else {
    const int dys[5] = {0, -1, 1, 0, 0}, dzs[5] = {0, 0, 0, -1, 1};
    for (int j = 0; j < 5; ++j)
      bulk_g2s(erow + j * rb, eps + ((long long)wrapi(z + dzs[j], nz) * ny + wrapi(y + dys[j], ny)) * nx, rb,
               bar);
  }
  if (tv) {
    const float *deps = static_cast<const float *>(L.deps);
    unsigned char *drow = erow + lay.eps_rows * rb;
    const int nd = LAT::D == 2 ? 3 : 5;
    const int dys[5] = {0, -1, 1, 0, 0}, dzs[5] = {0, 0, 0, -1, 1};
    for (int j = 0; j < nd; ++j) {
      const int dy = LAT::D == 2 ? j - 1 : dys[j], dz = LAT::D == 2 ? 0 : dzs[j];
      bulk_g2s(drow + j * rb, deps + ((long long)wrapi(z + dz, nz) * ny + wrapi(y + dy, ny)) * nx, rb, bar);
    }
  }
}

// Update the cells of row (y, z) owned by this thread from a staged row.
template <class LAT, class ST, bool ODD, bool RED>
__device__ __forceinline__ void update_row_cells(const LatticeDev &L, const RowLayout &lay,
                                                 const unsigned char *stage, long long n, int y, int z,
                                                 RedAcc &acc) {
  constexpr int Q = LAT::Q, D = LAT::D;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const ST *prow = reinterpret_cast<const ST *>(stage);
  const float *erow = reinterpret_cast<const float *>(stage + Q * lay.pop_bytes);
  const float *drow = erow + lay.eps_rows * nx;
  const bool tv = L.has_deps != 0;
  const float dn = (float)(n - L.n_eps);
  const float rho0 = (float)L.rho0;
  const float inv_scale = L.inv_scale, scale = L.scale;
  const float *__restrict__ eps_g = static_cast<const float *>(L.eps);
  const float *__restrict__ srd = L.sig_rd;
  const bool reshift = srd != eps_g;  // shift changed by the last set_epsilon
  const unsigned walls = L.walls;
  ST *__restrict__ pop = static_cast<ST *>(L.pop);
  const long long plane = L.plane;
  const int ym = wrapi(y - 1, ny), yp = wrapi(y + 1, ny);
  const int zm = D == 3 ? wrapi(z - 1, nz) : z, zp = D == 3 ? wrapi(z + 1, nz) : z;
  const int rowbase = (z * ny + y) * nx;
  // sigma (phi_ref) on the staged rows; reshift steps read sigma_rd from global
  auto E = [&](int dy, int dz, int xx) -> float { return erow[eps_row_index<LAT, ODD>(dy, dz) * nx + xx]; };
  auto Dd = [&](int dy, int dz, int xx) -> float { return drow[deps_row_index<LAT>(dy, dz) * nx + xx]; };

  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int xs[3] = {xm, x, xp};
    const int ys_[3] = {ym, y, yp};
    const int zs_[3] = {zm, z, zp};
    const int cell = rowbase + x;
    float s_x = rho0 * (reshift ? __ldg(srd + cell) : E(0, 0, x));

    // 1. decode
    float d[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      if (!ODD || i == 0) {
        d[i] = PopIO<ST>::ld(prow + i * nx + x) * inv_scale;
      } else if (walls && row_solid(L, ys_[1 - cy], zs_[1 - cz])) {
        d[i] = PopIO<ST>::ld(prow + i * nx + x) * inv_scale;
      } else {
        const int xsrc = xs[1 - cx];
        float sm;
        if (reshift)
          sm = __ldg(srd + (zs_[1 - cz] * ny + ys_[1 - cy]) * nx + xsrc);
        else
          sm = E(-cy, -cz, xsrc);
        d[i] = fmaf(PopIO<ST>::ld(prow + i * nx + xsrc), inv_scale, rho0 * sm - s_x);
      }
    }

    // 2. moments
    float dM = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const float wd = (float)LAT::w(i) * d[i];
      dM += wd;
      if (LAT::c(i, 0) == 1) j0 += wd;
      if (LAT::c(i, 0) == -1) j0 -= wd;
      if (LAT::c(i, 1) == 1) j1 += wd;
      if (LAT::c(i, 1) == -1) j1 -= wd;
      if (D == 3 && LAT::c(i, 2) == 1) j2 += wd;
      if (D == 3 && LAT::c(i, 2) == -1) j2 -= wd;
    }
    const float M0 = s_x + dM;

    // 3. phi at time n on the stencil (staged rows)
    auto phi = [&](int dy, int dz, int xx) {
      float e = E(dy, dz, xx);
      if (tv) e = fmaf(dn, Dd(dy, dz, xx), e);
      return e;
    };
    const float e_c = phi(0, 0, x);
    const float e_xp = phi(0, 0, xp), e_xm = phi(0, 0, xm);
    const float e_yp = phi(1, 0, x), e_ym = phi(-1, 0, x);
    float e_zp = e_c, e_zm = e_c;
    if (D == 3) {
      e_zp = phi(0, 1, x);
      e_zm = phi(0, -1, x);
    }

    // 4.-6. quadrature, density, forces, velocity
    const unsigned qa = L.quad_axes;
    float nb = 0.f;
    if (qa & 1u) nb += e_xp + e_xm;
    if (qa & 2u) nb += e_yp + e_ym;
    if (qa & 4u) nb += e_zp + e_zm;
    const float I = (float)L.qw0 * e_c + (float)L.qw1 * nb;
    const float rho = M0 / I;
    const float pc = rho * (1.0f / 3.0f);
    float F0 = (float)L.g[0] + pc * 0.5f * (e_xp - e_xm);
    float F1 = (float)L.g[1] + pc * 0.5f * (e_yp - e_ym);
    float F2 = D == 3 ? (float)L.g[2] + pc * 0.5f * (e_zp - e_zm) : 0.f;
    if (L.has_force) {
      const float *__restrict__ fo = static_cast<const float *>(L.force);
      const long long N = L.ncell;
      float a0 = __ldg(fo + cell), a1 = __ldg(fo + N + cell), a2 = D == 3 ? __ldg(fo + 2 * N + cell) : 0.f;
      if (L.has_dforce) {
        const float *__restrict__ df = static_cast<const float *>(L.dforce);
        const float dnf = (float)(n - L.n_force);
        a0 = fmaf(dnf, __ldg(df + cell), a0);
        a1 = fmaf(dnf, __ldg(df + N + cell), a1);
        if (D == 3) a2 = fmaf(dnf, __ldg(df + 2 * N + cell), a2);
      }
      F0 += a0;
      F1 += a1;
      F2 += a2;
    }
    const float invM = 1.0f / M0;
    const float u0 = (j0 + 0.5f * F0) * invM;
    const float u1 = (j1 + 0.5f * F1) * invM;
    const float u2 = D == 3 ? (j2 + 0.5f * F2) * invM : 0.f;
    const float usq = u0 * u0 + u1 * u1 + u2 * u2;
    const float uF = u0 * F0 + u1 * F1 + u2 * F2;

    if (RED) {
      const double m0 = (double)M0;
      acc.v[0] += m0;
      acc.v[1] += m0 * (double)u0;
      acc.v[2] += m0 * (double)u1;
      acc.v[3] += m0 * (double)u2;
      acc.v[5] += (double)usq;
      if (L.u_prev) {
        float *up = L.u_prev;
        const long long N = L.ncell;
        if (L.have_prev) {
          const double a = (double)u0 - (double)up[cell];
          const double b = (double)u1 - (double)up[N + cell];
          const double c = (double)u2 - (double)up[2 * N + cell];
          acc.v[4] += a * a + b * b + c * c;
        }
        up[cell] = u0;
        up[N + cell] = u1;
        up[2 * N + cell] = u2;
      }
      if (!isfinite(M0) || !isfinite(usq)) acc.v[6] += 1.0;
      acc.v[7] += (double)F0;
      acc.v[8] += (double)F1;
      acc.v[9] += (double)F2;
    }

    // 7.-8. collide and stream; the new shift is phi_ref (staged)
    const float omega = (float)L.omega, cf = (float)L.cf;
    const float s_new_x = rho0 * E(0, 0, x);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      float cu = 0.f, cF = 0.f;
      if (cx == 1) { cu += u0; cF += F0; }
      if (cx == -1) { cu -= u0; cF -= F0; }
      if (cy == 1) { cu += u1; cF += F1; }
      if (cy == -1) { cu -= u1; cF -= F1; }
      if (cz == 1) { cu += u2; cF += F2; }
      if (cz == -1) { cu -= u2; cF -= F2; }
      const float pm1 = cu * fmaf(4.5f, cu, 3.0f) - 1.5f * usq;
      const float deq = fmaf(M0, pm1, dM);
      const float src = cf * fmaf(9.0f * cu, cF, 3.0f * (cF - uF));
      // d*_i = f*_i/w_i - s_x, re-encoded against the storage cell's new
      // shift by adding the (small) shift difference, never by subtracting
      // two O(1) numbers
      const float dstar = fmaf(omega, deq - d[i], d[i]) + src;
      if (!ODD || i == 0) {
        PopIO<ST>::st(pop + (long long)opp_of(i) * plane + cell, (dstar + (s_x - s_new_x)) * scale);
      } else if (walls && row_solid(L, ys_[1 + cy], zs_[1 + cz])) {
        PopIO<ST>::st(pop + (long long)opp_of(i) * plane + cell, (dstar + (s_x - s_new_x)) * scale);
      } else {
        const int m = (zs_[1 + cz] * ny + ys_[1 + cy]) * nx + xs[1 + cx];
        const float s_m = rho0 * E(cy, cz, xs[1 + cx]);
        PopIO<ST>::st(pop + (long long)i * plane + m, (dstar + (s_x - s_m)) * scale);
      }
    }
  }
}

template <class LAT, class ST, bool ODD, bool RED, int MINB>
__global__ void __launch_bounds__(kRowThreads, MINB) step_row_kernel(const LatticeDev *__restrict__ Lp, int k) {
  constexpr int NSTAGE = 2;
  __shared__ LatticeDev Ls;
  __shared__ alignas(8) unsigned long long bars[NSTAGE];
  __shared__ int s_abort;
  extern __shared__ __align__(128) unsigned char stages[];
  const int tid = threadIdx.x;
  {
    const int *src = reinterpret_cast<const int *>(Lp);
    int *dst = reinterpret_cast<int *>(&Ls);
    for (int w = tid; w < (int)(sizeof(LatticeDev) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    s_abort = 0;
  }
  __syncthreads();
  const LatticeDev &L = Ls;
  const RowLayout lay = row_layout<LAT, ST, ODD>(L.nx, L.has_deps != 0);
  const RowGeom gm = row_geom(L);
  const int nrows = gm.nyf * gm.nzf;
  const long long n = L.n + k;
  RedAcc acc;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) acc.v[j] = 0.0;

  auto row_yz = [&](int r, int &y, int &z) {
    y = gm.y0 + r % gm.nyf;
    z = gm.z0 + r / gm.nyf;
  };
  // prologue: rows of the first NSTAGE-1 iterations
  if (tid == 0) {
    for (int j = 0; j < NSTAGE - 1; ++j) {
      const int r = blockIdx.x + j * gridDim.x;
      if (r < nrows) {
        int y, z;
        row_yz(r, y, z);
        issue_row<LAT, ST, ODD>(L, lay, stages + j * lay.stage_bytes, &bars[j], y, z);
      }
    }
  }
  int it = 0;
  for (int r = blockIdx.x; r < nrows; r += gridDim.x, ++it) {
    const int s = it % NSTAGE;
    if (tid == 0) {
      const int rn = r + (NSTAGE - 1) * gridDim.x;
      const int sn = (it + NSTAGE - 1) % NSTAGE;
      if (rn < nrows) {
        int y, z;
        row_yz(rn, y, z);
        issue_row<LAT, ST, ODD>(L, lay, stages + sn * lay.stage_bytes, &bars[sn], y, z);
      }
    }
    const bool ok = mbar_wait_bounded(&bars[s], (unsigned)((it / NSTAGE) & 1), L.wait_limit);
    if (__syncthreads_or(!ok)) {
      // a copy never completed: record it, drain what is in flight, leave
      if (tid == 0) {
        atomicExch(L.status, 1);
        for (int j = 0; j < NSTAGE; ++j) {
          const int rj = r + j * gridDim.x;
          if (rj < nrows) mbar_wait_bounded(&bars[(it + j) % NSTAGE], (unsigned)(((it + j) / NSTAGE) & 1));
        }
      }
      __syncthreads();
      return;
    }
    int y, z;
    row_yz(r, y, z);
    update_row_cells<LAT, ST, ODD, RED>(L, lay, stages + s * lay.stage_bytes, n, y, z, acc);
    __syncthreads();  // every thread is done with stage s before it is refilled
  }
  if (RED) block_reduce_store(acc, L.partials, blockIdx.x);
}

}  // namespace lbm

namespace lbm {

// Host side: launch and planning of the row kernel for one lattice type.
template <class LAT, class ST, int MINB>
cudaError_t launch_row_t(const LatticeDev *L_dev, bool odd, int red, int k, const StepLaunch &ls,
                         cudaStream_t s) {
  const int smem = odd ? ls.row_smem_odd : ls.row_smem_even;
  const dim3 grid(ls.row_grid), block(kRowThreads);
  if (odd) {
    if (red) step_row_kernel<LAT, ST, true, true, MINB><<<grid, block, smem, s>>>(L_dev, k);
    else step_row_kernel<LAT, ST, true, false, MINB><<<grid, block, smem, s>>>(L_dev, k);
  } else {
    if (red) step_row_kernel<LAT, ST, false, true, MINB><<<grid, block, smem, s>>>(L_dev, k);
    else step_row_kernel<LAT, ST, false, false, MINB><<<grid, block, smem, s>>>(L_dev, k);
  }
  return cudaGetLastError();
}

template <class LAT, class ST, int MINB>
int plan_row_t(int nx, int ny, int nz, unsigned walls, StepLaunch &ls) {
  constexpr int kMaxSmem = 200 * 1024;
  if (nx % 4 != 0 || (nx * (int)sizeof(ST)) % 16 != 0 || nx > 512 || nx < 32) return 0;
  if (walls & 1u) return 0;
  const int smem_odd = 2 * row_layout<LAT, ST, true>(nx, true).stage_bytes;
  const int smem_even = 2 * row_layout<LAT, ST, false>(nx, true).stage_bytes;
  if (smem_odd > kMaxSmem) return 0;
  if (cudaFuncSetAttribute(step_row_kernel<LAT, ST, true, false, MINB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_odd) != cudaSuccess ||
      cudaFuncSetAttribute(step_row_kernel<LAT, ST, true, true, MINB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_odd) != cudaSuccess ||
      cudaFuncSetAttribute(step_row_kernel<LAT, ST, false, false, MINB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_odd) != cudaSuccess ||
      cudaFuncSetAttribute(step_row_kernel<LAT, ST, false, true, MINB>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, smem_odd) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_row_kernel<LAT, ST, true, false, MINB>,
                                                    kRowThreads, smem_odd) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return 0;
  }
  const int nyf = (walls & 2u) ? ny - 2 : ny;
  const int nzf = (walls & 4u) ? nz - 2 : nz;
  const int nrows = nyf * nzf;
  if (nrows < 1) return 0;
  const int cap = sm_count() * occ;
  ls.row = 1;
  ls.row_grid = nrows < cap ? nrows : cap;
  ls.row_smem_odd = smem_odd;
  ls.row_smem_even = smem_even;
  return 1;
}

}  // namespace lbm
