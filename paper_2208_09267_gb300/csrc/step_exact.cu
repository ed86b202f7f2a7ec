// step_exact.cu -- FP64 step in the canonical evaluation order, and the FP64
// moment / initialisation / population kernels of every storage.
//
// This translation unit is compiled with -fmad=false: no multiply-add is
// fused, so every operation below rounds exactly as written.  The order is
// the canonical one of the method (Sec. 2.2), shared by the FP64 reference:
//   M0 = sum_i f_i and J_a = sum_i xi_ia f_i in ascending i from 0.0;
//   phi_n = phi_ref + (n - n_ref) d_t phi;
//   nb = sum over quadrature axes a of (phi(x+e_a) then phi(x-e_a)) from 0.0;
//   I = varpi_0 phi(x) + varpi_1 nb                           (eq. (quad))
//   rho~ = M0 / I                                             (eq. (density))
//   F_a = (g_a + field_a) + (rho~/3) (0.5 (phi(x+e_a) - phi(x-e_a)))
//                                                             (eq. (pressForce))
//   u_a = (J_a + 0.5 F_a) / M0                                (eq. (velocity))
//   usq = u0 u0 + u1 u1 + u2 u2, uF = u0 F0 + u1 F1 + u2 F2;
//   cu = sum_a xi_ia u_a, cF = sum_a xi_ia F_a from 0.0;
//   f^eq = (w_i M0)(((1 + 3 cu) + (4.5 cu) cu) - 1.5 usq)     (eq. (feq))
//   S = ((1 - 0.5/tau) w_i)((3 (cF - uF)) + (9 cu) cF)        (Guo term)
//   f* = (f + (1/tau)(f^eq - f)) + S                          (eq. (lbe))
// With that order the FP64 result is bit-identical to the reference.
#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"
#include "step_fast.cuh"

namespace lbm {

// Address (slot, cell) holding f_i(x, n) at the parity of n, AA pattern.
struct SlotAddr {
  int slot;
  long long cell;
};

template <class LAT>
__device__ __forceinline__ SlotAddr slot_of(const LatticeDev &L, const Coords &C, bool odd_layout,
                                            int i, int x, int y, int z) {
  SlotAddr a;
  const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
  if (!odd_layout || i == 0) {
    a.slot = i;
    a.cell = C.at(0, 0, 0);
  } else if (L.walls && solid_at(L.walls, x, y, z, -cx, -cy, -cz, L.nx, L.ny, L.nz)) {
    a.slot = i;
    a.cell = C.at(0, 0, 0);
  } else {
    a.slot = opp_of(i);
    a.cell = C.at(-cx, -cy, -cz);
  }
  return a;
}

// Read f_i(x, n) of any storage as a double.
template <class LAT>
__device__ __forceinline__ double load_f(const LatticeDev &L, const SlotAddr &a, int i) {
  const long long off = (long long)a.slot * L.plane + a.cell;
  if (L.storage == 0) return static_cast<const double *>(L.pop)[off];
  double q = L.storage == 1 ? (double)static_cast<const float *>(L.pop)[off]
                            : (double)__half2float(static_cast<const __half *>(L.pop)[off]);
  const double s = L.rho0 * (double)__half2float(L.sig_rd[a.cell]);
  return LAT::w(i) * (s + q * (double)L.inv_scale);
}

// Write f_i to a slot of any storage (encoding against sigma_wr).
template <class LAT>
__device__ __forceinline__ void store_f(const LatticeDev &L, int slot, long long cell, int i, double f) {
  const long long off = (long long)slot * L.plane + cell;
  if (L.storage == 0) {
    static_cast<double *>(L.pop)[off] = f;
    return;
  }
  const double s = L.rho0 * (double)__half2float(L.sig_wr[cell]);
  const double q = (f / LAT::w(i) - s) * (double)L.scale;
  if (L.storage == 1)
    static_cast<float *>(L.pop)[off] = (float)q;
  else
    static_cast<__half *>(L.pop)[off] = __double2half(q);
}

struct MacroD {
  double M0, J[3], I, rho, F[3], u[3];
};

template <class LAT>
__device__ __forceinline__ double eps_at(const LatticeDev &L, long long m, double dn) {
  if (L.storage == 0) {
    const double *e = static_cast<const double *>(L.eps);
    if (L.has_deps) return e[m] + dn * static_cast<const double *>(L.deps)[m];
    return e[m];
  }
  const float *e = static_cast<const float *>(L.eps);
  if (L.has_deps) return (double)e[m] + dn * (double)static_cast<const float *>(L.deps)[m];
  return (double)e[m];
}

template <class LAT>
__device__ __forceinline__ double force_at(const LatticeDev &L, int a, long long k, double dnf) {
  const long long off = (long long)a * L.ncell + k;
  if (L.storage == 0) {
    double fa = static_cast<const double *>(L.force)[off];
    if (L.has_dforce) fa = fa + dnf * static_cast<const double *>(L.dforce)[off];
    return fa;
  }
  double fa = (double)static_cast<const float *>(L.force)[off];
  if (L.has_dforce) fa = fa + dnf * (double)static_cast<const float *>(L.dforce)[off];
  return fa;
}

template <class LAT>
__device__ __forceinline__ void macro_exact(const LatticeDev &L, long long n, const Coords &C,
                                            const double *f, MacroD &m) {
  constexpr int Q = LAT::Q, D = LAT::D;
  m.M0 = 0.0;
#pragma unroll
  for (int i = 0; i < Q; ++i) m.M0 = m.M0 + f[i];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m.J[a] = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) m.J[a] = m.J[a] + (double)LAT::c(i, a) * f[i];
  }
  const double dn = (double)(n - L.n_eps);
  const double e_c = eps_at<LAT>(L, C.at(0, 0, 0), dn);
  double e_p[3], e_m[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < D) {
      e_p[a] = eps_at<LAT>(L, C.at(a == 0, a == 1, a == 2), dn);
      e_m[a] = eps_at<LAT>(L, C.at(-(a == 0), -(a == 1), -(a == 2)), dn);
    } else {
      e_p[a] = e_c;
      e_m[a] = e_c;
    }
  }
  double nb = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (L.quad_axes & (1u << a)) {
      nb = nb + e_p[a];
      nb = nb + e_m[a];
    }
  }
  m.I = L.qw0 * e_c + L.qw1 * nb;
  m.rho = m.M0 / m.I;
  const double pc = m.rho / 3.0;
  const double dnf = (double)(n - L.n_force);
  const long long k = C.at(0, 0, 0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double grad = 0.5 * (e_p[a] - e_m[a]);
    double fext = L.g[a];
    if (L.has_force) fext = fext + force_at<LAT>(L, a, k, dnf);
    m.F[a] = (a < D) ? fext + pc * grad : 0.0;
  }
  if (!L.drag_model) {
#pragma unroll
    for (int a = 0; a < 3; ++a) m.u[a] = (m.J[a] + 0.5 * m.F[a]) / m.M0;
    return;
  }
  // phase-interaction drag F_D = -(b_lin + b_q |u|) u (Ergun-type law of a
  // fixed bed, Sec. 2.2's force sum), implicit in eq. (velocity): with
  // b = J + F/2 the speed s = |u| is the positive root of
  // (b_q/2) s^2 + (M0 + b_lin/2) s - |b| = 0, u = b / (M0 + b_lin/2 + b_q s/2)
  const double one_m = 1.0 - e_c;
  const double nu = (L.tau0 - 0.5) / 3.0;
  const double blin = m.rho * L.drag_c1 * one_m * one_m * nu / (e_c * L.drag_d * L.drag_d);
  const double bq = m.rho * L.drag_c2 * one_m / L.drag_d;
  double b[3], bn = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    b[a] = m.J[a] + 0.5 * m.F[a];
    bn = bn + b[a] * b[a];
  }
  bn = sqrt(bn);
  const double A = m.M0 + 0.5 * blin;
  const double sp = 2.0 * bn / (A + sqrt(A * A + 2.0 * bq * bn));
  const double den = A + 0.5 * bq * sp;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m.u[a] = b[a] / den;
    const double fd = (blin + bq * sp) * m.u[a];
    m.F[a] = (a < D) ? m.F[a] - fd : 0.0;
  }
}

template <class LAT>
__device__ __forceinline__ double feq_exact(int i, double M0, const double *u, double usq) {
  double cu = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) cu = cu + (double)LAT::c(i, a) * u[a];
  return LAT::w(i) * M0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
}

template <class LAT>
__device__ __forceinline__ double guo_exact(int i, double cf, const double *u, const double *F,
                                            double uF) {
  double cu = 0.0, cF = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) cu = cu + (double)LAT::c(i, a) * u[a];
#pragma unroll
  for (int a = 0; a < 3; ++a) cF = cF + (double)LAT::c(i, a) * F[a];
  return cf * LAT::w(i) * (3.0 * (cF - uF) + 9.0 * cu * cF);
}

// ---- FP64 step --------------------------------------------------------------

template <class LAT, bool ODD, bool RED>
__global__ void __launch_bounds__(256) step_exact_kernel(const LatticeDev *__restrict__ Lp, int k) {
  constexpr int Q = LAT::Q;
  const LatticeDev &L = *Lp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  RedAcc acc;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) acc.v[j] = 0.0;
  const bool inside = x < L.nx && y < L.ny;
  const bool fluid = inside && !(L.walls && solid_at(L.walls, x, y, z, 0, 0, 0, L.nx, L.ny, L.nz));
  if (fluid) {
    const long long n = L.n + k;
    const Coords C = make_coords(x, y, z, L.nx, L.ny, L.nz, L.nxp);
    double *pop = static_cast<double *>(L.pop);
    double f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const SlotAddr a = slot_of<LAT>(L, C, ODD, i, x, y, z);
      f[i] = pop[(long long)a.slot * L.plane + a.cell];
    }
    MacroD m;
    macro_exact<LAT>(L, n, C, f, m);
    const double usq = m.u[0] * m.u[0] + m.u[1] * m.u[1] + m.u[2] * m.u[2];
    const double uF = m.u[0] * m.F[0] + m.u[1] * m.F[1] + m.u[2] * m.F[2];
    if (RED) {
      acc.v[0] += m.M0;
      acc.v[1] += m.J[0] + 0.5 * m.F[0];
      acc.v[2] += m.J[1] + 0.5 * m.F[1];
      acc.v[3] += m.J[2] + 0.5 * m.F[2];
      acc.v[5] += usq;
      if (L.u_prev) {
        float *up = L.u_prev;
        const long long N = L.ncell, c0 = C.at(0, 0, 0);
        if (L.have_prev) {
          const double a = m.u[0] - (double)up[c0], b = m.u[1] - (double)up[N + c0],
                       c = m.u[2] - (double)up[2 * N + c0];
          acc.v[4] += a * a + b * b + c * c;
        }
        up[c0] = (float)m.u[0];
        up[N + c0] = (float)m.u[1];
        up[2 * N + c0] = (float)m.u[2];
      }
      if (!isfinite(m.M0) || !isfinite(usq)) acc.v[6] += 1.0;
      acc.v[7] += m.F[0];
      acc.v[8] += m.F[1];
      acc.v[9] += m.F[2];
    }
    double omega = L.omega, cf = L.cf;
    if (L.les) {
      // Smagorinsky closure: Pi^neq_ab = sum_i xi_ia xi_ib (f_i - f_i^eq),
      // tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2 |Pi^neq| / M0)) / 2
      double pi[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) pi[a][b] = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const double fneq = f[i] - feq_exact<LAT>(i, m.M0, m.u, usq);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) pi[a][b] = pi[a][b] + (double)LAT::c(i, a) * (double)LAT::c(i, b) * fneq;
      }
      double q2 = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) q2 = q2 + pi[a][b] * pi[a][b];
      const double teff =
          0.5 * (L.tau0 + sqrt(L.tau0 * L.tau0 + 18.0 * sqrt(2.0) * L.les_cs * L.les_cs * sqrt(q2) / m.M0));
      omega = 1.0 / teff;
      cf = 1.0 - 0.5 / teff;
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const double feq = feq_exact<LAT>(i, m.M0, m.u, usq);
      const double S = guo_exact<LAT>(i, cf, m.u, m.F, uF);
      const double fstar = f[i] + omega * (feq - f[i]) + S;
      const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      long long cell;
      int slot;
      if (!ODD || i == 0) {
        slot = opp_of(i);
        cell = C.at(0, 0, 0);
      } else if (L.walls && solid_at(L.walls, x, y, z, cx, cy, cz, L.nx, L.ny, L.nz)) {
        slot = opp_of(i);
        cell = C.at(0, 0, 0);
      } else {
        slot = i;
        cell = C.at(cx, cy, cz);
      }
      pop[(long long)slot * L.plane + cell] = fstar;
    }
  }
  if (RED) {
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_reduce_store(acc, L.partials, b);
  }
}

// ---- moments, initialisation, populations (all storages, FP64 math) ---------

template <class LAT>
__global__ void moments_kernel(const LatticeDev *__restrict__ Lp, double *rho, double *p, double *u,
                               float *rho_f, float *p_f, float *u_f) {
  constexpr int Q = LAT::Q;
  const LatticeDev &L = *Lp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const Coords C = make_coords(x, y, z, L.nx, L.ny, L.nz, L.nxp);
  // outputs are dense: index (z*ny + y)*nx + x, N = nx*ny*nz
  const long long k = ((long long)z * L.ny + y) * L.nx + x;
  const long long N = (long long)L.nx * L.ny * L.nz;
  const bool odd = (L.n & 1) != 0;
  if (L.walls && solid_at(L.walls, x, y, z, 0, 0, 0, L.nx, L.ny, L.nz)) {
    if (rho) rho[k] = 0.0;
    if (p) p[k] = 0.0;
    if (rho_f) rho_f[k] = 0.f;
    if (p_f) p_f[k] = 0.f;
    for (int a = 0; a < 3; ++a) {
      if (u) u[a * N + k] = 0.0;
      if (u_f) u_f[a * N + k] = 0.f;
    }
    return;
  }
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = load_f<LAT>(L, slot_of<LAT>(L, C, odd, i, x, y, z), i);
  MacroD m;
  macro_exact<LAT>(L, L.n, C, f, m);
  const double pv = (m.rho - L.rho0) / 3.0;
  if (rho) rho[k] = m.rho;
  if (p) p[k] = pv;
  if (rho_f) rho_f[k] = (float)m.rho;
  if (p_f) p_f[k] = (float)pv;
  for (int a = 0; a < 3; ++a) {
    if (u) u[a * N + k] = m.u[a];
    if (u_f) u_f[a * N + k] = (float)m.u[a];
  }
}

template <class LAT>
__global__ void init_kernel(const LatticeDev *__restrict__ Lp, const double *p0, const double *u0,
                            int mode) {
  constexpr int Q = LAT::Q, D = LAT::D;
  const LatticeDev &L = *Lp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  if (L.walls && solid_at(L.walls, x, y, z, 0, 0, 0, L.nx, L.ny, L.nz)) return;
  const Coords C = make_coords(x, y, z, L.nx, L.ny, L.nz, L.nxp);
  const long long k = C.at(0, 0, 0);
  // p0, u0 are dense arrays: index (z*ny + y)*nx + x, N = nx*ny*nz
  const long long kd = ((long long)z * L.ny + y) * L.nx + x;
  const long long N = (long long)L.nx * L.ny * L.nz;
  const long long n = L.n;
  const bool odd = (n & 1) != 0;
  double u[3] = {0.0, 0.0, 0.0};
  if (u0)
    for (int a = 0; a < D; ++a) u[a] = u0[a * N + kd];
  double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double rt = L.rho0 + (p0 ? 3.0 * p0[kd] : 0.0);
  const double dn = (double)(n - L.n_eps);
  double mass;
  if (mode & 1) {
    double nb = 0.0;
    for (int a = 0; a < 3; ++a) {
      if (L.quad_axes & (1u << a)) {
        nb = nb + eps_at<LAT>(L, C.at(a == 0, a == 1, a == 2), dn);
        nb = nb + eps_at<LAT>(L, C.at(-(a == 0), -(a == 1), -(a == 2)), dn);
      }
    }
    mass = rt * (L.qw0 * eps_at<LAT>(L, k, dn) + L.qw1 * nb);
  } else {
    mass = rt * eps_at<LAT>(L, k, dn);
  }
  double f[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) f[i] = feq_exact<LAT>(i, mass, u, usq);
  if (mode & 2) {
    MacroD m;
    macro_exact<LAT>(L, n, C, f, m);
    for (int a = 0; a < 3; ++a) u[a] = u[a] - 0.5 * m.F[a] / m.M0;
    usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = feq_exact<LAT>(i, mass, u, usq);
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const SlotAddr a = slot_of<LAT>(L, C, odd, i, x, y, z);
    store_f<LAT>(L, a.slot, a.cell, i, f[i]);
  }
}

template <class LAT>
__global__ void getpop_kernel(const LatticeDev *__restrict__ Lp, double *out) {
  constexpr int Q = LAT::Q;
  const LatticeDev &L = *Lp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= L.nx || y >= L.ny) return;
  const Coords C = make_coords(x, y, z, L.nx, L.ny, L.nz, L.nxp);
  const long long kd = ((long long)z * L.ny + y) * L.nx + x;  // dense output index
  const bool solid = L.walls && solid_at(L.walls, x, y, z, 0, 0, 0, L.nx, L.ny, L.nz);
  const bool odd = (L.n & 1) != 0;
#pragma unroll
  for (int i = 0; i < Q; ++i)
    out[kd * Q + i] = solid ? 0.0 : load_f<LAT>(L, slot_of<LAT>(L, C, odd, i, x, y, z), i);
}

// ---- dispatch ----------------------------------------------------------------

template <class LAT>
static cudaError_t launch_exact_lat(const LatticeDev *L_dev, bool odd, int red, int k,
                                    const StepLaunch &ls, cudaStream_t s) {
  if (odd) {
    if (red) step_exact_kernel<LAT, true, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    else step_exact_kernel<LAT, true, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
  } else {
    if (red) step_exact_kernel<LAT, false, true><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
    else step_exact_kernel<LAT, false, false><<<ls.grid, ls.block, 0, s>>>(L_dev, k);
  }
  return cudaGetLastError();
}

cudaError_t launch_step_exact(int lattice, const LatticeDev *L_dev, bool odd, int red, int k,
                              const StepLaunch &ls, cudaStream_t s) {
  switch (lattice) {
    case 0: return launch_exact_lat<D2Q9>(L_dev, odd, red, k, ls, s);
    case 1: return launch_exact_lat<D3Q19>(L_dev, odd, red, k, ls, s);
    case 2: return launch_exact_lat<D3Q27>(L_dev, odd, red, k, ls, s);
    case 3: return launch_exact_lat<D1Q3>(L_dev, odd, red, k, ls, s);
  }
  return cudaErrorInvalidValue;
}

static StepLaunch aux_launch(const LatticeDev &h) { return make_launch(h.nx, h.ny, h.nz, 0, 0); }

cudaError_t launch_moments(const LatticeDev &h, const LatticeDev *L_dev, long long, double *rho,
                           double *p, double *u, float *rho_f, float *p_f, float *u_f,
                           cudaStream_t s) {
  const StepLaunch ls = aux_launch(h);
  switch (h.lattice) {
    case 0: moments_kernel<D2Q9><<<ls.grid, ls.block, 0, s>>>(L_dev, rho, p, u, rho_f, p_f, u_f); break;
    case 1: moments_kernel<D3Q19><<<ls.grid, ls.block, 0, s>>>(L_dev, rho, p, u, rho_f, p_f, u_f); break;
    case 2: moments_kernel<D3Q27><<<ls.grid, ls.block, 0, s>>>(L_dev, rho, p, u, rho_f, p_f, u_f); break;
    case 3: moments_kernel<D1Q3><<<ls.grid, ls.block, 0, s>>>(L_dev, rho, p, u, rho_f, p_f, u_f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_init(const LatticeDev &h, const LatticeDev *L_dev, long long, const double *p0,
                        const double *u0, int mode, cudaStream_t s) {
  const StepLaunch ls = aux_launch(h);
  switch (h.lattice) {
    case 0: init_kernel<D2Q9><<<ls.grid, ls.block, 0, s>>>(L_dev, p0, u0, mode); break;
    case 1: init_kernel<D3Q19><<<ls.grid, ls.block, 0, s>>>(L_dev, p0, u0, mode); break;
    case 2: init_kernel<D3Q27><<<ls.grid, ls.block, 0, s>>>(L_dev, p0, u0, mode); break;
    case 3: init_kernel<D1Q3><<<ls.grid, ls.block, 0, s>>>(L_dev, p0, u0, mode); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_get_populations(const LatticeDev &h, const LatticeDev *L_dev, long long, double *f,
                                   cudaStream_t s) {
  const StepLaunch ls = aux_launch(h);
  switch (h.lattice) {
    case 0: getpop_kernel<D2Q9><<<ls.grid, ls.block, 0, s>>>(L_dev, f); break;
    case 1: getpop_kernel<D3Q19><<<ls.grid, ls.block, 0, s>>>(L_dev, f); break;
    case 2: getpop_kernel<D3Q27><<<ls.grid, ls.block, 0, s>>>(L_dev, f); break;
    case 3: getpop_kernel<D1Q3><<<ls.grid, ls.block, 0, s>>>(L_dev, f); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace lbm
