// step_fast.cuh -- fused collide-and-stream step of the consistent VANSE
// lattice Boltzmann scheme, FP32 arithmetic on FP32 or FP16 storage.
//
// One thread updates one cell (Sec. 2.2):
//   1. load the Q populations of time n (AA pattern, see below) and decode
//      them into per-weight deviations d_i = f_i/w_i - s_x from the cell's
//      shift s_x = rho0 sigma(x);
//   2. zeroth and first moments: M0 = s_x + sum w_i d_i, J = sum w_i xi_i d_i;
//   3. phi at time n on the cell and its face neighbours,
//      phi_n = phi_ref + (n - n_ref) d_t phi;
//   4. eq. (quad): I = varpi_0 phi(x) + varpi_1 sum over the quadrature
//      axes of phi(x +- e_a);  eq. (density): rho~ = M0 / I;
//   5. eq. (pressForce): F = F_ext + c_s^2 rho~ grad_h phi, central
//      differences on every lattice axis;
//   6. eq. (velocity): u = (J + F/2) / M0;
//   7. BGK with the equilibrium of eq. (feq) (M0 in place of rho~ phi) and
//      the Guo term, in deviation form:
//        f^eq_i/w_i - s_x = dM + M0 (3 cu + 4.5 cu^2 - 1.5 u.u),
//        Omega_i/w_i = (1 - 1/(2 tau)) (3 (xi.F - u.F) + 9 (xi.u)(xi.F)),
//        d*_i = d_i + (d^eq_i - d_i)/tau + Omega_i/w_i;
//   8. encode against the shift of the slot's storage cell and store; FP32
//      stores the rest population last, with the value that keeps the mass
//      of the stored values (the zeroth moment) exactly balanced.
//
// AA pattern (in place, one array): at even n a cell reads its own slots i
// and writes f*_i to its own slot opp(i); at odd n it reads slot opp(i) of
// x - xi_i and writes slot i of x + xi_i.  Halfway bounce-back: at odd n a
// population whose source x - xi_i is solid is read from the cell's own
// slot i, and one whose target x + xi_i is solid is written to the cell's
// own slot opp(i).  Even steps never touch a neighbour.
//
// The shift of a stored value is that of the cell whose memory holds it
// (sigma_rd when read, sigma_wr when written), so only differences of
// sigma between neighbours enter the decode/encode, keeping the stored
// deviations small (the point of the reduced-precision storage).
#pragma once

#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"

namespace lbm {

template <class ST>
struct PopIO;

template <>
struct PopIO<float> {
  static __device__ __forceinline__ float ld(const float *p) { return *p; }
  static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};

template <>
struct PopIO<__half> {
  static __device__ __forceinline__ float ld(const __half *p) { return __half2float(*p); }
  static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};

// Stochastic rounding of the FP16 stores.  A stored deviation can be many
// times larger than its per-step change (a slowly accelerated flow changes
// u by O(g) per step); round-to-nearest then drops the change every step, a
// bias that accumulates.  Rounding up with probability equal to the
// discarded fraction keeps every stored value unbiased.  The random bits
// come from a counter-based generator keyed by (cell, time step), so runs
// are reproducible and independent of how cells are grouped into launches.
struct SRng {
  unsigned s;
  __device__ __forceinline__ explicit SRng(unsigned cell, long long n) {
    unsigned x = cell * 0x9E3779B9u ^ (unsigned)n * 0x85EBCA6Bu ^ (unsigned)(n >> 32);
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    s = x;
  }
  // 13 random bits: the float mantissa bits that a half does not keep
  __device__ __forceinline__ unsigned next13() {
    s = s * 1664525u + 1013904223u;
    return s >> 19;
  }
  // 32 random bits (the low half mixed with the high half: an LCG's low
  // bits alone repeat with short periods)
  __device__ __forceinline__ unsigned next32() {
    s = s * 1664525u + 1013904223u;
    return s ^ (s >> 16);
  }
};

// Two values rounded stochastically to half in one conversion (the
// conversion adds random bits below the kept mantissa and truncates, as
// half_sr does; 16 random bits per value): lo in the low half of the
// result, hi in the high half.
__device__ __forceinline__ unsigned half2_sr(float lo, float hi, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}

// v rounded stochastically to half: add random bits below the half
// mantissa to the float's magnitude, then truncate toward zero.
__device__ __forceinline__ __half half_sr(float v, unsigned r13) {
  return __float2half_rz(__uint_as_float(__float_as_uint(v) + r13));
}

template <class ST>
__device__ __forceinline__ void store_pop(ST *p, float v, SRng &rng, bool sr) {
  PopIO<ST>::st(p, v);
}

template <>
__device__ __forceinline__ void store_pop<__half>(__half *p, float v, SRng &rng, bool sr) {
  *p = sr ? half_sr(v, rng.next13()) : __float2half_rn(v);
}

// Store two populations (the members of an opposite pair) to their slots.
template <class ST>
__device__ __forceinline__ void store_pop_pair(ST *pa, float va, ST *pb, float vb, SRng &rng, bool sr) {
  PopIO<ST>::st(pa, va);
  PopIO<ST>::st(pb, vb);
}

template <>
__device__ __forceinline__ void store_pop_pair<__half>(__half *pa, float va, __half *pb, float vb, SRng &rng,
                                                       bool sr) {
  if (sr) {
    const unsigned h = half2_sr(va, vb, rng.next32());
    *pa = __ushort_as_half((unsigned short)(h & 0xffffu));
    *pb = __ushort_as_half((unsigned short)(h >> 16));
  } else {
    *pa = __float2half_rn(va);
    *pb = __float2half_rn(vb);
  }
}

struct Coords {
  int xs[3], ys[3], zs[3];  // coordinate of offset -1, 0, +1 (periodic)
  int nxp, ny;              // row pitch, rows per plane
  __device__ __forceinline__ long long at(int cx, int cy, int cz) const {
    return ((long long)zs[cz + 1] * ny + ys[cy + 1]) * nxp + xs[cx + 1];
  }
};

__device__ __forceinline__ Coords make_coords(int x, int y, int z, int nx, int ny, int nz, int nxp) {
  Coords c;
  c.nxp = nxp;
  c.ny = ny;
  c.xs[0] = x == 0 ? nx - 1 : x - 1;
  c.xs[1] = x;
  c.xs[2] = x == nx - 1 ? 0 : x + 1;
  c.ys[0] = y == 0 ? ny - 1 : y - 1;
  c.ys[1] = y;
  c.ys[2] = y == ny - 1 ? 0 : y + 1;
  c.zs[0] = z == 0 ? nz - 1 : z - 1;
  c.zs[1] = z;
  c.zs[2] = z == nz - 1 ? 0 : z + 1;
  return c;
}

// Is the cell at offset (cx,cy,cz) from (x,y,z) in a wall layer?
__device__ __forceinline__ bool solid_at(unsigned walls, int x, int y, int z, int cx, int cy,
                                         int cz, int nx, int ny, int nz) {
  const int X = x + cx, Y = y + cy, Z = z + cz;
  return ((walls & 1u) && (X <= 0 || X >= nx - 1)) || ((walls & 2u) && (Y <= 0 || Y >= ny - 1)) ||
         ((walls & 4u) && (Z <= 0 || Z >= nz - 1));
}

// Per-thread accumulators of a check step.
struct RedAcc {
  double v[kRedWidth];
};

// first: this step is the first since the descriptor's shifts were last
// committed (a pending refresh applies to it only); the batched kernels,
// which commit after a replay of several steps, pass false after the first.
template <class LAT, class ST, bool ODD, bool RED>
__device__ __forceinline__ void update_cell_fast(const LatticeDev &L, long long n, int x, int y,
                                                 int z, RedAcc &acc, bool first = true) {
  constexpr int Q = LAT::Q;
  constexpr int D = LAT::D;
  const int nx = L.nx, ny = L.ny, nz = L.nz;
  const unsigned walls = L.walls;
  if (walls && solid_at(walls, x, y, z, 0, 0, 0, nx, ny, nz)) return;

  const Coords C = make_coords(x, y, z, nx, ny, nz, L.nxp);
  const long long cell = C.at(0, 0, 0);
  const long long plane = L.plane;
  ST *__restrict__ pop = static_cast<ST *>(L.pop);
  const __half *__restrict__ swr = L.sig_wr;
  const __half *__restrict__ srd = first ? L.sig_rd : swr;
  const float rho0 = L.rho0f;
  const float inv_scale = L.inv_scale, scale = L.scale;
  const float s_x = rho0 * __half2float(srd[cell]);

  // 1. load and decode.  FP32 keeps the stored values q_i as read for the
  //    mass balance of step 8, and after a phi refresh the difference of the
  //    read and write shifts of the slots it reads.
  constexpr bool kMassFix = sizeof(ST) == 4;
  const bool reshift = srd != swr;
  float d[Q], qraw[Q];
  float frame = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    if (!ODD || i == 0 || (walls && solid_at(walls, x, y, z, -cx, -cy, -cz, nx, ny, nz))) {
      qraw[i] = PopIO<ST>::ld(pop + (long long)i * plane + cell);
      d[i] = qraw[i] * inv_scale;
      if (kMassFix && reshift) frame = fmaf((float)LAT::w(i), fmaf(-rho0, __half2float(swr[cell]), s_x), frame);
    } else {
      const long long m = C.at(-cx, -cy, -cz);
      qraw[i] = PopIO<ST>::ld(pop + (long long)opp_of(i) * plane + m);
      const float sm = __half2float(srd[m]);
      d[i] = fmaf(qraw[i], inv_scale, fmaf(rho0, sm, -s_x));
      if (kMassFix && reshift)
        frame = fmaf((float)LAT::w(i), rho0 * (sm - __half2float(swr[m])), frame);
    }
  }

  // 2. moments in deviation form
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

  // 3. phi at time n on the 2D+1 stencil
  const float *__restrict__ eps = static_cast<const float *>(L.eps);
  const float *__restrict__ deps = static_cast<const float *>(L.deps);
  const bool tv = L.has_deps != 0;
  const float dn = (float)(n - L.n_eps);
  auto phi = [&](long long m) {
    float e = __ldg(eps + m);
    if (tv) e = fmaf(dn, __ldg(deps + m), e);
    return e;
  };
  const float e_c = phi(cell);
  const float e_xp = phi(C.at(1, 0, 0)), e_xm = phi(C.at(-1, 0, 0));
  const float e_yp = phi(C.at(0, 1, 0)), e_ym = phi(C.at(0, -1, 0));
  float e_zp = e_c, e_zm = e_c;
  if (D == 3) {
    e_zp = phi(C.at(0, 0, 1));
    e_zm = phi(C.at(0, 0, -1));
  }

  // 4. eq. (quad) and eq. (density)
  const unsigned qa = L.quad_axes;
  float nb = 0.f;
  if (qa & 1u) nb += e_xp + e_xm;
  if (qa & 2u) nb += e_yp + e_ym;
  if (qa & 4u) nb += e_zp + e_zm;
  const float I = L.qw0f * e_c + L.qw1f * nb;
  const float rho = M0 / I;

  // 5. eq. (pressForce) plus the external force density
  const float pc = rho * (1.0f / 3.0f);
  float F0 = L.gf[0] + pc * 0.5f * (e_xp - e_xm);
  float F1 = L.gf[1] + pc * 0.5f * (e_yp - e_ym);
  float F2 = D == 3 ? L.gf[2] + pc * 0.5f * (e_zp - e_zm) : 0.f;
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

  // 6. eq. (velocity)
  float invM = 1.0f / M0;
  if (L.drag_model) {
    // phase-interaction drag F_D = -(b_lin + b_q |u|) u (Ergun-type law of a
    // fixed bed), implicit in eq. (velocity): with b = J + F/2 the speed s =
    // |u| is the positive root of (b_q/2) s^2 + (M0 + b_lin/2) s - |b| = 0
    // and u = b / (M0 + b_lin/2 + b_q s/2); F_D joins the force sum
    const float one_m = 1.0f - e_c;
    const float blin = rho * L.drag_linf * one_m * one_m / e_c;
    const float bq = rho * L.drag_qf * one_m;
    const float b0 = fmaf(0.5f, F0, j0), b1 = fmaf(0.5f, F1, j1), b2 = D == 3 ? fmaf(0.5f, F2, j2) : 0.f;
    const float bn = sqrtf(fmaf(b0, b0, fmaf(b1, b1, b2 * b2)));
    const float A = fmaf(0.5f, blin, M0);
    const float sp = 2.0f * bn / (A + sqrtf(fmaf(A, A, 2.0f * bq * bn)));
    invM = 1.0f / fmaf(0.5f * bq, sp, A);
    const float beta = fmaf(bq, sp, blin);
    F0 = fmaf(-beta * b0, invM, F0);
    F1 = fmaf(-beta * b1, invM, F1);
    if (D == 3) F2 = fmaf(-beta * b2, invM, F2);
    // then (J + F/2) / M0 = b / (A + b_q s/2): the velocity below
    invM = 1.0f / M0;
  }
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

  // 7. collide (deviation form) and 8. stream.  d*_i = d_i + (omega (d^eq_i
  //    - d_i) + Omega_i/w_i): one rounding at the size of d_i.  FP32 then
  //    balances the mass of the stored values through the rest population,
  //    stored last: every slot the cell reads is a slot it writes (AA
  //    pattern), so w_0 V_0 = w_0 q_0 + sum_{i>0} w_i (q_i - V_i) + frame
  //    conserves the zeroth moment of the stored state up to one rounding.
  float omega = L.omegaf, cf = L.cff;
  if (L.les) {
    // Smagorinsky closure: tau_eff = (tau + sqrt(tau^2 + 18 sqrt(2) C^2
    // |Pi^neq| / M0)) / 2 with Pi^neq_ab = sum_i xi_ia xi_ib (f_i - f_i^eq);
    // in deviation form f_i - f_i^eq = w_i (d_i - d^eq_i)
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      float cu = 0.f;
      if (cx == 1) cu += u0;
      if (cx == -1) cu -= u0;
      if (cy == 1) cu += u1;
      if (cy == -1) cu -= u1;
      if (cz == 1) cu += u2;
      if (cz == -1) cu -= u2;
      const float deq = fmaf(M0, fmaf(cu, fmaf(4.5f, cu, 3.0f), -1.5f * usq), dM);
      const float fn = (float)LAT::w(i) * (d[i] - deq);
      if (cx) pxx += fn;
      if (cy) pyy += fn;
      if (cz) pzz += fn;
      if (cx && cy) pxy = fmaf((float)(cx * cy), fn, pxy);
      if (cx && cz) pxz = fmaf((float)(cx * cz), fn, pxz);
      if (cy && cz) pyz = fmaf((float)(cy * cz), fn, pyz);
    }
    const float q = sqrtf(fmaf(pxx, pxx, fmaf(pyy, pyy, fmaf(pzz, pzz, 2.0f * fmaf(pxy, pxy, fmaf(pxz, pxz, pyz * pyz))))));
    const float t0 = L.tau0f;
    const float teff = 0.5f * (t0 + sqrtf(fmaf(t0, t0, L.les_cf * q / M0)));
    omega = 1.0f / teff;
    cf = 1.0f - 0.5f / teff;
  }
  SRng rng((unsigned)cell, n);
  const bool sr = L.fp16_nearest == 0;
  float R = frame;
#pragma unroll
  for (int ii = 1; ii <= Q; ++ii) {
    const int i = ii == Q ? 0 : ii;
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    float cu = 0.f, cF = 0.f;
    if (cx == 1) { cu += u0; cF += F0; }
    if (cx == -1) { cu -= u0; cF -= F0; }
    if (cy == 1) { cu += u1; cF += F1; }
    if (cy == -1) { cu -= u1; cF -= F1; }
    if (cz == 1) { cu += u2; cF += F2; }
    if (cz == -1) { cu -= u2; cF -= F2; }
    const float pm1 = fmaf(cu, fmaf(4.5f, cu, 3.0f), -1.5f * usq);
    const float deq = fmaf(M0, pm1, dM);
    const float src = cf * fmaf(9.0f * cu, cF, 3.0f * (cF - uF));
    const float ds = d[i] + fmaf(omega, deq - d[i], src);
    // the shift difference uses the exact product rho0*sigma (FMA) exactly
    // as the decode does, so that a stored value round-trips
    ST *slot;
    float q;
    if (!ODD || i == 0 || (walls && solid_at(walls, x, y, z, cx, cy, cz, nx, ny, nz))) {
      q = ds;
      if (reshift) q += fmaf(-rho0, __half2float(swr[cell]), s_x);
      slot = pop + (long long)opp_of(i) * plane + cell;
    } else {
      const long long m = C.at(cx, cy, cz);
      q = ds + fmaf(-rho0, __half2float(swr[m]), s_x);
      slot = pop + (long long)i * plane + m;
    }
    float v = q;
    if (kMassFix) {
      // FP32 (scale 1): the stored value is q itself
      if (i != 0) R = fmaf((float)LAT::w(i), qraw[i] - q, R);
      else v = fmaf(R, (float)(1.0 / LAT::w(0)), qraw[0]);
    }
    store_pop<ST>(slot, v * scale, rng, sr);
  }
}

// Sum a thread's accumulators over the block and write them to
// partials[block * kRedWidth + j] (fixed order, no atomics).
__device__ __forceinline__ void block_reduce_store(RedAcc &acc, double *partials, long long block) {
  __shared__ double sm[32][kRedWidth];
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) {
    double v = acc.v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sm[warp][j] = v;
  }
  __syncthreads();
  if (tid < kRedWidth) {
    double s = 0.0;
    const int nw = (nthreads + 31) >> 5;
    for (int w = 0; w < nw; ++w) s += sm[w][tid];
    partials[block * kRedWidth + tid] = s;
  }
}

template <class LAT, class ST, bool ODD, bool RED>
__global__ void __launch_bounds__(256) step_fast_kernel(const LatticeDev *__restrict__ Lp, int k) {
  const LatticeDev &L = *Lp;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  RedAcc acc;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) acc.v[j] = 0.0;
  if (x < L.nx && y < L.ny) update_cell_fast<LAT, ST, ODD, RED>(L, L.n + k, x, y, z, acc);
  if (RED) {
    const long long b = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
    block_reduce_store(acc, L.partials, b);
  }
}

}  // namespace lbm
