// step_row_pair.cuh -- the row kernel's per-cell update for two adjacent
// cells per lane, FP16-shifted storage, plain steps (no check sums, no
// pending shift change).
//
// Each operation of update_row_chunk is applied to the cells x and x + 1 at
// once as a packed FP32 pair operation (fma/add/mul .rn.f32x2: per
// component the same IEEE operation with the same rounding as the scalar
// one); divisions and the stochastic rounding stay per cell, with the same
// random bits.  So every stored value is bit-identical to update_row_chunk's
// for the same cell.  What the pair saves is issue slots: one instruction
// for two cells' arithmetic, one 4-byte shared-memory access for the two
// cells' halves of an unshifted row, and the index arithmetic done once for
// both cells.
#pragma once

#include <cuda_fp16.h>

namespace lbm {

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b, exactly as the scalar subtraction rounds it (b * -1 is exact)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2s(-1.0f), a); }

// two halves at an even index (one 4-byte load)
__device__ __forceinline__ float2 ld_h2(const __half *p) {
  return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
// two floats at an even index (one 8-byte load)
__device__ __forceinline__ float2 ld_f2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float ldh(const __half *p) { return __half2float(*p); }

// Store the low (hi = false) or high halves of the two cells' packed
// results: at the even index x (both cells, one 4-byte store) when the
// destinations are adjacent, else one by one (the second cell only if it
// exists).
__device__ __forceinline__ void st_h2(__half *row, unsigned ha, unsigned hb, bool hi, bool adjacent, int xa,
                                      int da, int db, bool vb) {
  if (adjacent) {
    *reinterpret_cast<unsigned *>(row + xa) = __byte_perm(ha, hb, hi ? 0x7632 : 0x5410);
  } else {
    row[da] = __ushort_as_half((unsigned short)(hi ? ha >> 16 : ha & 0xffffu));
    if (vb) row[db] = __ushort_as_half((unsigned short)(hi ? hb >> 16 : hb & 0xffffu));
  }
}

// Update cells xa and xa + 1 (xa even) of one staged row.  A second cell
// past the end of the row (odd nx) repeats the first one's indices; its
// results are discarded (the adjacent stores write the row's padding slot).
template <class LAT, bool ODD, bool WALLS, int PITCH, bool OUTS, bool TILED = true>
__device__ __forceinline__ void update_row_pair(const LatticeDev &L, const unsigned char *stage, int t,
                                                const RowCtx &rc, long long n, float dn, float dn_force,
                                                int xa, unsigned char *ostage) {
  using Lay = RowLayout<LAT, __half, ODD, PITCH>;
  constexpr int Q = LAT::Q, D = LAT::D;
  const int nx = L.nx;
  if (xa >= nx) return;
  const int sp = TILED ? L.nxp : PITCH, tt = TILED ? t : 0;
  // row t of the staged tile (the layout of update_row_chunk)
  const __half *prow = reinterpret_cast<const __half *>(stage) + tt * sp;
  const __half *srow = reinterpret_cast<const __half *>(stage + Lay::kSigOff) + (ODD ? tt + 1 : tt) * sp;
  const float *e0p = reinterpret_cast<const float *>(stage + Lay::kEpsOff) + (tt + 1) * sp;
  const float *ezm = reinterpret_cast<const float *>(stage + Lay::kEpsOff) + 3 * PITCH + tt * sp;
  const float *d0p = reinterpret_cast<const float *>(stage + Lay::kDepsOff) + (tt + 1) * sp;
  const float *dzm = reinterpret_cast<const float *>(stage + Lay::kDepsOff) + 3 * PITCH + tt * sp;
  const bool tv = L.has_deps != 0;
  const float rho0 = L.rho0f;
  const float inv_scale = L.inv_scale, scale = L.scale;
  __half *__restrict__ pop = static_cast<__half *>(L.pop);
  const long long plane = L.plane;
  const float omega = L.omegaf;
  const float om1 = 1.0f - omega;
  const float cf3 = L.cf3f, cf9 = L.cf9f;
  const unsigned qa = L.quad_axes;
  const bool vb = xa + 1 < nx;
  const int xb = vb ? xa + 1 : xa;
  const int xsa[3] = {xa == 0 ? nx - 1 : xa - 1, xa, xa == nx - 1 ? 0 : xa + 1};
  const int xsb[3] = {xb == 0 ? nx - 1 : xb - 1, xb, xb == nx - 1 ? 0 : xb + 1};
  const int cell = rc.base[1][1] + xa;

#define EPS_ROW(dy, dz) ((dz) == 0 ? e0p + (dy) * sp : ((dz) < 0 ? ezm : ezm + PITCH))
#define DEPS_ROW(dy, dz) ((dz) == 0 ? d0p + (dy) * sp : ((dz) < 0 ? dzm : dzm + PITCH))
#define SIG_ROW(dy, dz) (ODD ? srow + sig_block<LAT>(dz) * 3 * PITCH + (dy) * sp : srow)
  // a half row at the two cells' positions shifted by s in x (s = 0: the
  // cells themselves, one aligned load)
#define LD_H_SHIFT(row, s) ((s) == 0 ? ld_h2((row) + xa) : f2(ldh((row) + xsa[1 + (s)]), ldh((row) + xsb[1 + (s)])))
#define OWN_SRC(i) (!ODD || (i) == 0 || (WALLS && ((rc.solid >> ((1 - LAT::c((i), 2)) * 3 + (1 - LAT::c((i), 1)))) & 1u)))
#define OWN_DST(i) (!ODD || (i) == 0 || (WALLS && ((rc.solid >> ((1 + LAT::c((i), 2)) * 3 + (1 + LAT::c((i), 1)))) & 1u)))

  const float2 sig_own = ld_h2(SIG_ROW(0, 0) + xa);
  const float2 s_x = mul2(f2s(rho0), sig_own);
  const float2 ms_x = f2(-s_x.x, -s_x.y);
  const float2 rho2 = f2s(rho0), scale2 = f2s(scale);

  // 1. decode (update_row_chunk step 1, in storage units)
  float2 d[Q], delta[Q];
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    const __half *pr = prow + i * PITCH;
    if (OWN_SRC(i)) {
      delta[i] = f2s(0.f);
      d[i] = ld_h2(pr + xa);
    } else {
      const float2 q = LD_H_SHIFT(pr, -cx);
      const float2 sw = LD_H_SHIFT(SIG_ROW(-cy, -cz), -cx);
      delta[i] = fma2(rho2, sw, ms_x);
      d[i] = fma2(delta[i], scale2, q);
    }
  }

  // 2. moments
  float2 dM = f2s(0.f), j0 = f2s(0.f), j1 = f2s(0.f), j2 = f2s(0.f);
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float w = (float)LAT::w(i);
    dM = fma2(f2s(w), d[i], dM);
    if (LAT::c(i, 0) != 0) j0 = fma2(f2s(LAT::c(i, 0) > 0 ? w : -w), d[i], j0);
    if (LAT::c(i, 1) != 0) j1 = fma2(f2s(LAT::c(i, 1) > 0 ? w : -w), d[i], j1);
    if (D == 3 && LAT::c(i, 2) != 0) j2 = fma2(f2s(LAT::c(i, 2) > 0 ? w : -w), d[i], j2);
  }
  {
    const float2 is = f2s(inv_scale);
    dM = mul2(dM, is);
    j0 = mul2(j0, is);
    j1 = mul2(j1, is);
    j2 = mul2(j2, is);
  }
  const float2 M0 = add2(s_x, dM);

  // 3. phi at time n on the stencil (x - 1 of the second cell is the first
  //    cell; x + 1 of the first is the second, unless the first is the
  //    row's last cell)
  const float *e0r = EPS_ROW(0, 0);
  float2 e_c = ld_f2(e0r + xa);
  float2 e_xm = f2(e0r[xsa[0]], e_c.x), e_xp = f2(vb ? e_c.y : e0r[xsa[2]], e0r[xsb[2]]);
  float2 e_yp = ld_f2(EPS_ROW(1, 0) + xa), e_ym = ld_f2(EPS_ROW(-1, 0) + xa);
  float2 e_zp = e_c, e_zm = e_c;
  if (D == 3) {
    e_zp = ld_f2(EPS_ROW(0, 1) + xa);
    e_zm = ld_f2(EPS_ROW(0, -1) + xa);
  }
  if (tv) {
    const float2 dn2 = f2s(dn);
    const float *d0r = DEPS_ROW(0, 0);
    const float2 t_c = ld_f2(d0r + xa);
    e_c = fma2(dn2, t_c, e_c);
    e_xp = fma2(dn2, f2(vb ? t_c.y : d0r[xsa[2]], d0r[xsb[2]]), e_xp);
    e_xm = fma2(dn2, f2(d0r[xsa[0]], t_c.x), e_xm);
    e_yp = fma2(dn2, ld_f2(DEPS_ROW(1, 0) + xa), e_yp);
    e_ym = fma2(dn2, ld_f2(DEPS_ROW(-1, 0) + xa), e_ym);
    if (D == 3) {
      e_zp = fma2(dn2, ld_f2(DEPS_ROW(0, 1) + xa), e_zp);
      e_zm = fma2(dn2, ld_f2(DEPS_ROW(0, -1) + xa), e_zm);
    }
  }

  // 4.-6. quadrature, density, forces, velocity
  float2 nb = f2s(0.f);
  if (qa & 1u) nb = add2(nb, add2(e_xp, e_xm));
  if (qa & 2u) nb = add2(nb, add2(e_yp, e_ym));
  if (qa & 4u) nb = add2(nb, add2(e_zp, e_zm));
  const float2 I = fma2(f2s(L.qw0f), e_c, mul2(f2s(L.qw1f), nb));
  const float2 pc2 = mul2(f2(M0.x / I.x, M0.y / I.y), f2s(0.5f / 3.0f));
  float2 F0 = fma2(pc2, sub2(e_xp, e_xm), f2s(L.gf[0]));
  float2 F1 = fma2(pc2, sub2(e_yp, e_ym), f2s(L.gf[1]));
  float2 F2 = D == 3 ? fma2(pc2, sub2(e_zp, e_zm), f2s(L.gf[2])) : f2s(0.f);
  if (L.has_force) {
    const float *__restrict__ fo = static_cast<const float *>(L.force);
    const long long N = L.ncell;
    float2 a0 = ld_f2(fo + cell), a1 = ld_f2(fo + N + cell);
    float2 a2 = D == 3 ? ld_f2(fo + 2 * N + cell) : f2s(0.f);
    if (L.has_dforce) {
      const float *__restrict__ df = static_cast<const float *>(L.dforce);
      const float2 dnf = f2s(dn_force);
      a0 = fma2(dnf, ld_f2(df + cell), a0);
      a1 = fma2(dnf, ld_f2(df + N + cell), a1);
      if (D == 3) a2 = fma2(dnf, ld_f2(df + 2 * N + cell), a2);
    }
    F0 = add2(F0, a0);
    F1 = add2(F1, a1);
    F2 = add2(F2, a2);
  }
  const float2 invM = f2(1.0f / M0.x, 1.0f / M0.y);
  const float2 half2c = f2s(0.5f);
  const float2 u0 = mul2(fma2(half2c, F0, j0), invM);
  const float2 u1 = mul2(fma2(half2c, F1, j1), invM);
  const float2 u2 = D == 3 ? mul2(fma2(half2c, F2, j2), invM) : f2s(0.f);
  const float2 usq = fma2(u0, u0, fma2(u1, u1, mul2(u2, u2)));
  const float2 uF = fma2(u0, F0, fma2(u1, F1, mul2(u2, F2)));

  // 7.-8. collide and stream (update_row_chunk's FP16 branch)
  const float2 m15usq = mul2(f2s(-1.5f), usq);
  const float sc = scale;
  const float omega_s = omega * sc, cf3_s = cf3 * sc, cf9_s = cf9 * sc;
  const float2 m3uF_s = mul2(mul2(f2s(-cf3), uF), f2s(sc));
  SRng rng_a((unsigned)cell, n), rng_b((unsigned)(cell + 1), n);
  const bool sr = L.fp16_nearest == 0;
  const float2 om1_2 = f2s(om1), sc2 = f2s(sc), msc2 = f2s(-sc);
  __half *orow = OUTS ? reinterpret_cast<__half *>(ostage) + tt * sp : nullptr;

  // destination row of population i: the output stage's row i, or the
  // population plane (own slot: plane opp(i) of this row; else plane i of
  // row (y + c_iy, z + c_iz))
#define DST_ROW(i, own)                                                                              \
  ((OUTS) ? orow + (i) * PITCH                                                                       \
          : ((own) ? pop + opp_of(i) * plane + rc.base[1][1]                                         \
                   : pop + (i) * plane + rc.base[1 + LAT::c((i), 2)][1 + LAT::c((i), 1)]))

  {
    // rest population
    const float2 v = fma2(om1_2, d[0], fma2(f2s(omega_s), fma2(M0, m15usq, dM), m3uF_s));
    __half ha, hb;
    if (sr) {
      ha = half_sr(v.x, rng_a.next13());
      hb = half_sr(v.y, rng_b.next13());
    } else {
      ha = __float2half_rn(v.x);
      hb = __float2half_rn(v.y);
    }
    __half *row = DST_ROW(0, true);
    *reinterpret_cast<__half2 *>(row + xa) = __halves2half2(ha, hb);
  }
  const float2 oM03 = mul2(f2s(3.0f * omega_s), M0);
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    float2 cu = f2s(0.f), cF = f2s(0.f);
    if (cx == 1) { cu = add2(cu, u0); cF = add2(cF, F0); }
    if (cx == -1) { cu = sub2(cu, u0); cF = sub2(cF, F0); }
    if (cy == 1) { cu = add2(cu, u1); cF = add2(cF, F1); }
    if (cy == -1) { cu = sub2(cu, u1); cF = sub2(cF, F1); }
    if (cz == 1) { cu = add2(cu, u2); cF = add2(cF, F2); }
    if (cz == -1) { cu = sub2(cu, u2); cF = sub2(cF, F2); }
    const float2 t = fma2(M0, fma2(mul2(f2s(4.5f), cu), cu, m15usq), dM);
    const float2 A = fma2(f2s(omega_s), t, fma2(mul2(f2s(cf9_s), cu), cF, m3uF_s));
    const float2 B = fma2(oM03, cu, mul2(f2s(cf3_s), cF));
    float2 va = fma2(om1_2, d[i], add2(A, B));
    float2 vb2 = fma2(om1_2, d[i + 1], sub2(A, B));
    // encode against the shift of the storage cell (update_row_chunk's
    // ENCODE_POP without a pending shift change)
    const bool own_a = OWN_DST(i), own_b = OWN_DST(i + 1);
    if (!own_a) {
      if (!OWN_SRC(i + 1))
        va = fma2(delta[i + 1], msc2, va);
      else
        va = fma2(fma2(f2s(-rho0), LD_H_SHIFT(SIG_ROW(cy, cz), cx), s_x), sc2, va);
    }
    if (!own_b) {
      if (!OWN_SRC(i))
        vb2 = fma2(delta[i], msc2, vb2);
      else
        vb2 = fma2(fma2(f2s(-rho0), LD_H_SHIFT(SIG_ROW(-cy, -cz), -cx), s_x), sc2, vb2);
    }
    unsigned ha, hb;  // (population i, population i + 1) of each cell
    if (sr) {
      ha = half2_sr(va.x, vb2.x, rng_a.next32());
      hb = half2_sr(va.y, vb2.y, rng_b.next32());
    } else {
      ha = (unsigned)__half_as_ushort(__float2half_rn(va.x)) | ((unsigned)__half_as_ushort(__float2half_rn(vb2.x)) << 16);
      hb = (unsigned)__half_as_ushort(__float2half_rn(va.y)) | ((unsigned)__half_as_ushort(__float2half_rn(vb2.y)) << 16);
    }
    // population i goes to x + c_ix unless it stays; i + 1 to x - c_ix
    st_h2(DST_ROW(i, own_a), ha, hb, false, own_a || cx == 0, xa, own_a ? xa : xsa[1 + cx],
          own_a ? xb : xsb[1 + cx], vb);
    st_h2(DST_ROW(i + 1, own_b), ha, hb, true, own_b || cx == 0, xa, own_b ? xa : xsa[1 - cx],
          own_b ? xb : xsb[1 - cx], vb);
  }
#undef DST_ROW
#undef EPS_ROW
#undef DEPS_ROW
#undef SIG_ROW
#undef LD_H_SHIFT
#undef OWN_SRC
#undef OWN_DST
}

}  // namespace lbm
