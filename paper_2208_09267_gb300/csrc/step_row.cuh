// step_row.cuh -- persistent row kernel: the fused step of step_fast.cuh with
// its inputs staged in shared memory by TMA bulk copies.
//
// Work item: a tile of R consecutive fluid x-rows (y0 .. y0 + R - 1) of one
// z-plane, all nx cells of each, R = min(8, PITCH / nxp) (1 for rows of more
// than half the pitch).  A block keeps NSTAGE tiles in flight: while the
// threads update tile j, the bulk copies of tile j + NSTAGE - 1 are landing.
// Per tile and step the block stages, rows stored at their pitch nxp:
//   - the Q population blocks it reads (R rows each): at even n plane i of
//     its own rows; at odd n plane opp(i) of rows (y - c_iy, z - c_iz) (the x
//     shift of -c_ix is a modular index into the staged row), or plane i of
//     the own row where that neighbour row is a wall layer (halfway
//     bounce-back);
//   - the shift sigma (phi_ref rounded to half) of the rows y0 - 1 .. y0 + R
//     of the planes z - 1, z, z + 1 (odd steps: every neighbour's shift) or
//     of the own rows (even steps);
//   - phi_ref on the rows y0 - 1 .. y0 + R of plane z and on the tile's rows
//     of the planes z - 1 and z + 1 (the 5-point cross of every cell), and
//     d_t phi on the same rows when phi varies;
// each block as one cp.async.bulk of consecutive stored rows (more where the
// rows wrap around periodically or a wall layer substitutes the own row),
// completing on one mbarrier per stage.  Tiles of several short rows cut
// the number of copies per cell: the producer warp's copy issue, not DRAM,
// bounds rows of a few dozen cells staged one by one.
//
// Requirements (checked by the host before choosing this kernel): rows
// stored at a pitch nxp that is a multiple of 8 elements (so every copy
// starts and ends on a 16-byte boundary), nxp <= PITCH <= 512, fewer than
// 2^31 stored cells, walls only on y and/or z.  Every wait is bounded: a
// block that waits too long records the failure in L.status, drains its
// copies (again bounded) and leaves; the host reports LBM_ETIMEOUT.
#pragma once

#include <cuda_fp16.h>

#include "internal.h"
#include "lattice.cuh"
#include "step_fast.cuh"

namespace lbm {

#ifndef LBM_ROW_CONSUMERS
#define LBM_ROW_CONSUMERS 7
#endif
#ifndef LBM_ROW_CONSUMERS_F16
#define LBM_ROW_CONSUMERS_F16 6
#endif
#ifndef LBM_ROW_PRODUCERS
#define LBM_ROW_PRODUCERS 1  // producer warps per block of the single-lattice row kernel (1 or 2)
#endif
#ifndef LBM_ROW_OUTS_F16
#define LBM_ROW_OUTS_F16 1  // FP16 rows written back through output stages (0: direct stores)
#endif
// Consumer warps per block (+ one producer warp).  Two blocks per SM (MINB
// 2) take 7: every SM sub-partition then holds four warps of up to 128
// registers.  Where a stage is too large for two blocks per SM (MINB 1: rows
// of 512 cells, D3Q27) one block takes 15, so the SM keeps 16 warps.  FP16
// D2Q9/D3Q19 blocks also have a storer warp and update two cells per lane
// (more live registers): 6 consumers (14 with MINB 1) keep them at 16 warps
// per SM, 128 registers each.
template <int MINB, bool PAIR = false>
constexpr int row_consumers() {
  return PAIR ? (MINB == 1 ? 14 : LBM_ROW_CONSUMERS_F16) : (MINB == 1 ? 15 : LBM_ROW_CONSUMERS);
}
template <int MINB>
constexpr int row_threads() { return (row_consumers<MINB>() + 1) * 32; }
// the single-lattice kernel: producer warps per block, and consumers (one
// fewer per extra producer, so that the block keeps its warp count)
constexpr int kRowProducers = LBM_ROW_PRODUCERS;
template <int MINB, bool PAIR>
constexpr int row_consumers_single() { return row_consumers<MINB, PAIR>() - (kRowProducers - 1); }
// FP16 plain steps of D2Q9/D3Q19 update two adjacent cells per lane
// (update_row_pair); D3Q27's larger state would spill
template <class LAT, class ST>
constexpr bool row_pair_lattice() { return sizeof(ST) == 2 && LAT::Q <= 19; }
constexpr unsigned kWaitSpins = 1u << 22;  // bounded mbarrier wait
constexpr int kMaxTileRows = 8;

// rows per tile of a lattice with row pitch nxp in a kernel of stage pitch PITCH
__host__ __device__ constexpr int tile_rows(int pitch, int nxp) {
  return pitch / nxp < 1 ? 1 : (pitch / nxp > kMaxTileRows ? kMaxTileRows : pitch / nxp);
}

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

// Shared-memory layout of one stage, in slots of PITCH elements (a block of
// rows at pitch nxp fills at most its slots).  Order: the Q population
// blocks (R rows each); the shift blocks (half; odd steps: three slots per
// plane z + dz, dz = -1, 0, 1 (2D: plane z only), holding rows y0 - 1 ..
// y0 + R; even steps: one slot with the tile's own rows); phi_ref (plane z:
// three slots, rows y0 - 1 .. y0 + R; 3D: then one slot each for planes z - 1
// and z + 1, the tile's rows); d_t phi in the same layout.
template <class LAT, class ST, bool ODD, int PITCH>
struct RowLayout {
  static constexpr int kSigSlots = ODD ? (LAT::D == 2 ? 3 : 9) : 1;
  static constexpr int kEpsSlots = LAT::D == 2 ? 3 : 5;
  static constexpr int kPopBytes = PITCH * (int)sizeof(ST);
  static constexpr int kSigBytes = PITCH * 2;
  static constexpr int kRowBytes = PITCH * 4;
  static constexpr int kSigOff = LAT::Q * kPopBytes;
  static constexpr int kEpsOff = kSigOff + kSigSlots * kSigBytes;
  static constexpr int kDepsOff = kEpsOff + kEpsSlots * kRowBytes;
  static constexpr int kStageBytes = kDepsOff + kEpsSlots * kRowBytes;
};

// shift block of plane z + dz at odd steps
template <class LAT>
__host__ __device__ constexpr int sig_block(int dz) {
  return LAT::D == 2 ? 0 : dz + 1;
}

__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Per-row quantities (computed by the producer, once per row of a tile).
struct RowCtx {
  int base[3][3];   // cell index of x = 0 on row (y+dy, z+dz), [dz+1][dy+1]
  unsigned solid;   // bit (dz+1)*3+(dy+1): that neighbour row is a wall layer
};

// A staged tile: first row, plane, rows.
struct TileCtx {
  int y0, z, nr;
};

// Is row (y, z) a wall layer?
__device__ __forceinline__ bool wall_row(unsigned walls, int y, int z, int ny, int nz) {
  return ((walls & 2u) && (y <= 0 || y >= ny - 1)) || ((walls & 4u) && (z <= 0 || z >= nz - 1));
}

// (c_iy, c_iz) of direction i (runtime i), by unrolled selects: no table in
// local memory.
template <class LAT>
__device__ __forceinline__ void dir_yz(int i, int &cy, int &cz) {
  cy = 0;
  cz = 0;
#pragma unroll
  for (int k = 1; k < LAT::Q; ++k) {
    const bool hit = k == i;
    cy = hit ? LAT::c(k, 1) : cy;
    cz = hit ? LAT::c(k, 2) : cz;
  }
}

// One block of a tile's bulk copies, owned by one producer lane and set up
// once per launch (or per batch member): block row k (0 <= k < nr + extra)
// is source row (y0 + k + dy0, z + dz), wrapped periodically; a population
// block read from a neighbour row takes the own row (y0 + k, z) of plane
// src_own where that neighbour row is a wall layer.
struct TileCopy {
  const char *src;      // field (population plane included) at row base 0
  const char *src_own;  // population blocks: the own-row plane (bounce-back)
  unsigned dst;         // byte offset of the block in the stage
  int esize;            // bytes per element; 0: this lane has no such block
  int dy0, dz;          // source row offset of block row 0
  int extra;            // rows beyond the tile's (halo blocks: 2)
  int nb_pop;           // population block read from neighbour rows
};

template <class LAT, class ST, bool ODD, int PITCH>
__device__ __forceinline__ TileCopy make_tile_copy(const LatticeDev &L, int j) {
  using Lay = RowLayout<LAT, ST, ODD, PITCH>;
  constexpr int nsig = ODD ? (LAT::D == 2 ? 1 : 3) : 1;
  constexpr int nfb = LAT::D == 2 ? 1 : 3;  // field blocks: plane z (with halo rows), z - 1, z + 1
  TileCopy c;
  const bool tv = L.has_deps != 0;
  const int ncopies = LAT::Q + nsig + nfb * (tv ? 2 : 1);
  c.esize = 0;
  c.dy0 = c.dz = c.extra = c.nb_pop = 0;
  c.src = c.src_own = nullptr;
  c.dst = 0;
  if (j >= ncopies) return c;
  if (j < LAT::Q) {
    int cy, cz;
    dir_yz<LAT>(j, cy, cz);
    const char *pop = static_cast<const char *>(L.pop);
    const long long plane_bytes = L.plane * (long long)sizeof(ST);
    c.src_own = pop + j * plane_bytes;
    if (ODD && j != 0) {
      c.src = pop + opp_of(j) * plane_bytes;
      c.dy0 = -cy;
      c.dz = -cz;
      c.nb_pop = 1;
    } else {
      c.src = c.src_own;
    }
    c.dst = (unsigned)(j * Lay::kPopBytes);
    c.esize = (int)sizeof(ST);
  } else if (j < LAT::Q + nsig) {
    const int e = j - LAT::Q;
    c.src = reinterpret_cast<const char *>(L.sig_wr);
    c.esize = 2;
    if (ODD) {
      c.dz = LAT::D == 2 ? 0 : e - 1;
      c.dy0 = -1;
      c.extra = 2;
      c.dst = (unsigned)(Lay::kSigOff + e * 3 * Lay::kSigBytes);
    } else {
      c.dst = (unsigned)Lay::kSigOff;
    }
  } else {
    const int f = j - LAT::Q - nsig;
    const bool is_deps = f >= nfb;
    const int e = is_deps ? f - nfb : f;
    c.src = static_cast<const char *>(is_deps ? L.deps : L.eps);
    c.esize = 4;
    const unsigned off = (unsigned)(is_deps ? Lay::kDepsOff : Lay::kEpsOff);
    if (e == 0) {
      c.dy0 = -1;
      c.extra = 2;
      c.dst = off;
    } else {
      c.dz = e == 1 ? -1 : 1;
      c.dst = off + (unsigned)((e + 2) * Lay::kRowBytes);
    }
  }
  return c;
}

// Bytes one lane's block of a tile of nr rows copies.
__device__ __forceinline__ unsigned tile_copy_bytes(const TileCopy &c, int nr, int nxp) {
  return c.esize ? (unsigned)((nr + c.extra) * nxp * c.esize) : 0u;
}

// Issue the copies of block c for the tile (y0, z, nr) into `stage`,
// completing on `bar`: block row k lands at k * dst_row_bytes (the stored
// row size nxp * esize, or the slot size PITCH * esize of one-row tiles).
// Source rows inside the lattice, in one plane, with no wall substitution
// (every block but those at a periodic edge or next to a wall) go as one
// copy (or one per row when the two row sizes differ); the others are
// split into runs of rows consecutive in both places.
__device__ __forceinline__ void issue_tile_copy(const TileCopy &c, unsigned char *stage, unsigned long long *bar,
                                                int y0, int z, int nr, int ny, int nz, int nxp, unsigned walls,
                                                int dst_pitch) {
  if (!c.esize) return;
  const int n = nr + c.extra;
  const unsigned row_bytes = (unsigned)(nxp * c.esize);
  const unsigned dst_row_bytes = (unsigned)(dst_pitch * c.esize);
  const bool merge = dst_row_bytes == row_bytes;
  const int ys = y0 + c.dy0, zs = z + c.dz;
  const bool inside = ys >= 0 && ys + n <= ny && zs >= 0 && zs < nz;
  const bool sub = c.nb_pop && (((walls & 2u) && (ys <= 0 || ys + n - 1 >= ny - 1)) ||
                                ((walls & 4u) && (zs <= 0 || zs >= nz - 1)));
  if (inside && !sub) {
    const char *src = c.src + ((long long)zs * ny + ys) * row_bytes;
    unsigned char *dst = stage + c.dst;
    if (merge) {
      bulk_g2s(dst, src, (unsigned)n * row_bytes, bar);
    } else {
      for (int k = 0; k < n; ++k) bulk_g2s(dst + k * dst_row_bytes, src + k * row_bytes, row_bytes, bar);
    }
    return;
  }
  const char *run_src = nullptr;
  long long run_row = 0;
  int run_k = 0, run_len = 0;
  for (int k = 0; k < n; ++k) {
    int yy = ys + k, zz = zs;
    const char *src = c.src;
    if (c.nb_pop && walls && wall_row(walls, yy, zz, ny, nz)) {
      // halfway bounce-back: the population comes from the own row
      yy = y0 + k;
      zz = z;
      src = c.src_own;
    }
    const long long row = (long long)wrapi(zz, nz) * ny + wrapi(yy, ny);
    if (run_len && merge && src == run_src && row == run_row + run_len) {
      ++run_len;
      continue;
    }
    if (run_len)
      bulk_g2s(stage + c.dst + run_k * dst_row_bytes, run_src + run_row * row_bytes, run_len * row_bytes, bar);
    run_src = src;
    run_row = row;
    run_k = k;
    run_len = 1;
  }
  if (run_len)
    bulk_g2s(stage + c.dst + run_k * dst_row_bytes, run_src + run_row * row_bytes, run_len * row_bytes, bar);
}

// The row contexts of the tile (y0, z, nr), written by the producer warp
// (lanes in parallel) into rc[0 .. nr).
__device__ __forceinline__ void fill_row_ctx(RowCtx *rc, int y0, int z, int nr, int ny, int nz, int nxp,
                                             unsigned walls, int lane) {
  for (int idx = lane; idx < nr * 9; idx += 32) {
    const int t = idx / 9, e = idx - t * 9;
    const int dy = e % 3 - 1, dz = e / 3 - 1;
    rc[t].base[dz + 1][dy + 1] = (wrapi(z + dz, nz) * ny + wrapi(y0 + t + dy, ny)) * nxp;
  }
  if (lane < nr) {
    unsigned solid = 0;
    if (walls) {
#pragma unroll
      for (int e = 0; e < 9; ++e)
        if (wall_row(walls, y0 + lane + e % 3 - 1, z + e / 3 - 1, ny, nz)) solid |= 1u << e;
    }
    rc[lane].solid = solid;
  }
}

// Update the 32-cell chunk [x0, x0 + 32) of row t of a staged tile (one
// cell per lane).
// RS: the step after a phi refresh decodes with the old shift and encodes
// with the new one ("reshift").  0: no refresh pending, 1: pending (both
// known at launch), 2: read it from the descriptor.
// OUTS: the updated populations go to the output stage `ostage` in shared
// memory (row i holds f*_i at the position of its storage cell in the
// destination row) instead of straight to global memory; a storer warp
// writes the rows back with bulk copies.
template <class LAT, class ST, bool ODD, bool RED, bool WALLS, int PITCH, int RS = 2, bool OUTS = false,
          bool TILED = true>
__device__ __forceinline__ void update_row_chunk(const LatticeDev &L, const unsigned char *stage, int t,
                                                 const RowCtx &rc, long long n, float dn, float dn_force,
                                                 int x, RedAcc &acc, unsigned char *ostage = nullptr) {
  using Lay = RowLayout<LAT, ST, ODD, PITCH>;
  constexpr int Q = LAT::Q, D = LAT::D;
  // FP16 stores deviations times 2^k.  The update below runs in those
  // storage units (d, the sums and the collision output all times 2^k): a
  // power of two scales every rounding exactly, so the stored results are
  // those of the unscaled arithmetic, without a multiply per population on
  // load and store.
  constexpr bool kScaled = sizeof(ST) < 4;
  // FP32: per-population collision in the change form and a local mass
  // balance through the rest population (step 8 below)
  constexpr bool kMassFix = sizeof(ST) == 4;
  const int nx = L.nx;
  // smem row pitch and row of the tile: TILED, nxp and t (rows of the tile
  // copied together land at their stored pitch); else one row per stage at
  // the compile-time pitch PITCH (every offset below an immediate)
  const int sp = TILED ? L.nxp : PITCH, tt = TILED ? t : 0;
  // row t of the staged tile: population block i at prow + i PITCH; the
  // shift of row (y + dy, z + dz) at srow[sig_block(dz) 3 PITCH + dy sp]
  // (odd steps) or srow (even steps); phi_ref of row (y + dy, z) at
  // e0[dy sp], of rows (y, z -+ 1) at ezm, ezp (d_t phi likewise)
  const ST *prow = reinterpret_cast<const ST *>(stage) + tt * sp;
  const __half *srow = reinterpret_cast<const __half *>(stage + Lay::kSigOff) + (ODD ? tt + 1 : tt) * sp;
  const float *e0 = reinterpret_cast<const float *>(stage + Lay::kEpsOff) + (tt + 1) * sp;
  const float *ezm = reinterpret_cast<const float *>(stage + Lay::kEpsOff) + 3 * PITCH + tt * sp;
  const float *ezp = ezm + PITCH;
  const float *d0 = reinterpret_cast<const float *>(stage + Lay::kDepsOff) + (tt + 1) * sp;
  const float *dzm = reinterpret_cast<const float *>(stage + Lay::kDepsOff) + 3 * PITCH + tt * sp;
  const float *dzp = dzm + PITCH;
  const bool tv = L.has_deps != 0;
  const float rho0 = L.rho0f;
  const float inv_scale = L.inv_scale, scale = L.scale;
  const __half *__restrict__ srd = L.sig_rd;
  // shift changed by the last set_epsilon
  const bool reshift = RS == 2 ? srd != L.sig_wr : RS == 1;
  ST *__restrict__ pop = static_cast<ST *>(L.pop);
  // plane i starts i * plane elements into pop: a 64-bit offset (Q planes of
  // up to 2^31 stored cells pass the int range); offsets within a plane are
  // ints (fewer than 2^31 stored cells)
  const long long plane = L.plane;
  const float omega = L.omegaf;
  const float om1 = 1.0f - omega;
  const float cf3 = L.cf3f, cf9 = L.cf9f;
  const unsigned qa = L.quad_axes;

#define EPS_AT(dy, dz, xx) ((dz) == 0 ? e0[(dy) * sp + (xx)] : ((dz) < 0 ? ezm[xx] : ezp[xx]))
#define DEPS_AT(dy, dz, xx) ((dz) == 0 ? d0[(dy) * sp + (xx)] : ((dz) < 0 ? dzm[xx] : dzp[xx]))
#define SIG_AT(dy, dz, xx) \
  __half2float(ODD ? srow[sig_block<LAT>(dz) * 3 * PITCH + (dy) * sp + (xx)] : srow[xx])
  // slot of population i read from / written to this cell's own memory?
#define OWN_SRC(i) (!ODD || (i) == 0 || (WALLS && ((rc.solid >> ((1 - LAT::c((i), 2)) * 3 + (1 - LAT::c((i), 1)))) & 1u)))
#define OWN_DST(i) (!ODD || (i) == 0 || (WALLS && ((rc.solid >> ((1 + LAT::c((i), 2)) * 3 + (1 + LAT::c((i), 1)))) & 1u)))

  if (x >= nx) return;  // lane past the end of a row that is not a multiple of 32
  const int xs[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
  const int cell = rc.base[1][1] + x;
  const float e_own = EPS_AT(0, 0, x);
  const float sig_own = SIG_AT(0, 0, x);  // sigma_wr of this cell
  // the cell's frame: its own shift as stored (sigma_rd)
  const float s_x = rho0 * (reshift ? __half2float(srd[cell]) : sig_own);

  // 1. decode: d_i = f_i/w_i - s_x (in storage units).  A value stored in
  //    another cell m carries that cell's shift: add delta_i = rho0 sigma(m)
  //    - s_x (exact product in the FMA; the encode below uses the same form,
  //    so the round trip is exact up to the final rounding).  Own-cell values
  //    need no shift.
  //    FP32 also keeps the stored values q_i as read (the mass balance of
  //    step 8 is taken on them) and, after a phi refresh, the difference
  //    between the read and write shifts of the slots it reads.
  float d[Q], delta[Q], qraw[Q];
  float frame = 0.f;  // sum_i w_i rho0 (sigma_rd - sigma_wr) of the slots read (FP32, refresh steps)
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    const bool own = OWN_SRC(i);
    const float q = PopIO<ST>::ld(prow + i * PITCH + (own ? x : xs[1 - cx]));
    qraw[i] = q;
    if (own) {
      delta[i] = 0.f;
      d[i] = q;
      if (kMassFix && reshift) frame = fmaf((float)LAT::w(i), fmaf(-rho0, sig_own, s_x), frame);
    } else {
      const float sw = SIG_AT(-cy, -cz, xs[1 - cx]);
      const float sm = reshift ? __half2float(srd[rc.base[1 - cz][1 - cy] + xs[1 - cx]]) : sw;
      delta[i] = fmaf(rho0, sm, -s_x);
      // delta 2^k is exact, so the FMA rounds once, as q + delta 2^k does
      d[i] = kScaled ? fmaf(delta[i], scale, q) : q + delta[i];
      if (kMassFix && reshift) frame = fmaf((float)LAT::w(i), rho0 * (sm - sw), frame);
    }
  }

  // 2. moments: dM = sum w d, J = sum w xi d
  float dM = 0.f, j0 = 0.f, j1 = 0.f, j2 = 0.f;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    const float w = (float)LAT::w(i);
    dM = fmaf(w, d[i], dM);
    if (LAT::c(i, 0) != 0) j0 = fmaf(LAT::c(i, 0) > 0 ? w : -w, d[i], j0);
    if (LAT::c(i, 1) != 0) j1 = fmaf(LAT::c(i, 1) > 0 ? w : -w, d[i], j1);
    if (D == 3 && LAT::c(i, 2) != 0) j2 = fmaf(LAT::c(i, 2) > 0 ? w : -w, d[i], j2);
  }
  if (kScaled) {
    dM *= inv_scale;
    j0 *= inv_scale;
    j1 *= inv_scale;
    j2 *= inv_scale;
  }
  const float M0 = s_x + dM;

  // 3. phi at time n on the stencil
  float e_c = e_own, e_xp = EPS_AT(0, 0, xs[2]), e_xm = EPS_AT(0, 0, xs[0]);
  float e_yp = EPS_AT(1, 0, x), e_ym = EPS_AT(-1, 0, x);
  float e_zp = e_c, e_zm = e_c;
  if (D == 3) {
    e_zp = EPS_AT(0, 1, x);
    e_zm = EPS_AT(0, -1, x);
  }
  if (tv) {
    e_c = fmaf(dn, DEPS_AT(0, 0, x), e_c);
    e_xp = fmaf(dn, DEPS_AT(0, 0, xs[2]), e_xp);
    e_xm = fmaf(dn, DEPS_AT(0, 0, xs[0]), e_xm);
    e_yp = fmaf(dn, DEPS_AT(1, 0, x), e_yp);
    e_ym = fmaf(dn, DEPS_AT(-1, 0, x), e_ym);
    if (D == 3) {
      e_zp = fmaf(dn, DEPS_AT(0, 1, x), e_zp);
      e_zm = fmaf(dn, DEPS_AT(0, -1, x), e_zm);
    }
  }

  // 4.-6. quadrature, density, forces, velocity
  float nb = 0.f;
  if (qa & 1u) nb += e_xp + e_xm;
  if (qa & 2u) nb += e_yp + e_ym;
  if (qa & 4u) nb += e_zp + e_zm;
  const float I = fmaf(L.qw0f, e_c, L.qw1f * nb);
  const float pc2 = M0 / I * (0.5f / 3.0f);  // c_s^2 rho~ / 2
  float F0 = fmaf(pc2, e_xp - e_xm, L.gf[0]);
  float F1 = fmaf(pc2, e_yp - e_ym, L.gf[1]);
  float F2 = D == 3 ? fmaf(pc2, e_zp - e_zm, L.gf[2]) : 0.f;
  if (L.has_force) {
    const float *__restrict__ fo = static_cast<const float *>(L.force);
    const long long N = L.ncell;
    float a0 = __ldg(fo + cell), a1 = __ldg(fo + N + cell), a2 = D == 3 ? __ldg(fo + 2 * N + cell) : 0.f;
    if (L.has_dforce) {
      const float *__restrict__ df = static_cast<const float *>(L.dforce);
      const float dnf = dn_force;
      a0 = fmaf(dnf, __ldg(df + cell), a0);
      a1 = fmaf(dnf, __ldg(df + N + cell), a1);
      if (D == 3) a2 = fmaf(dnf, __ldg(df + 2 * N + cell), a2);
    }
    F0 += a0;
    F1 += a1;
    F2 += a2;
  }
  const float invM = 1.0f / M0;
  const float u0 = fmaf(0.5f, F0, j0) * invM;
  const float u1 = fmaf(0.5f, F1, j1) * invM;
  const float u2 = D == 3 ? fmaf(0.5f, F2, j2) * invM : 0.f;
  const float usq = fmaf(u0, u0, fmaf(u1, u1, u2 * u2));
  const float uF = fmaf(u0, F0, fmaf(u1, F1, u2 * F2));

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

  // 7.-8. collide and stream:
  //   d*_i = (1 - omega) d_i + omega (dM + M0 (3 cu + 4.5 cu^2 - 1.5 u.u))
  //          + (1 - 1/(2 tau)) (3 (cF - u.F) + 9 cu cF)
  //   stored: d*_i + s_x - rho0 sigma_wr(storage cell).  sigma_wr is the new
  //   phi_ref; without a pending shift change it equals sigma_rd, and the
  //   shift difference of the neighbour x + xi_i is -delta of the opposite
  //   direction.
  const float m15usq = -1.5f * usq;
  // coefficients of the collision output, in storage units
  const float sc = kScaled ? scale : 1.0f;
  const float omega_s = omega * sc, cf3_s = cf3 * sc, cf9_s = cf9 * sc;
  const float m3uF_s = (-cf3 * uF) * sc;
  const float enc_own = reshift ? fmaf(-rho0, sig_own, s_x) : 0.f;
  SRng rng((unsigned)cell, n);
  const bool sr = L.fp16_nearest == 0;
  ST *orow = OUTS ? reinterpret_cast<ST *>(ostage) + tt * sp : nullptr;
  // encode population i (compile-time index) with post-collision deviation
  // DSTAR (storage units): P_ = its slot, V_ = the value to store against
  // the shift of the cell whose memory holds it
#define ENCODE_POP(i, DSTAR, P_, V_)                                                               \
  ST *P_;                                                                                          \
  float V_;                                                                                        \
  {                                                                                                \
    const int cx_ = LAT::c((i), 0), cy_ = LAT::c((i), 1), cz_ = LAT::c((i), 2);                    \
    const float ds_ = (DSTAR);                                                                     \
    if (OWN_DST(i)) {                                                                              \
      V_ = reshift ? fmaf(enc_own, sc, ds_) : ds_;                                                 \
      P_ = OUTS ? orow + (i) * PITCH + x : (pop + opp_of(i) * plane) + cell;                   \
    } else {                                                                                       \
      const int xm_ = xs[1 + cx_];                                                                 \
      float enc_;                                                                                  \
      if (!reshift && !OWN_SRC(opp_of(i)))                                                         \
        enc_ = -delta[opp_of(i)];                                                                  \
      else                                                                                         \
        enc_ = fmaf(-rho0, SIG_AT(cy_, cz_, xm_), s_x);                                            \
      V_ = fmaf(enc_, sc, ds_);                                                                    \
      P_ = OUTS ? orow + (i) * PITCH + xm_                                                        \
                : (pop + (i) * plane) + (rc.base[1 + cz_][1 + cy_] + xm_);                         \
    }                                                                                              \
  }
  if (kMassFix) {
    // FP32.  d*_i = d_i + (omega (d^eq_i - d_i) + Omega_i/w_i): the final sum
    // is the only rounding at the size of d_i (the bracket is the small
    // non-equilibrium change).  Then the mass the stored values carry is
    // balanced exactly: every slot the cell reads is a slot it writes (AA
    // pattern; the same set of storage cells, so the shift terms cancel
    // except after a refresh), hence
    //   w_0 V_0 = w_0 q_0 + sum_{i>0} w_i (q_i - V_i) + frame
    // with the stored values V_i as rounded.  The rest population absorbs
    // the rounding of the others: the zeroth moment of the stored state is
    // conserved cell by cell up to one rounding, instead of drifting with
    // the rounding of every population.
    float R = frame;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
      const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
      float cu = 0.f, cF = 0.f;
      if (cx == 1) { cu += u0; cF += F0; }
      if (cx == -1) { cu -= u0; cF -= F0; }
      if (cy == 1) { cu += u1; cF += F1; }
      if (cy == -1) { cu -= u1; cF -= F1; }
      if (cz == 1) { cu += u2; cF += F2; }
      if (cz == -1) { cu -= u2; cF -= F2; }
      // d^eq of the pair: dM + M0 (+-3 cu + 4.5 cu^2 - 1.5 u.u)
      const float deqa = fmaf(M0, fmaf(cu, fmaf(4.5f, cu, 3.0f), m15usq), dM);
      const float deqb = fmaf(M0, fmaf(cu, fmaf(4.5f, cu, -3.0f), m15usq), dM);
      // Guo term / w of the pair: cf (9 cu cF - 3 u.F) +- 3 cf cF
      // (every sum written as an explicit FMA: the rounding is then the same
      // in every instantiation of this code, single-lattice and batched)
      const float sA = fmaf(cf9 * cu, cF, m3uF_s);
      const float sa = fmaf(cf3, cF, sA), sb = fmaf(-cf3, cF, sA);
      ENCODE_POP(i, d[i] + fmaf(omega, deqa - d[i], sa), pa_, va_);
      ENCODE_POP(i + 1, d[i + 1] + fmaf(omega, deqb - d[i + 1], sb), pb_, vb_);
      PopIO<ST>::st(pa_, va_);
      PopIO<ST>::st(pb_, vb_);
      const float w = (float)LAT::w(i);
      R = fmaf(w, qraw[i] - va_, R);
      R = fmaf(w, qraw[i + 1] - vb_, R);
    }
    ENCODE_POP(0, d[0], p0_, v0_);
    (void)v0_;
    PopIO<ST>::st(p0_, fmaf(R, (float)(1.0 / LAT::w(0)), qraw[0]));
  } else {
  // rest population: cu = cF = 0
  {
    ENCODE_POP(0, fmaf(om1, d[0], fmaf(omega_s, fmaf(M0, m15usq, dM), m3uF_s)), p0_, v0_);
    store_pop<ST>(p0_, v0_, rng, sr);
  }
  // opposite pairs (i, i+1): cu and cF change sign, so
  //   omega d^eq + Omega = A +- B,  A = omega (dM + M0 (4.5 cu^2 - 1.5 u.u)) + cf (9 cu cF - 3 u.F),
  //                                 B = 3 omega M0 cu + 3 cf cF
  const float oM03 = 3.0f * omega_s * M0;
#pragma unroll
  for (int i = 1; i < Q; i += 2) {
    const int cx = LAT::c(i, 0), cy = LAT::c(i, 1), cz = LAT::c(i, 2);
    float cu = 0.f, cF = 0.f;
    if (cx == 1) { cu += u0; cF += F0; }
    if (cx == -1) { cu -= u0; cF -= F0; }
    if (cy == 1) { cu += u1; cF += F1; }
    if (cy == -1) { cu -= u1; cF -= F1; }
    if (cz == 1) { cu += u2; cF += F2; }
    if (cz == -1) { cu -= u2; cF -= F2; }
    const float t = fmaf(M0, fmaf(4.5f * cu, cu, m15usq), dM);
    const float A = fmaf(omega_s, t, fmaf(cf9_s * cu, cF, m3uF_s));
    const float B = fmaf(oM03, cu, cf3_s * cF);
    ENCODE_POP(i, fmaf(om1, d[i], A + B), pa_, va_);
    ENCODE_POP(i + 1, fmaf(om1, d[i + 1], A - B), pb_, vb_);
    store_pop_pair<ST>(pa_, va_, pb_, vb_, rng, sr);
  }
  }
#undef ENCODE_POP
#undef EPS_AT
#undef DEPS_AT
#undef SIG_AT
#undef OWN_SRC
#undef OWN_DST
}

}  // namespace lbm

#include "step_row_pair.cuh"

namespace lbm {

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up when another warp has raised `abort`.
__device__ __forceinline__ bool mbar_wait_or_abort(unsigned long long *bar, unsigned parity, unsigned limit,
                                                   volatile int *abort) {
  for (unsigned i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort) return false;
  }
  return false;
}

// Bulk copy of `bytes` from shared to global memory (both 16-byte aligned, a
// multiple of 16 bytes), tracked in this thread's bulk async-group.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until this thread's bulk stores have read their shared-memory source
__device__ __forceinline__ void bulk_wait_read_all() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// wait until this thread's bulk stores have completed
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// make this thread's shared-memory writes visible to the bulk-copy engine
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Write population i's output block of the tile (y0, z, nr) back (storer
// lane i; block row t at t * src_pitch elements): row t goes to row (y0 + t
// + c_iy, z + c_iz) of plane i at odd steps (i > 0) unless that row is a
// wall layer, else to the own row of plane opp(i); one bulk store per run of
// rows consecutive in both places.
template <class LAT, class ST, bool ODD>
__device__ __forceinline__ void store_tile_block(const LatticeDev &L, const unsigned char *oblock, int i, int cy,
                                                 int cz, int y0, int z, int nr, int src_pitch) {
  const int ny = L.ny, nz = L.nz, nxp = L.nxp;
  const unsigned walls = L.walls;
  const long long plane_bytes = L.plane * (long long)sizeof(ST);
  char *pop = static_cast<char *>(L.pop);
  const unsigned row_bytes = (unsigned)nxp * (unsigned)sizeof(ST);
  const unsigned src_row_bytes = (unsigned)src_pitch * (unsigned)sizeof(ST);
  const bool merge = src_row_bytes == row_bytes;
  const bool moves = ODD && i != 0;
  char *run_dst = nullptr;
  int run_t = 0, run_len = 0;
  long long run_row = 0;
  for (int t = 0; t < nr; ++t) {
    const int y = y0 + t;
    const bool to_nb = moves && !(walls && wall_row(walls, y + cy, z + cz, ny, nz));
    const int yy = to_nb ? wrapi(y + cy, ny) : y, zz = to_nb ? wrapi(z + cz, nz) : z;
    char *dst = pop + (to_nb ? i : opp_of(i)) * plane_bytes;
    const long long row = (long long)zz * ny + yy;
    if (run_len && merge && dst == run_dst && row == run_row + run_len) {
      ++run_len;
      continue;
    }
    if (run_len) bulk_s2g(run_dst + run_row * row_bytes, oblock + run_t * src_row_bytes, run_len * row_bytes);
    run_dst = dst;
    run_row = row;
    run_t = t;
    run_len = 1;
  }
  if (run_len) bulk_s2g(run_dst + run_row * row_bytes, oblock + run_t * src_row_bytes, run_len * row_bytes);
}

// Shape of one row kernel instantiation.  FP16 rows are written back
// through two output stages in shared memory by bulk copies (fewer
// instructions per cell than scattered 2-byte stores: measured -8 % on the
// odd step, +2 % GLUPS at 256^3), where that fits with at least two input
// stages; FP32 keeps three input stages and stores directly (with output
// staging it would drop to two input stages: measured 0.78 instead of 0.88
// of the copy bandwidth).
template <class LAT, class ST, int P, int MINB>
struct RowCfg {
  static constexpr int kIn = RowLayout<LAT, ST, true, P>::kStageBytes;  // the odd step's (larger) stage
  static constexpr int kOut = (LAT::Q * P * (int)sizeof(ST) + 127) / 128 * 128;
  static constexpr int kBudget = MINB > 1 ? 110 * 1024 : 216 * 1024;
  static constexpr int kMaxIn = MINB > 1 ? 3 : 6;
  static constexpr int kInWithOut = (kBudget - 2 * kOut) / kIn;
  static constexpr bool kOuts = LBM_ROW_OUTS_F16 && sizeof(ST) == 2 && kInWithOut >= 2;
  static constexpr int kInOnly = kBudget / kIn;
  static constexpr int kNS = kOuts ? (kInWithOut < kMaxIn ? kInWithOut : kMaxIn) : (kInOnly < kMaxIn ? kInOnly : kMaxIn);
  static constexpr int kNOut = kOuts ? 2 : 0;
  static constexpr int kConsumers = row_consumers_single<MINB, row_pair_lattice<LAT, ST>()>();
  static constexpr int kThreads = (kConsumers + kRowProducers + (kOuts ? 1 : 0)) * 32;
  static constexpr int kSmem = kNS * kIn + kNOut * kOut;
  // static phi (no d_t phi blocks): a stage ends where the d_t phi blocks
  // would start; one-block-per-SM shapes then fit more stages in up to
  // 226 KB (D3Q27 at pitch 512: 3 instead of 2)
  static constexpr int kInS = RowLayout<LAT, ST, true, P>::kDepsOff;
  static constexpr int kBudgetS = MINB > 1 ? kBudget : 226 * 1024;
  static constexpr int kNSS0 = (kBudgetS - kNOut * kOut) / kInS;
  static constexpr int kNSS = kNSS0 > kNS ? (kNSS0 < kMaxIn ? kNSS0 : kMaxIn) : kNS;
  static constexpr int kSmemS = kNSS * kInS + kNOut * kOut;
};

// Warp-specialised row kernel.  Warps kConsumerWarps .. + kRowProducers - 1
// are the producers (one by default; producer p takes the block's tiles j =
// p, p + P, ...): a producer stages tile j into stage j % NSTAGE once the
// consumers have released the
// tile that used it before (empty barrier), writes the tile's row contexts
// and arms the full barrier with the byte count of the copies.  Each
// producer lane owns up to two blocks of the tile's copies, set up once per
// launch, so staging a tile costs a few instructions per lane per row
// besides the copies.  The consumer warps wait on the full barrier, update
// their chunks of the tile's rows and release the stage, one arrival per
// warp.
// NOUT > 0: the consumers write the updated tile into output stage j % NOUT
// (after the storer has released it: oempty), then arrive on ofull; the
// storer warp (the one after the producers) waits on ofull, copies the Q output blocks
// to their destination rows with bulk copies (lane i: population i), waits
// until the copies have read the stage and releases it.  No block-wide
// barrier is taken inside the loop.
// TUNED = false: row_consumers_single() consumer warps and RowCfg's input
// stages (kNS; kNSS when the launch asks for the static-phi layout),
// compile-time constants (the default shape).  TUNED = true: the launch
// chooses the consumer warps (blockDim.x / 32 minus the producer and storer
// warps, at most the default) and the input stages `nstage` (2 <= nstage <=
// MAXSTAGE), the autotuner's knobs; this generic form costs 2-5 % at the
// default shape (measured), so it runs only when a tuned shape differs from
// the default, and only for plain steps.
template <class LAT, class ST, bool ODD, bool RED, bool WALLS, int PITCH, int MAXSTAGE, int MINB, int RS, int NOUT,
          bool TILED, bool TUNED = false>
__global__ void __launch_bounds__((row_consumers_single<MINB, row_pair_lattice<LAT, ST>()>() + kRowProducers +
                                   (NOUT ? 1 : 0)) * 32, MINB)
    step_row_kernel(const LatticeDev *__restrict__ Lp, int k, int nstage, int lay_static) {
  constexpr int Q = LAT::Q;
  using Lay = RowLayout<LAT, ST, ODD, PITCH>;
  constexpr int kOutBytes = (Q * PITCH * (int)sizeof(ST) + 127) / 128 * 128;
  // FP16 plain steps of D2Q9/D3Q19 update two adjacent cells per lane
  // (update_row_pair: bit-identical results, fewer instructions per cell)
  constexpr bool kPair = row_pair_lattice<LAT, ST>() && !RED && RS == 0;
  constexpr int kChunk = kPair ? 64 : 32;
  const int kConsumerWarps = TUNED ? (int)(blockDim.x >> 5) - kRowProducers - (NOUT ? 1 : 0)
                                   : row_consumers_single<MINB, row_pair_lattice<LAT, ST>()>();
  // input stages: MAXSTAGE is the static-phi count (RowCfg::kNSS); with
  // lay_static (phi without d_t phi, set by the launch) stages end where the
  // d_t phi blocks would start
  using Cfg = RowCfg<LAT, ST, PITCH, MINB>;
  const bool stat = Cfg::kNSS > Cfg::kNS && lay_static != 0;
  const int NSTAGE = TUNED ? nstage : (stat ? Cfg::kNSS : Cfg::kNS);
  const int kInStride = stat ? Lay::kDepsOff : Lay::kStageBytes;
  const int kInRegion = NSTAGE * (stat ? RowLayout<LAT, ST, true, PITCH>::kDepsOff
                                       : RowLayout<LAT, ST, true, PITCH>::kStageBytes);
  __shared__ LatticeDev Ls;
  __shared__ alignas(8) unsigned long long full[MAXSTAGE];
  __shared__ alignas(8) unsigned long long empty[MAXSTAGE];
  __shared__ alignas(8) unsigned long long ofull[NOUT > 0 ? NOUT : 1];
  __shared__ alignas(8) unsigned long long oempty[NOUT > 0 ? NOUT : 1];
  __shared__ RowCtx ctx[MAXSTAGE][TILED ? kMaxTileRows : 1];
  __shared__ volatile int abort_flag;
  extern __shared__ __align__(128) unsigned char stages[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  {
    const int *src = reinterpret_cast<const int *>(Lp);
    int *dst = reinterpret_cast<int *>(&Ls);
    for (int w = tid; w < (int)(sizeof(LatticeDev) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    for (int o = 0; o < NOUT; ++o) {
      mbar_init(&ofull[o], kConsumerWarps);
      mbar_init(&oempty[o], 1);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  const LatticeDev &L = Ls;
  if (stat && L.has_deps) {
    // launched for the static layout on a lattice whose phi has a time
    // derivative (the host keys its graphs by that, so this does not
    // happen): the d_t phi blocks would overrun a stage; report and leave
    if (tid == 0) atomicExch(L.status, 1);
    return;
  }
  const bool wy = (L.walls & 2u) != 0, wz = (L.walls & 4u) != 0;
  const int y_first = wy ? 1 : 0, nyf = wy ? L.ny - 2 : L.ny;
  const int z_first = wz ? 1 : 0, nzf = wz ? L.nz - 2 : L.nz;
  // tiles of R rows of one plane: tile it is rows y_first + (it % tpp) R ..
  // of plane z_first + it / tpp (the plane's last tile may be shorter);
  // TILED = false: one row per tile, staged at the compile-time pitch
  const int R = TILED ? tile_rows(PITCH, L.nxp) : 1;
  const int spitch = TILED ? L.nxp : PITCH;
  const int tpp = (nyf + R - 1) / R;
  const int ntiles = tpp * nzf;
  const unsigned limit = L.wait_limit;
  RedAcc acc;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) acc.v[j] = 0.0;

  if (warp >= kConsumerWarps && warp < kConsumerWarps + kRowProducers) {
    // ---------------- producer warp p: tiles j = p, p + P, p + 2P, ... of the
    // block (P producers), so that one warp's copy issue overlaps the other's
    const int pw = warp - kConsumerWarps;
    const bool withhold = L.withhold_copies != 0;
    const int ny = L.ny, nz = L.nz, nxp = L.nxp;
    const unsigned walls = L.walls;
    const TileCopy c0 = make_tile_copy<LAT, ST, ODD, PITCH>(L, lane);
    const TileCopy c1 = make_tile_copy<LAT, ST, ODD, PITCH>(L, lane + 32);
    // bytes of a tile of nr rows: per_row * nr + fixed
    const unsigned per_row = __reduce_add_sync(0xffffffffu, tile_copy_bytes(c0, 1, nxp) - tile_copy_bytes(c0, 0, nxp) +
                                                               tile_copy_bytes(c1, 1, nxp) - tile_copy_bytes(c1, 0, nxp));
    const unsigned fixed = __reduce_add_sync(0xffffffffu, tile_copy_bytes(c0, 0, nxp) + tile_copy_bytes(c1, 0, nxp));
    // tile it = blockIdx.x + j G is (ty, tz) = (it % tpp, it / tpp), carried
    // incrementally from one tile of this producer to its next
    const unsigned stride = (unsigned)kRowProducers * gridDim.x;
    const int it0 = (int)blockIdx.x + pw * (int)gridDim.x;
    const int step_y = (int)(stride % (unsigned)tpp), step_z = (int)(stride / (unsigned)tpp);
    int ty = it0 % tpp, tz = it0 / tpp;
    int issued_upto = -1;  // last tile index j whose copies this warp issued
    int j = pw;
    for (int it = it0; it < ntiles; it += (int)stride, j += kRowProducers) {
      const int s = j % NSTAGE;
      if (j >= NSTAGE) {
        // the consumers released tile j - NSTAGE from this stage
        if (!mbar_wait_or_abort(&empty[s], (unsigned)(((j / NSTAGE) - 1) & 1), limit, &abort_flag)) {
          if (lane == 0 && !abort_flag) {
            abort_flag = 1;
            atomicExch(L.status, 1);
          }
          break;
        }
      }
      const int y0 = y_first + ty * R, z = z_first + tz, nr = min(R, nyf - ty * R);
      ty += step_y;
      tz += step_z;
      if (ty >= tpp) {
        ty -= tpp;
        ++tz;
      }
      fill_row_ctx(ctx[s], y0, z, nr, ny, nz, nxp, walls, lane);
      const unsigned bytes = per_row * (unsigned)nr + fixed;
      __syncwarp();
      if (!withhold) {
        if (lane == 0) mbar_arrive_expect_tx(&full[s], bytes);
        __syncwarp();
        unsigned char *stage = stages + s * kInStride;
        issue_tile_copy(c0, stage, &full[s], y0, z, nr, ny, nz, nxp, walls, spitch);
        issue_tile_copy(c1, stage, &full[s], y0, z, nr, ny, nz, nxp, walls, spitch);
        issued_upto = j;
      }
      __syncwarp();
    }
    if (abort_flag && lane == 0) {
      // drain: wait (full limit) for every stage whose copies this warp may
      // still have in flight
      for (int jj = issued_upto; jj >= 0 && jj > issued_upto - NSTAGE * kRowProducers; jj -= kRowProducers)
        mbar_wait_bounded(&full[jj % NSTAGE], (unsigned)((jj / NSTAGE) & 1));
    }
  } else if (NOUT > 0 && warp == kConsumerWarps + kRowProducers) {
    // ---------------- storer warp: lane i writes population i's block back
    int cy = 0, cz = 0;
    if (lane < Q) dir_yz<LAT>(lane, cy, cz);
    int j = 0;
    for (int it = blockIdx.x; it < ntiles; it += gridDim.x, ++j) {
      const int o = j % NOUT;
      if (!mbar_wait_or_abort(&ofull[o], (unsigned)((j / NOUT) & 1), limit, &abort_flag)) {
        if (lane == 0 && !abort_flag) {
          abort_flag = 1;
          atomicExch(L.status, 1);
        }
        break;
      }
      const int tz = it / tpp, ty = it - tz * tpp;
      const int y0 = y_first + ty * R, z = z_first + tz, nr = min(R, nyf - ty * R);
      if (lane < Q) {
        store_tile_block<LAT, ST, ODD>(L, stages + kInRegion + o * kOutBytes + lane * PITCH * (int)sizeof(ST), lane,
                                       cy, cz, y0, z, nr, spitch);
        bulk_commit();
        bulk_wait_read_all();
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&oempty[o]);
    }
    if (lane < Q) bulk_wait_all();
  } else {
    // ---------------- consumer warps
    const long long n = L.n + k;
    // steps since the phi and force references, converted once per launch
    const float dn = (float)(n - L.n_eps), dn_force = (float)(n - L.n_force);
    const int ncr = (L.nx + kChunk - 1) / kChunk;  // chunks per row
    int rot = 0;  // chunks dealt so far, modulo the consumer warps (all warps agree)
    int j = 0;
    for (int it = blockIdx.x; it < ntiles; it += gridDim.x, ++j) {
      const int s = j % NSTAGE;
      if (!mbar_wait_or_abort(&full[s], (unsigned)((j / NSTAGE) & 1), limit, &abort_flag)) {
        if (lane == 0 && !abort_flag) {
          abort_flag = 1;
          atomicExch(L.status, 1);
        }
        break;
      }
      unsigned char *ostage = nullptr;
      if (NOUT > 0) {
        const int o = j % NOUT;
        // the storer has finished reading tile j - NOUT from this output stage
        if (j >= NOUT && !mbar_wait_or_abort(&oempty[o], (unsigned)(((j / NOUT) - 1) & 1), limit, &abort_flag)) {
          if (lane == 0 && !abort_flag) {
            abort_flag = 1;
            atomicExch(L.status, 1);
          }
          break;
        }
        ostage = stages + kInRegion + o * kOutBytes;
      }
      const int tz = it / tpp, ty = it - tz * tpp;
      const int nr = min(R, nyf - ty * R);
      // the tile's chunks (row t, chunk c of the row), dealt round-robin to
      // the consumer warps across tiles so that every warp gets the same share
      const int nch = nr * ncr;
      const int first = (warp - rot + kConsumerWarps) % kConsumerWarps;
      const unsigned char *stage = stages + s * kInStride;
      for (int c = first; c < nch; c += kConsumerWarps) {
        const int t = c / ncr, xc = c - t * ncr;
        if constexpr (kPair)
          update_row_pair<LAT, ODD, WALLS, PITCH, (NOUT > 0), TILED>(L, stage, t, ctx[s][t], n, dn, dn_force,
                                                                     xc * kChunk + 2 * lane, ostage);
        else
          update_row_chunk<LAT, ST, ODD, RED, WALLS, PITCH, RS, (NOUT > 0), TILED>(
              L, stage, t, ctx[s][t], n, dn, dn_force, xc * kChunk + lane, acc, ostage);
      }
      rot = (rot + nch) % kConsumerWarps;
      if (NOUT > 0) fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&empty[s]);
        if (NOUT > 0) mbar_arrive(&ofull[j % NOUT]);
      }
    }
  }
  __syncthreads();
  if (RED) block_reduce_store(acc, L.partials, blockIdx.x);
}

}  // namespace lbm

namespace lbm {

// Host side: launch and planning of the row kernel for one lattice type.
// ls.row encodes the variant: bit 0 set = in use, bit 1 = walls, bit 2 =
// pitch 512 (else 256), bit 3 = tiles of several rows (rows of at most half
// the pitch).
template <class LAT, class ST, bool W, int P, int MINB, int RS, bool TL>
cudaError_t launch_row_rs(const LatticeDev *L_dev, bool odd, bool red, bool stat, int k, const StepLaunch &ls,
                          cudaStream_t s) {
  using C = RowCfg<LAT, ST, P, MINB>;
  constexpr int NS = C::kNSS, NO = C::kNOut;
  // static phi with a larger stage count: the static layout (stat)
  const bool st = stat && C::kNSS > C::kNS;
  const int ns_def = st ? C::kNSS : C::kNS;
  // a tuned shape (row_consumers, row_stages) other than the default runs the
  // generic instantiation, for plain steps only
  const int nc = ls.row_consumers > 0 && ls.row_consumers <= C::kConsumers ? ls.row_consumers : C::kConsumers;
  // (a planned stage count equal to the default is the default)
  const int ns = ls.row_stages >= 2 && ls.row_stages < C::kNS ? ls.row_stages : ns_def;
  const dim3 grid(ls.row_grid);
  const int lay = st ? 1 : 0;
  if (RS == 0 && !red && (nc != C::kConsumers || ns != ns_def)) {
    const dim3 block((nc + kRowProducers + (NO ? 1 : 0)) * 32);
    const int smem = ns * (st ? C::kInS : C::kIn) + NO * C::kOut;
    if (odd)
      step_row_kernel<LAT, ST, true, false, W, P, NS, MINB, RS, NO, TL, true><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
    else
      step_row_kernel<LAT, ST, false, false, W, P, NS, MINB, RS, NO, TL, true><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
    return cudaGetLastError();
  }
  const dim3 block(C::kThreads);
  const int smem = st ? C::kSmemS : C::kSmem;
  if (odd) {
    if (red) step_row_kernel<LAT, ST, true, true, W, P, NS, MINB, RS, NO, TL><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
    else step_row_kernel<LAT, ST, true, false, W, P, NS, MINB, RS, NO, TL><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
  } else {
    if (red) step_row_kernel<LAT, ST, false, true, W, P, NS, MINB, RS, NO, TL><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
    else step_row_kernel<LAT, ST, false, false, W, P, NS, MINB, RS, NO, TL><<<grid, block, smem, s>>>(L_dev, k, ns, lay);
  }
  return cudaGetLastError();
}

// red: bit 0 a check step, bit 1 the step decodes with the shift of the
// previous phi (the first step after a refresh), bit 2 phi has no time
// derivative (static layout where it fits more stages)
template <class LAT, class ST, bool W, int P, int MINB, bool TL>
cudaError_t launch_row_v(const LatticeDev *L_dev, bool odd, int red, int k, const StepLaunch &ls,
                         cudaStream_t s) {
  if (red & 2) return launch_row_rs<LAT, ST, W, P, MINB, 1, TL>(L_dev, odd, (red & 1) != 0, (red & 4) != 0, k, ls, s);
  return launch_row_rs<LAT, ST, W, P, MINB, 0, TL>(L_dev, odd, (red & 1) != 0, (red & 4) != 0, k, ls, s);
}

template <class LAT, class ST, int MINB>
cudaError_t launch_row_t(const LatticeDev *L_dev, bool odd, int red, int k, const StepLaunch &ls,
                         cudaStream_t s) {
  const bool w = (ls.row & 2) != 0, p512 = (ls.row & 4) != 0, tl = (ls.row & 8) != 0;
  if (p512) {
    if (w) return launch_row_v<LAT, ST, true, 512, (MINB > 1 ? MINB - 1 : 1), false>(L_dev, odd, red, k, ls, s);
    return launch_row_v<LAT, ST, false, 512, (MINB > 1 ? MINB - 1 : 1), false>(L_dev, odd, red, k, ls, s);
  }
  if (tl) {
    if (w) return launch_row_v<LAT, ST, true, 256, MINB, true>(L_dev, odd, red, k, ls, s);
    return launch_row_v<LAT, ST, false, 256, MINB, true>(L_dev, odd, red, k, ls, s);
  }
  if (w) return launch_row_v<LAT, ST, true, 256, MINB, false>(L_dev, odd, red, k, ls, s);
  return launch_row_v<LAT, ST, false, 256, MINB, false>(L_dev, odd, red, k, ls, s);
}

template <class LAT, class ST, bool W, int P, int MINB, bool TL, bool ODD, bool RED, int RS, bool TUNED = false>
cudaError_t configure_row_one(int smem) {
  using C = RowCfg<LAT, ST, P, MINB>;
  return cudaFuncSetAttribute(step_row_kernel<LAT, ST, ODD, RED, W, P, C::kNSS, MINB, RS, C::kNOut, TL, TUNED>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class LAT, class ST, bool W, int P, int MINB, bool TL>
int configure_row_v(int &occ, int &nc, int &ns) {
  using C = RowCfg<LAT, ST, P, MINB>;
  static_assert(C::kNS >= 2, "a row kernel needs at least two stages");
  nc = nc > 0 && nc <= C::kConsumers ? nc : C::kConsumers;
  ns = ns >= 2 && ns <= C::kNS ? ns : C::kNS;
  const int smem_max = C::kSmemS > C::kSmem ? C::kSmemS : C::kSmem;
  if (smem_max > 226 * 1024) return 0;
  cudaError_t e = cudaSuccess;
#define LBM_CFG(ODD, RED, RS) \
  if (e == cudaSuccess) e = configure_row_one<LAT, ST, W, P, MINB, TL, ODD, RED, RS>(smem_max)
  LBM_CFG(true, false, 0);
  LBM_CFG(true, true, 0);
  LBM_CFG(false, false, 0);
  LBM_CFG(false, true, 0);
  LBM_CFG(true, false, 1);
  LBM_CFG(true, true, 1);
  LBM_CFG(false, false, 1);
  LBM_CFG(false, true, 1);
#undef LBM_CFG
  if (e == cudaSuccess) e = configure_row_one<LAT, ST, W, P, MINB, TL, true, false, 0, true>(smem_max);
  if (e == cudaSuccess) e = configure_row_one<LAT, ST, W, P, MINB, TL, false, false, 0, true>(smem_max);
  const int threads = (nc + kRowProducers + (C::kNOut ? 1 : 0)) * 32;
  const int smem = ns * C::kIn + C::kNOut * C::kOut;
  const bool tuned = nc != C::kConsumers || ns != C::kNS;
  if (e == cudaSuccess)
    e = tuned ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &occ, step_row_kernel<LAT, ST, true, false, W, P, C::kNSS, MINB, 0, C::kNOut, TL, true>, threads,
                    smem)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &occ, step_row_kernel<LAT, ST, true, false, W, P, C::kNSS, MINB, 0, C::kNOut, TL>, threads, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ >= 1;
}

template <class LAT, class ST, int MINB>
int plan_row_t(int nx, int nxp, int ny, int nz, unsigned walls, StepLaunch &ls) {
  if (nxp % 8 != 0 || nxp > 512 || nx < 8) return 0;
  if ((long long)nxp * ny * nz > 0x7fffffffLL) return 0;  // int cell indices
  if (walls & 1u) return 0;
  const bool w = (walls & 6u) != 0, p512 = nxp > 256;
  // rows of at most half the pitch are staged several at a time
  const int R = p512 ? 1 : tile_rows(256, nxp);
  // FP32 rows narrower than the pitch also take the tiled layout with
  // one-row tiles (halo blocks merged into one copy: 28 instead of 38 copies
  // per row; measured +11 % at 192^3, +9 % at 224^3); FP16, whose consumers
  // bound it, keeps the compile-time offsets
  const bool tl = R > 1 || (sizeof(ST) == 4 && !p512 && nxp < 256);
  int occ = 0, ok, nc = ls.row_consumers, ns = ls.row_stages;
  if (p512)
    ok = w ? configure_row_v<LAT, ST, true, 512, (MINB > 1 ? MINB - 1 : 1), false>(occ, nc, ns)
           : configure_row_v<LAT, ST, false, 512, (MINB > 1 ? MINB - 1 : 1), false>(occ, nc, ns);
  else if (tl)
    ok = w ? configure_row_v<LAT, ST, true, 256, MINB, true>(occ, nc, ns)
           : configure_row_v<LAT, ST, false, 256, MINB, true>(occ, nc, ns);
  else
    ok = w ? configure_row_v<LAT, ST, true, 256, MINB, false>(occ, nc, ns)
           : configure_row_v<LAT, ST, false, 256, MINB, false>(occ, nc, ns);
  if (!ok) return 0;
  ls.row_consumers = nc;
  ls.row_stages = ns;
  const int nyf = (walls & 2u) ? ny - 2 : ny;
  const int nzf = (walls & 4u) ? nz - 2 : nz;
  if (nyf < 1 || nzf < 1) return 0;
  // work items: tiles of R rows of one plane
  const long long ntiles = (long long)((nyf + R - 1) / R) * nzf;
  const int cap = sm_count() * occ;
  ls.row = 1 | (w ? 2 : 0) | (p512 ? 4 : 0) | (tl ? 8 : 0);
  ls.row_grid = ntiles < cap ? (int)ntiles : cap;
  ls.row_smem_odd = ls.row_smem_even = 0;
  return 1;
}

}  // namespace lbm
