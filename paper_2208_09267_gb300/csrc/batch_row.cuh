// batch_row.cuh -- the row-staged fused step (step_row.cuh) over the tiles
// of many lattices in one persistent launch.
//
// A batch class is one (lattice, storage, row pitch, walls or none)
// combination.  Its work items are the tiles (R consecutive fluid rows of
// one plane, R = min(8, PITCH / nxp): short rows are staged several at a
// time) of every member of the class, member after member; the class item
// table maps an item to its member.  The items are dealt to the blocks in
// runs of up to 8 consecutive items (block b takes runs b, b + G, b + 2G,
// ..., G = grid size; shorter runs when the class has few items, so that
// every block gets work), so that a block's next tile is usually the next
// tile of the same member.  Each item carries its own member: the producer
// warp looks the member up when the item leaves the current member's range,
// copies the member's device descriptor into the stage beside the tile's
// populations and fields, and records in the stage context whether the
// tile is skipped (member's step budget spent) or a check step.  Members keep
// their own time: the items of a class are split by the parity of the
// member's time at the start of a replay, and each part is stepped by the
// even or odd instantiation as the steps alternate.  The consumers update
// the tile with the same per-cell code as a lattice stepped alone
// (update_row_chunk), so a member's populations are bit-identical alone and
// in any batch.
//
// Check-step sums are reduced per warp and added into per-member FP64 sums
// with atomics when the item's member changes (their summation order, not
// the per-cell values, depends on the schedule).
#pragma once

#include "step_row.cuh"

namespace lbm {

static_assert(sizeof(LatticeDev) % 16 == 0, "the descriptor is staged by one bulk copy");
constexpr int kDescBytes = (int)sizeof(LatticeDev);

// Stage context of the batched kernel.
struct BatchRowCtx {
  RowCtx rc[kMaxTileRows];
  int nr;      // rows of the tile
  int member;  // slot in the member table
  int flags;   // bit 0: skip, bit 2: check step
  float dn, dn_force;  // steps since the member's phi and force references
};

// Item sequence of a block: runs blockIdx.x, blockIdx.x + G, ... of len
// items each (len = nitems / (8 G), clamped to 1..8), cut at nitems.
// Producer and consumers walk it identically.
struct RowRuns {
  int run, t, nrows, len;
  __device__ __forceinline__ explicit RowRuns(int n) : run(blockIdx.x), t(0), nrows(n) {
    const int l = n / (8 * (int)gridDim.x);
    len = l < 1 ? 1 : (l > 8 ? 8 : l);
  }
  // current row, or -1 when the block is done
  __device__ __forceinline__ int row() {
    int r = run * len + t;
    if (r >= nrows && t != 0) {
      t = 0;
      run += gridDim.x;
      r = run * len;
    }
    return r < nrows ? r : -1;
  }
  __device__ __forceinline__ void next() {
    if (++t == len) {
      t = 0;
      run += gridDim.x;
    }
  }
};

// Shape of a class's kernel.  The batched kernel is bound by its producer
// warps (one per block, issuing every tile's copies; tiles of short rows
// keep the consumers waiting), so where two-stage blocks fit three to an SM
// it runs three blocks of 4 consumer warps (three producers per SM; measured
// +13 % on 64^3 lattices against two blocks of 7); else two blocks of 7
// consumers with as many stages as fit, or one block of 15.
template <class LAT, class ST, int P>
struct BatchRowCfg {
  static constexpr int kStage = RowLayout<LAT, ST, true, P>::kStageBytes;
  static constexpr int kMinB = 2 * kStage <= 70 * 1024 ? 3 : (2 * kStage <= 110 * 1024 ? 2 : 1);
  static constexpr int kBudget = kMinB == 3 ? 2 * kStage : (kMinB == 2 ? 110 * 1024 : 216 * 1024);
  static constexpr int kFit = kBudget / kStage;
  static constexpr int kStages = kFit > 12 ? 12 : kFit;
  static constexpr int kConsumers = kMinB == 3 ? 4 : row_consumers<kMinB>();
  static constexpr int kThreads = (kConsumers + 1) * 32;
};

// Warp sum of acc, added into the member's sums by lane 0; acc is cleared.
__device__ __forceinline__ void flush_member_sums(RedAcc &acc, double *sums) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kRedWidth; ++j) {
    double v = acc.v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0 && v != 0.0) atomicAdd(sums + j, v);
    acc.v[j] = 0.0;
  }
}

// REDC: a launch of a check replay (tiles may carry the check flag).  RS 2:
// the first step of a replay, where a member's phi refresh since its last
// step is still pending (its descriptor tells); RS 0: later steps (the
// descriptors' shifts are committed only after the replay, so they must not
// be read as pending there).
template <class LAT, class ST, int P, bool WALLS, bool ODD, bool REDC, int RS, int NSTAGE, int MINB>
__global__ void __launch_bounds__(BatchRowCfg<LAT, ST, P>::kThreads, MINB)
    batch_row_kernel(const BatchMember *__restrict__ members, const int *__restrict__ item_member,
                     const int *__restrict__ item_begin, const int2 *__restrict__ cls,
                     double *__restrict__ member_sums, int *status, int k, int kmax, int check) {
  constexpr int kStage = BatchRowCfg<LAT, ST, P>::kStage;
  constexpr int kConsumerWarps = BatchRowCfg<LAT, ST, P>::kConsumers;
  __shared__ alignas(8) unsigned long long full[NSTAGE];
  __shared__ alignas(8) unsigned long long empty[NSTAGE];
  __shared__ BatchRowCtx ctx[NSTAGE];
  // each stage's member descriptor (a named shared array, so that the
  // consumers' reads of it compile to shared-memory loads)
  __shared__ alignas(16) LatticeDev descs[NSTAGE];
  __shared__ volatile int abort_flag;
  extern __shared__ __align__(128) unsigned char stages[];
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    abort_flag = 0;
    mbar_fence_init();
  }
  __syncthreads();
  // the class's items are item_member[base, base + nitems)
  const int base = cls->x, nitems = cls->y;
  const unsigned limit = kWaitSpins;

  if (warp == kConsumerWarps) {
    // ---------------- producer warp
    int cur = -1;  // member whose copies c0, c1 are set up
    TileCopy c0, c1;
    float dn_m = 0.f, dnf_m = 0.f;
    int ny = 1, nz = 1, nxp = 8, y_first = 0, z_first = 0, nyf = 1, R = 1, tpp = 1, rb = 0, re = 0, flags_m = 0;
    unsigned walls = 0;
    const LatticeDev *Lg = nullptr;
    int issued_upto = -1;
    RowRuns runs(nitems);
    int j = 0;
    for (int r = runs.row(); r >= 0; runs.next(), r = runs.row(), ++j) {
      const int s = j % NSTAGE;
      if (j >= NSTAGE) {
        if (!mbar_wait_or_abort(&empty[s], (unsigned)(((j / NSTAGE) - 1) & 1), limit, &abort_flag)) {
          if (lane == 0 && !abort_flag) {
            abort_flag = 1;
            atomicExch(status, 1);
          }
          break;
        }
      }
      // the item's member: the current one while r stays in its item range
      const int m = (r >= rb && r < re) ? cur : item_member[base + r];
      if (m != cur) {
        cur = m;
        const BatchMember &M = members[m];
        Lg = M.L;
        const long long budget = M.budget;
        const long long last = (budget < kmax ? budget : kmax) - 1;
        rb = item_begin[m];
        ny = Lg->ny;
        nz = Lg->nz;
        nxp = Lg->nxp;
        walls = Lg->walls;
        y_first = (walls & 2u) ? 1 : 0;
        z_first = (walls & 4u) ? 1 : 0;
        nyf = (walls & 2u) ? ny - 2 : ny;
        R = tile_rows(P, nxp);
        tpp = (nyf + R - 1) / R;
        re = rb + tpp * ((walls & 4u) ? nz - 2 : nz);
        c0 = make_tile_copy<LAT, ST, ODD, P>(*Lg, lane);
        c1 = make_tile_copy<LAT, ST, ODD, P>(*Lg, lane + 32);
        flags_m = (k >= budget ? 1 : 0) | (REDC && check && k == last ? 4 : 0);
        // converted once per member, not per cell
        const long long n = Lg->n + k;
        dn_m = (float)(n - Lg->n_eps);
        dnf_m = (float)(n - Lg->n_force);
      }
      const int lt = r - rb;
      const int tz = lt / tpp, ty = lt - tz * tpp;
      const int y0 = y_first + ty * R, z = z_first + tz, nr = min(R, nyf - ty * R);
      fill_row_ctx(ctx[s].rc, y0, z, nr, ny, nz, nxp, walls, lane);
      const unsigned bytes =
          __reduce_add_sync(0xffffffffu, tile_copy_bytes(c0, nr, nxp) + tile_copy_bytes(c1, nr, nxp)) +
          (unsigned)kDescBytes;
      if (lane == 0) {
        ctx[s].nr = nr;
        ctx[s].member = m;
        ctx[s].flags = flags_m;
        ctx[s].dn = dn_m;
        ctx[s].dn_force = dnf_m;
      }
      __syncwarp();
      unsigned char *stage = stages + s * kStage;
      if (flags_m & 1) {
        if (lane == 0) mbar_arrive(&full[s]);  // nothing to stage: the phase completes
      } else {
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[s], bytes);
          bulk_g2s(&descs[s], Lg, (unsigned)kDescBytes, &full[s]);
        }
        __syncwarp();
        issue_tile_copy(c0, stage, &full[s], y0, z, nr, ny, nz, nxp, walls, nxp);
        issue_tile_copy(c1, stage, &full[s], y0, z, nr, ny, nz, nxp, walls, nxp);
      }
      issued_upto = j;
      __syncwarp();
    }
    if (abort_flag && lane == 0) {
      for (int jj = issued_upto - NSTAGE + 1; jj <= issued_upto; ++jj)
        if (jj >= 0) mbar_wait_bounded(&full[jj % NSTAGE], (unsigned)((jj / NSTAGE) & 1));
    }
  } else {
    // ---------------- consumer warps
    RedAcc acc;
#pragma unroll
    for (int q = 0; q < kRedWidth; ++q) acc.v[q] = 0.0;
    int red_m = -1;  // member whose check sums acc holds
    int rot = 0;     // chunks dealt so far, modulo the consumer warps (all warps agree)
    RowRuns runs(nitems);
    int j = 0;
    for (int r = runs.row(); r >= 0; runs.next(), r = runs.row(), ++j) {
      const int s = j % NSTAGE;
      if (!mbar_wait_or_abort(&full[s], (unsigned)((j / NSTAGE) & 1), limit, &abort_flag)) {
        if (lane == 0 && !abort_flag) {
          abort_flag = 1;
          atomicExch(status, 1);
        }
        break;
      }
      const int flags = ctx[s].flags;
      if (!(flags & 1)) {
        const unsigned char *data = stages + s * kStage;
        const LatticeDev &Lm = descs[s];
        const int m = ctx[s].member;
        const bool red = REDC && (flags & 4) != 0;
        if (red && m != red_m) {
          if (red_m >= 0) flush_member_sums(acc, member_sums + (long long)red_m * kRedWidth);
          red_m = m;
        }
        const long long n = Lm.n + k;
        const float dn = ctx[s].dn, dn_force = ctx[s].dn_force;
        // FP16 D2Q9/D3Q19 tiles without a check or a pending shift change
        // update two cells per lane, as a lattice stepped alone does
        // (update_row_pair: bit-identical to the one-cell update)
        constexpr bool kPairOK = row_pair_lattice<LAT, ST>() && RS == 0;
        const bool pair = kPairOK && !red;
        const int ncr = pair ? (Lm.nx + 63) >> 6 : (Lm.nx + 31) >> 5;
        const int nch = ctx[s].nr * ncr;
        const int first = (warp - rot + kConsumerWarps) % kConsumerWarps;
        for (int c = first; c < nch; c += kConsumerWarps) {
          const int t = c / ncr, xc = c - t * ncr;
          if constexpr (kPairOK) {
            if (pair) {
              update_row_pair<LAT, ODD, WALLS, P, false>(Lm, data, t, ctx[s].rc[t], n, dn, dn_force,
                                                         (xc << 6) + 2 * lane, nullptr);
              continue;
            }
          }
          const int x = (xc << 5) + lane;
          if (red)
            update_row_chunk<LAT, ST, ODD, REDC, WALLS, P, RS>(Lm, data, t, ctx[s].rc[t], n, dn, dn_force, x, acc);
          else
            update_row_chunk<LAT, ST, ODD, false, WALLS, P, RS>(Lm, data, t, ctx[s].rc[t], n, dn, dn_force, x, acc);
        }
        rot = (rot + nch) % kConsumerWarps;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    if (REDC && red_m >= 0) flush_member_sums(acc, member_sums + (long long)red_m * kRedWidth);
  }
}

// Host side: launch of one class part.
template <class LAT, class ST, int P, bool WALLS, bool ODD, bool REDC, int RS>
cudaError_t launch_batch_row_t(const BatchMember *members, const int *item_member, const int *item_begin,
                               const int2 *cls, double *member_sums, int *status, int k, int kmax,
                               int check, int grid, cudaStream_t s) {
  using C = BatchRowCfg<LAT, ST, P>;
  const int smem = C::kStage * C::kStages;
  batch_row_kernel<LAT, ST, P, WALLS, ODD, REDC, RS, C::kStages, C::kMinB><<<grid, C::kThreads, smem, s>>>(
      members, item_member, item_begin, cls, member_sums, status, k, kmax, check);
  return cudaGetLastError();
}

template <class LAT, class ST, int P, bool WALLS, bool ODD, bool REDC>
cudaError_t launch_batch_row_rs(bool first, const BatchMember *members, const int *item_member,
                                const int *item_begin, const int2 *cls, double *member_sums, int *status, int k,
                                int kmax, int check, int grid, cudaStream_t s) {
  if (first)
    return launch_batch_row_t<LAT, ST, P, WALLS, ODD, REDC, 2>(members, item_member, item_begin, cls, member_sums,
                                                               status, k, kmax, check, grid, s);
  return launch_batch_row_t<LAT, ST, P, WALLS, ODD, REDC, 0>(members, item_member, item_begin, cls, member_sums,
                                                             status, k, kmax, check, grid, s);
}

// first: the first step of the replay (k == 0)
template <class LAT, class ST, int P, bool WALLS>
cudaError_t launch_batch_row_t(bool odd, bool redc, bool first, const BatchMember *members,
                               const int *item_member, const int *item_begin, const int2 *cls,
                               double *member_sums, int *status, int k, int kmax, int check, int grid,
                               cudaStream_t s) {
  if (odd) {
    if (redc) return launch_batch_row_rs<LAT, ST, P, WALLS, true, true>(first, members, item_member, item_begin, cls,
                                                                         member_sums, status, k, kmax, check, grid, s);
    return launch_batch_row_rs<LAT, ST, P, WALLS, true, false>(first, members, item_member, item_begin, cls,
                                                                member_sums, status, k, kmax, check, grid, s);
  }
  if (redc) return launch_batch_row_rs<LAT, ST, P, WALLS, false, true>(first, members, item_member, item_begin, cls,
                                                                        member_sums, status, k, kmax, check, grid, s);
  return launch_batch_row_rs<LAT, ST, P, WALLS, false, false>(first, members, item_member, item_begin, cls,
                                                               member_sums, status, k, kmax, check, grid, s);
}

template <class LAT, class ST, int P, bool WALLS, bool ODD, bool REDC, int RS>
int configure_batch_row_v() {
  using C = BatchRowCfg<LAT, ST, P>;
  const int smem = C::kStage * C::kStages;
  auto *fn = batch_row_kernel<LAT, ST, P, WALLS, ODD, REDC, RS, C::kStages, C::kMinB>;
  int occ = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, C::kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ;
}

// Resident blocks per SM of a class: the least over its instantiations
// (after the shared-memory opt-in); 0 on failure.
template <class LAT, class ST, int P, bool WALLS>
int configure_batch_row_t() {
  static_assert(BatchRowCfg<LAT, ST, P>::kStages >= 2, "a class needs at least two stages");
  const int o[8] = {configure_batch_row_v<LAT, ST, P, WALLS, false, false, 0>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, true, false, 0>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, false, true, 0>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, true, true, 0>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, false, false, 2>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, true, false, 2>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, false, true, 2>(),
                    configure_batch_row_v<LAT, ST, P, WALLS, true, true, 2>()};
  int occ = o[0];
  for (int i = 1; i < 8; ++i) occ = o[i] < occ ? o[i] : occ;
  return occ;
}

}  // namespace lbm
