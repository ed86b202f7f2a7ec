// batch.cu -- many independent lattices advanced by persistent,
// graph-captured kernels over device work tables.
//
// Members whose rows fit the row-staged kernel are grouped in classes
// (lattice, storage, row pitch 64/128/256/512, with or without y/z walls);
// each class has a row table and is stepped by one persistent batched row
// kernel per step (batch_row.cuh).  Other members (nx < 8, nx > 512, walls
// on x, or created for the one-cell-per-thread kernel) are listed as tiles
// (member, first cell, cell count) grouped by (lattice, storage) type and
// stepped by the tiled one-cell-per-thread kernel below.  Each member keeps
// its own descriptor (time counter, parity, phi, force), so members of any
// size, parity and age share one launch.  A replay of k steps is a CUDA
// graph: one chain of k launches per type and per class part (the members
// of a class whose time is even, or odd, at the replay start), concurrent
// (members of different classes are independent), then one advance kernel;
// the tables live in device memory, so members can join and leave
// (continuous batching) without re-capturing the graph.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm_vanse.h"
#include "internal.h"
#include "step_fast.cuh"

namespace lbm {
LatticeDev *handle_device_desc(lbm_vanse_t h);
const LatticeDev &handle_mirror(lbm_vanse_t h);
LatticeDev &handle_mirror_mut(lbm_vanse_t h);
int handle_push(lbm_vanse_t h);
int handle_push_changed(lbm_vanse_t h, LatticeDev *last, int *pushed);
cudaStream_t handle_stream(lbm_vanse_t h);
void set_global_error(const char *msg);
int sm_count();
// batched row kernel, one entry per lattice type and storage
// (batch_row_*_f32.cu, batch_row_*_f16.cu); the shape class selects the row
// pitch 64, 128, 256 or 512 (bits 0-1) and walls on y/z (bit 2)
#define LBM_BR_DECL(NAME)                                                                                   \
  cudaError_t launch_batch_row_##NAME(int, int, int, int, const BatchMember *, const int *, const int *,     \
                                      const int2 *, double *, int *, int, int, int, int, cudaStream_t);      \
  int configure_batch_row_##NAME(int shape);
LBM_BR_DECL(d2q9_f32)
LBM_BR_DECL(d2q9_f16)
LBM_BR_DECL(d3q19_f32)
LBM_BR_DECL(d3q19_f16)
LBM_BR_DECL(d3q27_f32)
LBM_BR_DECL(d3q27_f16)
#undef LBM_BR_DECL
}  // namespace lbm

using namespace lbm;

namespace {

constexpr int kTypes = 8;  // (lattice 0..3) x (storage fp32, fp16); D1Q3 members use the tiled kernel only
constexpr int kBatchBlock = 256;
constexpr int kPitchClasses = 8;                     // shape codes: row pitch 256/512 (2, 3), with or without y/z walls (+4)
constexpr int kRowClasses = kTypes * kPitchClasses;  // batched row kernel classes
constexpr int kParts = 2 * kRowClasses;  // class x parity of the member's time at the replay start
constexpr int kLanes = kTypes + kParts;  // concurrent chains of a replay

int type_of(int lattice, int storage) { return lattice * 2 + (storage == 2 ? 1 : 0); }

// Per-type tile ranges [begin, count] live at type_range[2*type].
struct BatchRange {
  int begin, count;
};

template <class LAT, class ST, bool RED>
__global__ void __launch_bounds__(kBatchBlock) batch_step_kernel(const BatchMember *__restrict__ members,
                                                                 const BatchTile *__restrict__ tiles,
                                                                 const BatchRange *__restrict__ range,
                                                                 int k, int kmax, double *tile_partials) {
  const int begin = range->begin, count = range->count;
  for (int t = blockIdx.x; t < count; t += gridDim.x) {
    const BatchTile tile = tiles[begin + t];
    const BatchMember &M = members[tile.member];
    const long long budget = M.budget;
    if (k >= budget) continue;  // member finished inside this replay
    const LatticeDev &L = *M.L;
    const long long n = L.n + k;
    const long long last = (budget < kmax ? budget : kmax) - 1;
    const bool red_here = RED && k == last;
    const int nx = L.nx, ny = L.ny, nxp = L.nxp;
    const int c_end = tile.y0 + tile.ny;  // y0 = first stored cell, ny = cell count (linear tile)
    RedAcc acc;
#pragma unroll
    for (int j = 0; j < kRedWidth; ++j) acc.v[j] = 0.0;
    for (int c = tile.y0 + threadIdx.x; c < c_end; c += blockDim.x) {
      const int x = c % nxp;
      if (x >= nx) continue;  // row padding
      const int r = c / nxp;
      const int y = r % ny;
      const int z = r / ny;
      if (red_here) {
        if (n & 1) update_cell_fast<LAT, ST, true, true>(L, n, x, y, z, acc, k == 0);
        else update_cell_fast<LAT, ST, false, true>(L, n, x, y, z, acc, k == 0);
      } else {
        if (n & 1) update_cell_fast<LAT, ST, true, false>(L, n, x, y, z, acc, k == 0);
        else update_cell_fast<LAT, ST, false, false>(L, n, x, y, z, acc, k == 0);
      }
    }
    if (red_here) {
      block_reduce_store(acc, tile_partials, begin + t);
      __syncthreads();
    }
  }
}

// After a replay of k steps: every member advances by min(k, budget).
__global__ void batch_advance_kernel(BatchMember *members, const int *nmembers, int k) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= *nmembers) return;
  BatchMember &M = members[m];
  const long long s = M.budget < k ? M.budget : k;
  if (s <= 0) return;
  M.L->n += s;
  M.L->sig_rd = M.L->sig_wr;
  M.budget -= s;
}

// Per-member sums of its tiles' partials, in tile order.
// Row members: their sums were accumulated by the batched row kernel.
__global__ void batch_finalize_kernel(const BatchMember *members, const int *nmembers,
                                      const double *tile_partials, const double *member_sums, double *out) {
  const int m = blockIdx.x;
  if (m >= *nmembers) return;
  const int j = threadIdx.x;
  if (j >= kRedWidth) return;
  const BatchMember &M = members[m];
  double s = 0.0;
  if (M.row) {
    s = member_sums[(long long)m * kRedWidth + j];
  } else {
    for (int t = M.tile_begin; t < M.tile_end; ++t) s += tile_partials[(long long)t * kRedWidth + j];
  }
  out[(long long)m * kRedWidth + j] = s;
}

cudaError_t launch_row_class(int cls, int odd, const BatchMember *members, const int *row_member,
                             const int *row_begin, const int2 *cls_dev, double *member_sums, int *status, int k,
                             int kmax, int red, int grid, cudaStream_t s) {
  const int type = cls / kPitchClasses, pclass = cls % kPitchClasses;
  const int first = k == 0;
#define LBM_BR_CALL(NAME) \
  return launch_batch_row_##NAME(pclass, odd, red, first, members, row_member, row_begin, cls_dev, member_sums, \
                                 status, k, kmax, red, grid, s)
  switch (type) {
    case 0: LBM_BR_CALL(d2q9_f32);
    case 1: LBM_BR_CALL(d2q9_f16);
    case 2: LBM_BR_CALL(d3q19_f32);
    case 3: LBM_BR_CALL(d3q19_f16);
    case 4: LBM_BR_CALL(d3q27_f32);
    case 5: LBM_BR_CALL(d3q27_f16);
  }
#undef LBM_BR_CALL
  return cudaErrorInvalidValue;
}

// Resident blocks x SMs of a row class; 0 when it cannot run.
int row_class_grid(int cls) {
  const int type = cls / kPitchClasses, pclass = cls % kPitchClasses;
  int occ = 0;
  switch (type) {
    case 0: occ = configure_batch_row_d2q9_f32(pclass); break;
    case 1: occ = configure_batch_row_d2q9_f16(pclass); break;
    case 2: occ = configure_batch_row_d3q19_f32(pclass); break;
    case 3: occ = configure_batch_row_d3q19_f16(pclass); break;
    case 4: occ = configure_batch_row_d3q27_f32(pclass); break;
    case 5: occ = configure_batch_row_d3q27_f16(pclass); break;
  }
  return occ > 0 ? occ * sm_count() : 0;
}

template <class LAT, class ST>
cudaError_t launch_type(const BatchMember *members, const BatchTile *tiles, const BatchRange *range,
                        int k, int kmax, int red, double *partials, int grid, cudaStream_t s) {
  if (red)
    batch_step_kernel<LAT, ST, true><<<grid, kBatchBlock, 0, s>>>(members, tiles, range, k, kmax, partials);
  else
    batch_step_kernel<LAT, ST, false><<<grid, kBatchBlock, 0, s>>>(members, tiles, range, k, kmax, partials);
  return cudaGetLastError();
}

cudaError_t launch_batch_type(int type, const BatchMember *members, const BatchTile *tiles,
                              const BatchRange *range, int k, int kmax, int red, double *partials,
                              int grid, cudaStream_t s) {
  switch (type) {
    case 0: return launch_type<D2Q9, float>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 1: return launch_type<D2Q9, __half>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 2: return launch_type<D3Q19, float>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 3: return launch_type<D3Q19, __half>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 4: return launch_type<D3Q27, float>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 5: return launch_type<D3Q27, __half>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 6: return launch_type<D1Q3, float>(members, tiles, range, k, kmax, red, partials, grid, s);
    case 7: return launch_type<D1Q3, __half>(members, tiles, range, k, kmax, red, partials, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

struct HostMember {
  lbm_vanse_t h;
  long long budget;
  int type;
  int row_class;  // batched row kernel class, or -1 (one-cell-per-thread tiles)
  LatticeDev pushed;  // the descriptor as the device holds it (valid after the first push)
  int group;      // parity of the member's time when the row tables were built
  int nrows;      // work items of the batched row kernel (tiles of up to 8 fluid rows)
  long long last_check_n;
  bool have_prev;
  double stats[kRedWidth];
  long long stats_n;
  long long check_k;
};

struct lbm_vanse_batch {
  cudaStream_t stream = nullptr;
  int max_members = 0, max_tiles = 0, tile_cells = 0;
  std::vector<HostMember> members;
  BatchMember *members_dev = nullptr;
  BatchTile *tiles_dev = nullptr;
  BatchRange *ranges_dev = nullptr;  // kTypes entries
  int *nmembers_dev = nullptr;
  double *tile_partials = nullptr;
  double *out_dev = nullptr;
  double *out_host = nullptr;
  bool dirty = true;
  int ntiles = 0;
  int grid = 0;
  // (chains present: one character per lane, k*2+red)
  std::map<std::pair<std::string, long long>, cudaGraphExec_t> graphs;
  std::vector<BatchMember> members_host;
  BatchMember *members_pinned = nullptr;  // max_members: the per-replay upload of the member table
  std::vector<BatchTile> tiles_host;
  std::vector<BatchRange> ranges_host;
  // batched row kernel: class row tables, per-member sums, wait status
  int *row_member_dev = nullptr;
  long long row_cap = 0;
  int *row_begin_dev = nullptr;   // max_members
  int2 *cls_dev = nullptr;        // kParts (first row, rows)
  double *member_sums = nullptr;  // max_members x kRedWidth
  int *status_dev = nullptr;
  int *status_host = nullptr;
  int class_grid[kRowClasses] = {};  // 0: not configured yet, -1: cannot run
  // capture: every class (and cell-kernel type) runs its k steps as its own
  // chain on a side stream; the chains are independent and run concurrently
  cudaStream_t side[kLanes] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kLanes] = {};
  std::vector<int> rows_host, row_begin_host;
  std::vector<int2> cls_host;
};

static int bfail(int code, const char *msg) {
  set_global_error(msg);
  return code;
}

extern "C" int lbm_vanse_batch_create(int max_members, int max_tiles, int tile_cells, void *stream,
                                      lbm_vanse_batch_t *out) {
  if (!out) return bfail(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_members < 1 || max_tiles < 1) return bfail(LBM_EINVAL, "max_members and max_tiles must be >= 1");
  if (tile_cells < 0) return bfail(LBM_EINVAL, "tile_cells must be >= 0");
  lbm_vanse_batch_t b = new lbm_vanse_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  b->max_members = max_members;
  b->max_tiles = max_tiles;
  b->tile_cells = tile_cells > 0 ? tile_cells : 4096;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_step_kernel<D3Q19, __half, false>, kBatchBlock, 0);
  if (occ < 1) occ = 1;
  b->grid = sm_count() * occ;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&b->members_dev, sizeof(BatchMember) * max_members);
  if (e == cudaSuccess) e = cudaMalloc(&b->tiles_dev, sizeof(BatchTile) * max_tiles);
  if (e == cudaSuccess) e = cudaMalloc(&b->ranges_dev, sizeof(BatchRange) * kTypes);
  if (e == cudaSuccess) e = cudaMalloc(&b->nmembers_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->tile_partials, sizeof(double) * kRedWidth * max_tiles);
  if (e == cudaSuccess) e = cudaMalloc(&b->out_dev, sizeof(double) * kRedWidth * max_members);
  if (e == cudaSuccess) e = cudaMallocHost(&b->out_host, sizeof(double) * kRedWidth * max_members);
  if (e == cudaSuccess) e = cudaMalloc(&b->row_begin_dev, sizeof(int) * max_members);
  if (e == cudaSuccess) e = cudaMalloc(&b->cls_dev, sizeof(int2) * kParts);
  if (e == cudaSuccess) e = cudaMalloc(&b->member_sums, sizeof(double) * kRedWidth * max_members);
  if (e == cudaSuccess) e = cudaMalloc(&b->status_dev, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->status_host, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->members_pinned, sizeof(BatchMember) * max_members);
  if (e == cudaSuccess) e = cudaMemset(b->status_dev, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbm_vanse_batch_destroy(b);
    return bfail(LBM_ENOMEM, "batch table allocation failed");
  }
  *out = b;
  return LBM_OK;
}

extern "C" void lbm_vanse_batch_destroy(lbm_vanse_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
  cudaFree(b->members_dev);
  cudaFree(b->tiles_dev);
  cudaFree(b->ranges_dev);
  cudaFree(b->nmembers_dev);
  cudaFree(b->tile_partials);
  cudaFree(b->out_dev);
  if (b->out_host) cudaFreeHost(b->out_host);
  cudaFree(b->row_member_dev);
  cudaFree(b->row_begin_dev);
  cudaFree(b->cls_dev);
  cudaFree(b->member_sums);
  cudaFree(b->status_dev);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->members_pinned) cudaFreeHost(b->members_pinned);
  for (int i = 0; i < kLanes; ++i) {
    if (b->side[i]) cudaStreamDestroy(b->side[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
}

static int tiles_needed(const lbm_vanse_batch *b, long long ncell) {
  return (int)((ncell + b->tile_cells - 1) / b->tile_cells);
}

extern "C" int lbm_vanse_batch_add(lbm_vanse_batch_t b, lbm_vanse_t h, long long max_steps) {
  if (!b || !h) return bfail(LBM_EINVAL, "NULL argument");
  if (max_steps < 0) return bfail(LBM_EINVAL, "max_steps must be >= 0");
  const LatticeDev &m = handle_mirror(h);
  if (m.storage == 0) return bfail(LBM_EINVAL, "batch members must use FP32 or FP16 storage");
  for (auto &hm : b->members)
    if (hm.h == h) return bfail(LBM_EINVAL, "lattice is already a member");
  if ((int)b->members.size() >= b->max_members) return bfail(LBM_ENOMEM, "batch member table is full");
  // residual tracking needs the previous check's velocity
  LatticeDev &mm = handle_mirror_mut(h);
  if (!mm.u_prev) {
    void *p = nullptr;
    if (cudaMallocAsync(&p, (size_t)3 * mm.ncell * sizeof(float), handle_stream(h)) != cudaSuccess) {
      cudaGetLastError();
      return bfail(LBM_ENOMEM, "residual buffer allocation failed");
    }
    mm.u_prev = static_cast<float *>(p);
  }
  HostMember hm;
  memset(&hm, 0, sizeof(hm));
  hm.h = h;
  hm.budget = max_steps;
  hm.type = type_of(m.lattice, m.storage);
  hm.row_class = -1;
  // the batched row kernel takes the member unless its lattice was created
  // for the one-cell-per-thread kernel (explicitly, or by its drag law or
  // closure), is one-dimensional, or its rows do not fit the kernel
  lbm_vanse_params p;
  if (lbm_vanse_get_params(h, &p) == LBM_OK && p.kernel != 1 /* one cell per thread */ && !p.drag_model &&
      !(p.les_cs > 0.0) && m.lattice != LBM_D1Q3 && m.nx >= 8 && m.nxp <= 512 && !(m.walls & 1u) &&
      m.ncell <= 0x7fffffffLL) {
    const int nyf = (m.walls & 2u) ? m.ny - 2 : m.ny, nzf = (m.walls & 4u) ? m.nz - 2 : m.nz;
    const int pitch = m.nxp <= 256 ? 256 : 512;
    const int pclass = (pitch == 256 ? 2 : 3) | ((m.walls & 6u) ? 4 : 0);
    const int cls = hm.type * kPitchClasses + pclass;
    if (b->class_grid[cls] == 0) {
      const int g = row_class_grid(cls);
      b->class_grid[cls] = g > 0 ? g : -1;
    }
    if (nyf >= 1 && nzf >= 1 && b->class_grid[cls] > 0) {
      hm.row_class = cls;
      // tiles of R rows of one plane (the kernel's tile_rows)
      const int R = std::max(1, std::min(8, pitch / (int)m.nxp));
      hm.nrows = (nyf + R - 1) / R * nzf;
    }
  }
  if (hm.row_class < 0) {
    // one-cell-per-thread members hold tiles of the tile table
    int used = 0;
    for (auto &o : b->members)
      if (o.row_class < 0) used += tiles_needed(b, handle_mirror(o.h).ncell);
    if (used + tiles_needed(b, m.ncell) > b->max_tiles) return bfail(LBM_ENOMEM, "batch tile table is full");
  }
  hm.last_check_n = -1;
  hm.stats_n = -1;
  b->members.push_back(hm);
  b->dirty = true;
  return (int)b->members.size() - 1;
}

extern "C" int lbm_vanse_batch_remove(lbm_vanse_batch_t b, lbm_vanse_t h) {
  if (!b || !h) return bfail(LBM_EINVAL, "NULL argument");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i].h == h) {
      b->members.erase(b->members.begin() + i);
      b->dirty = true;
      return LBM_OK;
    }
  return bfail(LBM_EINVAL, "lattice is not a member");
}

extern "C" int lbm_vanse_batch_size(lbm_vanse_batch_t b) { return b ? (int)b->members.size() : 0; }

// Rebuild and upload the member and tile tables (sorted by type).
static int upload_tables(lbm_vanse_batch_t b) {
  const int nm = (int)b->members.size();
  if (!b->dirty) {
    // membership unchanged: only the budgets move; one asynchronous copy
    // from pinned memory (the previous replay's copy has completed: its
    // replay was synchronised)
    for (int i = 0; i < nm; ++i) {
      b->members_host[i].budget = b->members[i].budget;
      b->members_pinned[i] = b->members_host[i];
    }
    if (nm && cudaMemcpyAsync(b->members_dev, b->members_pinned, sizeof(BatchMember) * nm, cudaMemcpyHostToDevice,
                              b->stream) != cudaSuccess)
      return bfail(LBM_ECUDA, "member table upload failed");
    return LBM_OK;
  }
  b->members_host.assign(nm, BatchMember());
  b->tiles_host.clear();
  b->ranges_host.assign(kTypes, BatchRange{0, 0});
  for (int t = 0; t < kTypes; ++t) {
    b->ranges_host[t].begin = (int)b->tiles_host.size();
    for (int i = 0; i < nm; ++i) {
      HostMember &hm = b->members[i];
      if (hm.type != t) continue;
      const LatticeDev &m = handle_mirror(hm.h);
      BatchMember &bm = b->members_host[i];
      bm.L = handle_device_desc(hm.h);
      bm.budget = hm.budget;
      bm.lattice = m.lattice;
      bm.storage = m.storage;
      bm.row = hm.row_class >= 0 ? 1 : 0;
      bm.tile_begin = (int)b->tiles_host.size();
      for (long long c = 0; !bm.row && c < m.ncell; c += b->tile_cells) {
        BatchTile tl;
        tl.member = i;
        tl.z = 0;
        tl.y0 = (int)c;
        tl.ny = (int)((m.ncell - c) < b->tile_cells ? (m.ncell - c) : b->tile_cells);
        tl.x0 = 0;
        tl.nxt = 0;
        b->tiles_host.push_back(tl);
      }
      bm.tile_end = (int)b->tiles_host.size();
    }
    b->ranges_host[t].count = (int)b->tiles_host.size() - b->ranges_host[t].begin;
  }
  b->ntiles = (int)b->tiles_host.size();
  cudaStream_t s = b->stream;
  cudaError_t e = cudaSuccess;
  if (b->dirty) {
    // class item tables: the tiles of each class, member after member
    b->rows_host.clear();
    b->row_begin_host.assign(nm, 0);
    b->cls_host.assign(kParts, make_int2(0, 0));
    for (int c = 0; c < kParts; ++c) {
      const int base = (int)b->rows_host.size();
      for (int i = 0; i < nm; ++i) {
        const HostMember &hm = b->members[i];
        if (hm.row_class < 0 || hm.row_class * 2 + hm.group != c) continue;
        b->row_begin_host[i] = (int)b->rows_host.size() - base;
        b->rows_host.insert(b->rows_host.end(), (size_t)hm.nrows, i);
      }
      b->cls_host[c] = make_int2(base, (int)b->rows_host.size() - base);
    }
    const long long nrows = (long long)b->rows_host.size();
    if (nrows > b->row_cap) {
      // a new table: graphs that captured the old pointer are dropped
      if (b->stream) cudaStreamSynchronize(b->stream);
      else cudaDeviceSynchronize();
      cudaFree(b->row_member_dev);
      b->row_member_dev = nullptr;
      b->row_cap = 0;
      for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
      b->graphs.clear();
      const long long cap = nrows + nrows / 2 + 1024;
      if (cudaMalloc(&b->row_member_dev, sizeof(int) * cap) != cudaSuccess) {
        cudaGetLastError();
        return bfail(LBM_ENOMEM, "batch row table allocation failed");
      }
      b->row_cap = cap;
    }
    if (nrows)
      e = cudaMemcpyAsync(b->row_member_dev, b->rows_host.data(), sizeof(int) * nrows, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nm)
      e = cudaMemcpyAsync(b->row_begin_dev, b->row_begin_host.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->cls_dev, b->cls_host.data(), sizeof(int2) * kParts, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && nm)
    e = cudaMemcpyAsync(b->members_dev, b->members_host.data(), sizeof(BatchMember) * nm, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && b->ntiles)
    e = cudaMemcpyAsync(b->tiles_dev, b->tiles_host.data(), sizeof(BatchTile) * b->ntiles, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->ranges_dev, b->ranges_host.data(), sizeof(BatchRange) * kTypes, cudaMemcpyHostToDevice, s);
  static thread_local int nm_host;
  nm_host = nm;
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->nmembers_dev, &nm_host, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  b->dirty = false;
  return LBM_OK;
}

// lanes: one character per chain ('1' present): kTypes cell-kernel types,
// then the row-class parts (class * 2 + parity group)
static int batch_graph(lbm_vanse_batch_t b, const std::string &lanes, int k, int red, cudaGraphExec_t *out) {
  auto key = std::make_pair(lanes, (long long)k * 2 + red);
  auto it = b->graphs.find(key);
  if (it != b->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  for (int lane = 0; lane < kLanes; ++lane)
    if (lanes[lane] == '1' && !b->side[lane]) {
      if (cudaStreamCreateWithFlags(&b->side[lane], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_join[lane], cudaEventDisableTiming) != cudaSuccess)
        return bfail(LBM_ECUDA, "side stream create");
    }
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return bfail(LBM_ECUDA, "stream create");
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess && red && lanes.find('1', kTypes) != std::string::npos)
    e = cudaMemsetAsync(b->member_sums, 0, sizeof(double) * kRedWidth * b->max_members, cs);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, cs);
  if (e == cudaSuccess) {
    // one chain of k launches per cell-kernel type and per row class
    for (int lane = 0; lane < kLanes && e == cudaSuccess; ++lane) {
      if (lanes[lane] != '1') continue;
      const bool cell = lane < kTypes;
      const int c = cell ? lane : lane - kTypes;  // type, or part = class * 2 + parity group
      cudaStream_t ss = b->side[lane];
      e = cudaStreamWaitEvent(ss, b->ev_fork, 0);
      for (int j = 0; j < k && e == cudaSuccess; ++j)
        e = cell ? launch_batch_type(c, b->members_dev, b->tiles_dev, b->ranges_dev + c, j, k, red,
                                     b->tile_partials, b->grid, ss)
                 : launch_row_class(c / 2, (c + j) & 1, b->members_dev, b->row_member_dev, b->row_begin_dev,
                                    b->cls_dev + c, b->member_sums, b->status_dev, j, k, red,
                                    b->class_grid[c / 2], ss);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev_join[lane], ss);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->ev_join[lane], 0);
    }
    if (e == cudaSuccess) {
      batch_advance_kernel<<<(b->max_members + 127) / 128, 128, 0, cs>>>(b->members_dev, b->nmembers_dev, k);
      e = cudaGetLastError();
    }
    if (red && e == cudaSuccess) {
      batch_finalize_kernel<<<b->max_members, 32, 0, cs>>>(b->members_dev, b->nmembers_dev, b->tile_partials,
                                                           b->member_sums, b->out_dev);
      e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) {
    cudaGraphExec_t ge;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) {
      b->graphs[key] = ge;
      *out = ge;
    }
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" int lbm_vanse_batch_step(lbm_vanse_batch_t b, int k, int check) {
  if (!b) return bfail(LBM_EINVAL, "batch is NULL");
  if (k < 1) return bfail(LBM_EINVAL, "k must be >= 1");
  if (b->members.empty()) return LBM_OK;
  int rc;
  // members' descriptors must be current on the device (their own streams
  // may have pending uploads): synchronise those streams first
  std::string lanes(kLanes, '0');
  for (auto &hm : b->members) {
    LatticeDev &m = handle_mirror_mut(hm.h);
    m.have_prev = hm.have_prev ? 1 : 0;
    int pushed = 0;
    if ((rc = handle_push_changed(hm.h, &hm.pushed, &pushed))) return bfail(rc, "member descriptor upload failed");
    if (pushed || handle_stream(hm.h) != b->stream) cudaStreamSynchronize(handle_stream(hm.h));
    if (hm.row_class >= 0) {
      // members of one class are split by the parity of their time
      const int g = (int)(m.n & 1);
      if (g != hm.group) {
        hm.group = g;
        b->dirty = true;
      }
      lanes[kTypes + hm.row_class * 2 + g] = '1';
    } else {
      lanes[hm.type] = '1';
    }
  }
  if ((rc = upload_tables(b))) return rc;
  cudaGraphExec_t ge;
  if ((rc = batch_graph(b, lanes, k, check ? 1 : 0, &ge))) return rc;
  cudaError_t e = cudaGraphLaunch(ge, b->stream);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  count_launches((long long)k * (long long)std::count(lanes.begin(), lanes.end(), '1') + 1 + (check ? 1 : 0));
  if (check) {
    e = cudaMemcpyAsync(b->out_host, b->out_dev, sizeof(double) * kRedWidth * b->members.size(),
                        cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  }
  e = cudaMemcpyAsync(b->status_host, b->status_dev, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(LBM_ECUDA, cudaGetErrorString(e));
  if (*b->status_host) {
    cudaMemsetAsync(b->status_dev, 0, sizeof(int), b->stream);
    *b->status_host = 0;
    return bfail(LBM_ETIMEOUT, "a bounded wait in the batched row kernel gave up");
  }
  // host mirrors follow the device
  for (size_t i = 0; i < b->members.size(); ++i) {
    HostMember &hm = b->members[i];
    const long long s = hm.budget < k ? hm.budget : k;
    if (s <= 0) continue;
    LatticeDev &m = handle_mirror_mut(hm.h);
    const long long n_check = m.n + s - 1;
    m.n += s;
    m.sig_rd = m.sig_wr;
    // the device's copy moved the same way (advance kernel)
    hm.pushed.n += s;
    hm.pushed.sig_rd = hm.pushed.sig_wr;
    hm.budget -= s;
    if (check) {
      memcpy(hm.stats, b->out_host + i * kRedWidth, sizeof(hm.stats));
      hm.check_k = hm.last_check_n >= 0 ? n_check - hm.last_check_n : 0;
      hm.stats_n = n_check;
      hm.last_check_n = n_check;
      hm.have_prev = true;
    }
  }
  return LBM_OK;
}

extern "C" int lbm_vanse_batch_stats(lbm_vanse_batch_t b, lbm_vanse_t h, lbm_vanse_stats *out) {
  if (!b || !h || !out) return bfail(LBM_EINVAL, "NULL argument");
  for (auto &hm : b->members)
    if (hm.h == h) {
      memset(out, 0, sizeof(*out));
      const double *s = hm.stats;
      out->mass = s[0];
      out->momentum[0] = s[1];
      out->momentum[1] = s[2];
      out->momentum[2] = s[3];
      out->u_norm = std::sqrt(s[5]);
      out->force[0] = s[7];
      out->force[1] = s[8];
      out->force[2] = s[9];
      out->residual = (hm.check_k > 0 && s[5] > 0.0) ? std::sqrt(s[4]) / (hm.check_k * std::sqrt(s[5])) : -1.0;
      out->steps_done = handle_mirror(h).n;
      out->step_of_stats = hm.stats_n;
      out->nan_seen = s[6] > 0.0 || !std::isfinite(s[0]) || !std::isfinite(s[5]);
      out->converged = 0;
      return LBM_OK;
    }
  return bfail(LBM_EINVAL, "lattice is not a member");
}
