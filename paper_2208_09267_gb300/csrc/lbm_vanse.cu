// lbm_vanse.cu -- host implementation of the single-lattice C ABI
// (include/lbm_vanse.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbm_vanse.h"
#include "internal.h"
#include "lattice.cuh"

using lbm::LatticeDev;

namespace {

thread_local std::string g_last_error;

const int kQ[4] = {9, 19, 27, 3};
const int kD[4] = {2, 3, 3, 1};
const size_t kElem[3] = {8, 4, 2};
constexpr int kGraphChunk = 64;  // steps per captured graph (even)
constexpr size_t kRowGridBound = 4096;  // upper bound of the row kernel's grid

}  // namespace

struct lbm_vanse {
  lbm_vanse_params p;
  LatticeDev h;             // host mirror of the device descriptor
  LatticeDev *d = nullptr;  // device descriptor
  cudaStream_t stream = nullptr;
  int Q = 0, D = 0;
  long long N = 0;        // cells, nx*ny*nz (the caller's dense layout)
  long long Ni = 0;       // stored cells, nxp*ny*nz (rows padded to the pitch)
  int nxp = 0;
  void *pop = nullptr;
  void *eps_buf[2] = {nullptr, nullptr};
  __half *sig_buf[2] = {nullptr, nullptr};  // shift sigma of each phi_ref buffer
  int eps_cur = 0;
  void *deps_buf[2] = {nullptr, nullptr};  // d_t phi beside each phi_ref buffer
  void *force = nullptr, *dforce = nullptr;
  float *u_prev = nullptr;
  double *partials = nullptr;
  int nblocks = 0;
  double *stats_dev = nullptr;
  double *stats_host = nullptr;
  int *status = nullptr;
  lbm::StepLaunch ls;
  long long last_check_n = -1;
  std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;  // (parity, steps, phi has d_t phi)
  std::string err;
  size_t field_elem = 4;  // bytes of one phi / force value on the device
  // a phi refresh staged into the spare buffers (lbm_vanse_stage_epsilon)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_order = nullptr, ev_staged = nullptr;
  int staged = 0;          // awaits lbm_vanse_commit_epsilon
  int staged_deps = 0;     // carries d_t phi
  int staged_checked = 0;  // host values: scanned on the copy stream
  long long staged_n_ref = 0;
};

// ---------------------------------------------------------------- errors

static int fail(lbm_vanse_t h, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  if (h) h->err = buf;
  return code;
}

#define CUDA_TRY(h, call)                                                                     \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail((h), LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                  __FILE__, __LINE__);                                                        \
  } while (0)

extern "C" const char *lbm_vanse_version(void) { return "lbm_vanse 0.1 (sm_103a)"; }

extern "C" const char *lbm_vanse_last_error(lbm_vanse_t h) {
  if (h) return h->err.c_str();
  return g_last_error.c_str();
}

extern "C" int lbm_vanse_params_default(lbm_vanse_params *p) {
  if (!p) return fail(nullptr, LBM_EINVAL, "params is NULL");
  memset(p, 0, sizeof(*p));
  p->lattice = LBM_D3Q19;
  p->storage = LBM_FP32;
  p->nx = p->ny = p->nz = 32;
  p->tau = 0.6;
  p->rho0 = 1.0;
  p->fp16_scale_log2 = 10;
  return LBM_OK;
}

static int validate_params(const lbm_vanse_params *p, std::string &why) {
  char buf[256];
  if (!p) { why = "params is NULL"; return 0; }
  if (p->lattice < 0 || p->lattice > 3) {
    why = "lattice must be LBM_D2Q9, LBM_D3Q19, LBM_D3Q27 or LBM_D1Q3";
    return 0;
  }
  if (p->storage < 0 || p->storage > 2) { why = "storage must be LBM_FP64, LBM_FP32 or LBM_FP16_SHIFTED"; return 0; }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "nx, ny, nz must be >= 1"; return 0; }
  if (p->lattice == LBM_D2Q9 && p->nz != 1) { why = "D2Q9 needs nz = 1"; return 0; }
  if (p->lattice == LBM_D1Q3 && (p->ny != 1 || p->nz != 1)) { why = "D1Q3 needs ny = nz = 1"; return 0; }
  if (p->ny > 65535 * 256 || p->nz > 65535) { why = "ny or nz too large for the launch grid"; return 0; }
  if (!(p->tau > 0.5) || !std::isfinite(p->tau)) { why = "tau must be a finite value > 0.5"; return 0; }
  if (!(p->rho0 > 0.0) || !std::isfinite(p->rho0)) { why = "rho0 must be positive"; return 0; }
  const unsigned axes_mask = (1u << kD[p->lattice]) - 1u;
  if (p->quad_axes & ~axes_mask) { why = "quad_axes names an axis the lattice does not have"; return 0; }
  if (p->walls & ~axes_mask) { why = "walls names an axis the lattice does not have"; return 0; }
  const unsigned qa = p->quad_axes ? p->quad_axes : axes_mask;
  const int nbits = __builtin_popcount(qa);
  const int qd = p->quad_dim ? p->quad_dim : nbits;
  if (qd != -1 && (qd < 1 || qd > 3)) { why = "quad_dim must be 1, 2, 3 or -1 (pointwise)"; return 0; }
  for (int a = 0; a < 3; ++a) {
    const int n = a == 0 ? p->nx : (a == 1 ? p->ny : p->nz);
    if ((p->walls >> a) & 1u) {
      if (n < 3) {
        snprintf(buf, sizeof(buf), "a wall axis needs at least 3 cells (axis %d has %d)", a, n);
        why = buf;
        return 0;
      }
    }
  }
  if (p->storage == LBM_FP16_SHIFTED && (p->fp16_scale_log2 < -20 || p->fp16_scale_log2 > 24)) {
    why = "fp16_scale_log2 out of range [-20, 24]";
    return 0;
  }
  if (p->kernel < 0 || p->kernel > 2) { why = "kernel must be 0, 1 or 2"; return 0; }
  if (p->fp16_rounding < 0 || p->fp16_rounding > 1) { why = "fp16_rounding must be 0 or 1"; return 0; }
  if (p->quad_auto < 0 || p->quad_auto > 1) { why = "quad_auto must be 0 or 1"; return 0; }
  if (p->drag_model < 0 || p->drag_model > 1) { why = "drag_model must be 0 or 1"; return 0; }
  if (p->drag_model &&
      !(std::isfinite(p->drag_c1) && std::isfinite(p->drag_c2) && p->drag_c1 >= 0.0 && p->drag_c2 >= 0.0 &&
        std::isfinite(p->drag_d) && p->drag_d > 0.0)) {
    why = "drag needs finite c1, c2 >= 0 and a particle diameter d > 0";
    return 0;
  }
  if (!(std::isfinite(p->les_cs) && p->les_cs >= 0.0)) { why = "les_cs must be a finite value >= 0"; return 0; }
  if (p->row_consumers < 0 || p->row_consumers > 32 || p->row_stages < 0 || p->row_stages > 16) {
    why = "row_consumers must be in 0..32 and row_stages in 0..16";
    return 0;
  }
  if (p->kernel == 2 && (p->drag_model || p->les_cs > 0.0)) {
    why = "drag and the Smagorinsky closure run in the one-cell-per-thread kernel (kernel 0 or 1)";
    return 0;
  }
  if (p->kernel == 2 && p->storage == LBM_FP64) { why = "the row-staged kernel needs FP32 or FP16 storage"; return 0; }
  if (p->block_x < 0 || p->block_y < 0 || p->block_x * p->block_y > 256 ||
      (p->block_x > 0 && p->block_x % 32 != 0 && p->block_x * p->block_y % 32 != 0)) {
    why = "block shape must have at most 256 threads";
    return 0;
  }
  return 1;
}

static long long plane_of(long long N) { return (N + 63) / 64 * 64; }

// Stored row pitch: nx rounded up to 8 elements, so that every row of every
// field starts on a 16-byte boundary and is a whole number of 16-byte units
// (the bulk-copy rule), for 2-, 4- and 8-byte elements alike.
static int pitch_of(int nx) { return (nx + 7) / 8 * 8; }

extern "C" size_t lbm_vanse_device_bytes(const lbm_vanse_params *p, int with_deps, int with_force_field) {
  std::string why;
  if (!validate_params(p, why)) return 0;
  const long long N = (long long)pitch_of(p->nx) * p->ny * p->nz;  // stored cells
  const int Q = kQ[p->lattice];
  const size_t fe = p->storage == LBM_FP64 ? 8 : 4;
  size_t b = (size_t)Q * plane_of(N) * kElem[p->storage];  // populations
  b += 2 * (size_t)N * fe;                                  // phi double buffer
  if (p->storage != LBM_FP64) b += 2 * (size_t)N * 2;       // shift double buffer
  if (with_deps) b += 2 * (size_t)N * fe;                   // d_t phi double buffer
  if (with_force_field) b += 2 * 3 * (size_t)N * fe;
  const lbm::StepLaunch ls = lbm::make_launch(p->nx, p->ny, p->nz, p->block_x, p->block_y);
  size_t nb = (size_t)ls.grid.x * ls.grid.y * ls.grid.z;
  if (nb < kRowGridBound) nb = kRowGridBound;
  b += nb * lbm::kRedWidth * sizeof(double);
  b += 64 * sizeof(double) + sizeof(LatticeDev);
  return b;
}

static void sync_mirror_ptrs(lbm_vanse_t h) {
  LatticeDev &m = h->h;
  m.rho0f = (float)m.rho0;
  m.omegaf = (float)m.omega;
  m.cf3f = 3.0f * (float)m.cf;
  m.cf9f = 9.0f * (float)m.cf;
  m.qw0f = (float)m.qw0;
  m.qw1f = (float)m.qw1;
  for (int a = 0; a < 3; ++a) m.gf[a] = (float)m.g[a];
  m.cff = (float)m.cf;
  h->h.pop = h->pop;
  h->h.eps = h->eps_buf[h->eps_cur];
  h->h.deps = h->h.has_deps ? h->deps_buf[h->eps_cur] : nullptr;
  h->h.force = h->h.has_force ? h->force : nullptr;
  h->h.dforce = h->h.has_dforce ? h->dforce : nullptr;
  h->h.partials = h->partials;
  h->h.u_prev = h->u_prev;
  h->h.status = h->status;
}

static int push_mirror(lbm_vanse_t h) {
  sync_mirror_ptrs(h);
  CUDA_TRY(h, cudaMemcpyAsync(h->d, &h->h, sizeof(LatticeDev), cudaMemcpyHostToDevice, h->stream));
  return LBM_OK;
}

static void free_graphs(lbm_vanse_t h) {
  for (auto &kv : h->graphs) cudaGraphExecDestroy(kv.second);
  h->graphs.clear();
}

extern "C" void lbm_vanse_destroy(lbm_vanse_t h) {
  if (!h) return;
  free_graphs(h);
  cudaStream_t s = h->stream;
  // a staged copy may still be writing the spare buffers
  if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
  void *ptrs[] = {h->pop,       h->eps_buf[0], h->eps_buf[1], h->sig_buf[0], h->sig_buf[1],
                  h->deps_buf[0], h->deps_buf[1], h->force,     h->dforce,     h->u_prev,
                  h->partials,  h->stats_dev,  h->status,    h->d};
  for (void *q : ptrs)
    if (q) cudaFreeAsync(q, s);
  if (h->stats_host) cudaFreeHost(h->stats_host);
  cudaStreamSynchronize(s);
  if (h->ev_order) cudaEventDestroy(h->ev_order);
  if (h->ev_staged) cudaEventDestroy(h->ev_staged);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  delete h;
}

static int dev_alloc(lbm_vanse_t h, void **ptr, size_t bytes) {
  cudaError_t e = cudaMallocAsync(ptr, bytes, h->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(h, LBM_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  return LBM_OK;
}

extern "C" int lbm_vanse_create(const lbm_vanse_params *p, lbm_vanse_t *out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (!validate_params(p, why)) return fail(nullptr, LBM_EINVAL, "%s", why.c_str());
  const size_t need = lbm_vanse_device_bytes(p, 0, 0);
  if (p->hbm_budget_bytes && need > p->hbm_budget_bytes)
    return fail(nullptr, LBM_ENOMEM, "lattice needs %zu device bytes, budget is %zu", need,
                p->hbm_budget_bytes);

  lbm_vanse_t h = new lbm_vanse();
  h->p = *p;
  h->stream = static_cast<cudaStream_t>(p->cuda_stream);
  h->Q = kQ[p->lattice];
  h->D = kD[p->lattice];
  h->N = (long long)p->nx * p->ny * p->nz;
  h->nxp = pitch_of(p->nx);
  h->Ni = (long long)h->nxp * p->ny * p->nz;
  h->field_elem = p->storage == LBM_FP64 ? 8 : 4;
  const unsigned axes_mask = (1u << kD[p->lattice]) - 1u;
  const unsigned qa = p->quad_axes ? p->quad_axes : axes_mask;
  const int qd = p->quad_dim ? p->quad_dim : __builtin_popcount(qa);
  h->p.quad_axes = qa;
  h->p.quad_dim = qd;

  LatticeDev &m = h->h;
  memset(&m, 0, sizeof(m));
  m.nx = p->nx;
  m.ny = p->ny;
  m.nz = p->nz;
  m.lattice = p->lattice;
  m.ncell = h->Ni;
  m.plane = plane_of(h->Ni);
  m.nxp = h->nxp;
  m.walls = p->walls;
  m.quad_axes = qa;
  m.storage = p->storage;
  m.omega = 1.0 / p->tau;
  m.cf = 1.0 - 0.5 / p->tau;
  m.rho0 = p->rho0;
  m.wait_limit = 1u << 22;
  m.fp16_nearest = p->fp16_rounding == 1 ? 1 : 0;
  m.qw0 = lbm::quad_w0(qd);
  m.qw1 = lbm::quad_w1(qd);
  m.tau0 = p->tau;
  m.tau0f = (float)p->tau;
  m.drag_model = p->drag_model;
  if (p->drag_model) {
    m.drag_c1 = p->drag_c1;
    m.drag_c2 = p->drag_c2;
    m.drag_d = p->drag_d;
    const double nu = (p->tau - 0.5) / 3.0;
    m.drag_linf = (float)(p->drag_c1 * nu / (p->drag_d * p->drag_d));
    m.drag_qf = (float)(p->drag_c2 / p->drag_d);
  }
  m.les = p->les_cs > 0.0 ? 1 : 0;
  m.les_cs = p->les_cs;
  m.les_cf = (float)(18.0 * std::sqrt(2.0) * p->les_cs * p->les_cs);
  if (p->storage == LBM_FP16_SHIFTED) {
    m.scale = ldexpf(1.0f, p->fp16_scale_log2);
    m.inv_scale = ldexpf(1.0f, -p->fp16_scale_log2);
  } else {
    m.scale = m.inv_scale = 1.0f;
  }

  h->ls = lbm::make_launch(p->nx, p->ny, p->nz, p->block_x, p->block_y);
  h->nblocks = (int)(h->ls.grid.x * h->ls.grid.y * h->ls.grid.z);
  h->ls.row_consumers = p->row_consumers;
  h->ls.row_stages = p->row_stages;
  if (p->kernel != 1 && p->storage != LBM_FP64 && !p->drag_model && !(p->les_cs > 0.0)) {
    const int ok = lbm::plan_row_kernel(p->lattice, p->storage, p->nx, h->nxp, p->ny, p->nz, p->walls, h->ls);
    if (!ok && p->kernel == 2) {
      delete h;
      return fail(nullptr, LBM_EINVAL, "the row-staged kernel does not fit this lattice");
    }
    if (ok && p->kernel == 0 && p->nx < 32) h->ls.row = 0;  // short rows: one cell per thread
    if (h->ls.row) h->nblocks = h->ls.row_grid;
  }
  const int nblocks_alloc = h->nblocks > (int)kRowGridBound ? h->nblocks : (int)kRowGridBound;

  int rc;
  const size_t pop_bytes = (size_t)h->Q * m.plane * kElem[p->storage];
  if ((rc = dev_alloc(h, &h->pop, pop_bytes)) ||
      (rc = dev_alloc(h, &h->eps_buf[0], (size_t)h->Ni * h->field_elem)) ||
      (rc = dev_alloc(h, &h->eps_buf[1], (size_t)h->Ni * h->field_elem)) ||
      (rc = dev_alloc(h, (void **)&h->partials, (size_t)nblocks_alloc * lbm::kRedWidth * sizeof(double))) ||
      (rc = dev_alloc(h, (void **)&h->stats_dev, 64 * sizeof(double))) ||
      (rc = dev_alloc(h, (void **)&h->status, 64)) ||
      (rc = dev_alloc(h, (void **)&h->d, sizeof(LatticeDev))) ||
      (p->storage != LBM_FP64 && ((rc = dev_alloc(h, (void **)&h->sig_buf[0], (size_t)h->Ni * 2)) ||
                                  (rc = dev_alloc(h, (void **)&h->sig_buf[1], (size_t)h->Ni * 2))))) {
    g_last_error = h->err;
    lbm_vanse_destroy(h);
    return rc;
  }
  if (cudaMallocHost((void **)&h->stats_host, 64 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    g_last_error = "pinned host allocation failed";
    lbm_vanse_destroy(h);
    return LBM_ENOMEM;
  }
  // phi = 1 everywhere, rest state
  std::vector<double> ones_d;
  std::vector<float> ones_f;
  const void *src;
  if (h->field_elem == 8) {
    ones_d.assign(h->Ni, 1.0);
    src = ones_d.data();
  } else {
    ones_f.assign(h->Ni, 1.0f);
    src = ones_f.data();
  }
  // both phi buffers start as 1 everywhere, row padding included (padding
  // keeps a valid value that no kernel uses)
  cudaError_t e = cudaMemcpyAsync(h->eps_buf[0], src, (size_t)h->Ni * h->field_elem,
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->eps_buf[1], src, (size_t)h->Ni * h->field_elem, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->pop, 0, pop_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, 64, h->stream);
  if (e != cudaSuccess) {
    fail(h, LBM_ECUDA, "initial upload failed: %s", cudaGetErrorString(e));
    g_last_error = h->err;
    lbm_vanse_destroy(h);
    return LBM_ECUDA;
  }
  h->eps_cur = 0;
  m.sig_rd = m.sig_wr = h->sig_buf[0];
  if (p->storage != LBM_FP64 &&
      lbm::launch_shift(m, static_cast<const float *>(h->eps_buf[0]), h->sig_buf[0], h->stream) != cudaSuccess) {
    fail(h, LBM_ECUDA, "shift kernel launch failed");
    g_last_error = h->err;
    lbm_vanse_destroy(h);
    return LBM_ECUDA;
  }
  if ((rc = push_mirror(h)) ||
      (rc = lbm::launch_init(h->h, h->d, 0, nullptr, nullptr, 0, h->stream) == cudaSuccess
                ? LBM_OK
                : fail(h, LBM_ECUDA, "init kernel launch failed"))) {
    g_last_error = h->err;
    lbm_vanse_destroy(h);
    return rc;
  }
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    fail(h, LBM_ECUDA, "create: %s", cudaGetErrorString(e));
    g_last_error = h->err;
    lbm_vanse_destroy(h);
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

// Copy `ncomp` dense fields (nx*ny*nz values each, x fastest) of the
// caller's element type into a pitched device buffer of the handle's field
// type (component a at a*Ni, rows at pitch nxp).  Host sources are copied
// before the call returns.
// With sync = false a host source must stay valid until the caller
// synchronises the stream.
static int upload_field(lbm_vanse_t h, void *dst, const void *src, int ncomp, int src_is_f64,
                        int on_device, bool sync = true) {
  const bool dst_f64 = h->field_elem == 8;
  const int nx = h->p.nx, nxp = h->nxp;
  const long long rows = (long long)h->p.ny * h->p.nz * ncomp;
  const size_t fe = h->field_elem;
  if ((bool)src_is_f64 == dst_f64) {
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nx == nxp)  // unpadded rows: one contiguous copy
      CUDA_TRY(h, cudaMemcpyAsync(dst, src, (size_t)nx * fe * (size_t)rows, kind, h->stream));
    else
      CUDA_TRY(h, cudaMemcpy2DAsync(dst, (size_t)nxp * fe, src, (size_t)nx * fe, (size_t)nx * fe, (size_t)rows,
                                    kind, h->stream));
    // a pinned host source would be read after the return: wait for the copy
    if (!on_device && sync) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LBM_OK;
  }
  if (on_device) {
    CUDA_TRY(h, lbm::launch_pitch_convert(src, src_is_f64, dst, dst_f64, nx, nxp, rows, h->stream));
    return LBM_OK;
  }
  const long long n = (long long)nx * rows;
  if (dst_f64) {
    std::vector<double> tmp(n);
    const float *sp = static_cast<const float *>(src);
    for (long long i = 0; i < n; ++i) tmp[i] = (double)sp[i];
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, (size_t)nxp * 8, tmp.data(), (size_t)nx * 8, (size_t)nx * 8, (size_t)rows,
                                  cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  } else {
    std::vector<float> tmp(n);
    const double *sp = static_cast<const double *>(src);
    for (long long i = 0; i < n; ++i) tmp[i] = (float)sp[i];
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, (size_t)nxp * 4, tmp.data(), (size_t)nx * 4, (size_t)nx * 4, (size_t)rows,
                                  cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

template <class T>
static int check_host_values(lbm_vanse_t h, const T *v, long long n, bool unit_interval, const char *what) {
  for (long long i = 0; i < n; ++i) {
    const double x = (double)v[i];
    if (!std::isfinite(x)) return fail(h, LBM_EINVAL, "%s[%lld] is not finite", what, i);
    if (unit_interval && !(x > 0.0 && x <= 1.0))
      return fail(h, LBM_EINVAL, "%s[%lld] = %g is outside (0, 1]", what, i, x);
  }
  return LBM_OK;
}

// Check uploaded copies of host values on the device (one scan kernel per
// field, one readback of the first bad indices); synchronises the stream.
// Field b may be absent (dev_b null).
static int check_uploaded2(lbm_vanse_t h, const void *dev_a, bool unit_a, const char *what_a, const void *dev_b,
                           bool unit_b, const char *what_b, long long n, int is_f64) {
  long long *flag = reinterpret_cast<long long *>(h->stats_dev + 48);
  long long *host = reinterpret_cast<long long *>(h->stats_host + 48);
  // 0x7f.. bytes: a value above every index ("none"); the scan keeps the minimum
  CUDA_TRY(h, cudaMemsetAsync(flag, 0x7f, 2 * sizeof(long long), h->stream));
  CUDA_TRY(h, lbm::launch_validate(dev_a, n, is_f64, unit_a ? 1 : 0, flag, h->stream));
  if (dev_b) CUDA_TRY(h, lbm::launch_validate(dev_b, n, is_f64, unit_b ? 1 : 0, flag + 1, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(host, flag, 2 * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  for (int f = 0; f < (dev_b ? 2 : 1); ++f)
    if (host[f] < n) {
      // report the caller's dense index of the stored cell
      const long long i = host[f], row = i / h->nxp, x = i % h->nxp;
      const bool unit = f == 0 ? unit_a : unit_b;
      return fail(h, LBM_EINVAL, "%s[%lld] is %s", f == 0 ? what_a : what_b, row * h->p.nx + x,
                  unit ? "not finite or outside (0, 1]" : "not finite");
    }
  return LBM_OK;
}

// d_t phi buffer b, allocated on first use and zeroed (the row padding must
// pass the finite-value check of later uploads).
static int ensure_deps_buf(lbm_vanse_t h, int b) {
  if (h->deps_buf[b]) return LBM_OK;
  int rc;
  if ((rc = dev_alloc(h, &h->deps_buf[b], (size_t)h->Ni * h->field_elem))) return rc;
  CUDA_TRY(h, cudaMemsetAsync(h->deps_buf[b], 0, (size_t)h->Ni * h->field_elem, h->stream));
  return LBM_OK;
}

// Make the spare phi_ref / d_t phi buffers (already filled and checked) the
// current ones: the shift sigma of the new phi_ref is computed into the
// spare shift buffer, and the next step decodes with the old one.
// quad_auto: the quadrature rule from the directions in which phi_ref (and
// d_t phi) vary (Sec. 2.2, eq. (quad) and Table "weights"), every lattice
// axis when phi is uniform.  Scans buffer `b` on the device; synchronises.
static int choose_quadrature(lbm_vanse_t h, int b, int has_deps) {
  unsigned *mask = reinterpret_cast<unsigned *>(h->stats_dev + 40);
  CUDA_TRY(h, cudaMemsetAsync(mask, 0, sizeof(unsigned), h->stream));
  const int f64 = h->field_elem == 8;
  CUDA_TRY(h, lbm::launch_variation(h->eps_buf[b], f64, h->p.nx, h->nxp, h->p.ny, h->p.nz, h->D, mask, h->stream));
  if (has_deps)
    CUDA_TRY(h, lbm::launch_variation(h->deps_buf[b], f64, h->p.nx, h->nxp, h->p.ny, h->p.nz, h->D, mask,
                                      h->stream));
  unsigned *host = reinterpret_cast<unsigned *>(h->stats_host + 40);
  CUDA_TRY(h, cudaMemcpyAsync(host, mask, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  const unsigned all = (1u << h->D) - 1u;
  const unsigned qa = (*host & all) ? (*host & all) : all;
  const int qd = __builtin_popcount(qa);
  h->p.quad_axes = qa;
  h->p.quad_dim = qd;
  h->h.quad_axes = qa;
  h->h.qw0 = lbm::quad_w0(qd);
  h->h.qw1 = lbm::quad_w1(qd);
  return LBM_OK;
}

static int adopt_epsilon(lbm_vanse_t h, int next, int has_deps, long long n_ref) {
  if (h->p.quad_auto) {
    const int rc = choose_quadrature(h, next, has_deps);
    if (rc) return rc;
  }
  h->h.has_deps = has_deps;
  h->eps_cur = next;
  h->h.n_eps = n_ref;
  if (h->p.storage != LBM_FP64) {
    // the data stays encoded with the old shift until the next step
    CUDA_TRY(h, lbm::launch_shift(h->h, static_cast<const float *>(h->eps_buf[next]), h->sig_buf[next],
                                  h->stream));
    h->h.sig_wr = h->sig_buf[next];
  }
  return push_mirror(h);
}

static int set_epsilon_any(lbm_vanse_t h, const void *eps, const void *deps, long long n_ref,
                           int on_device, int is_f64) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!eps) return fail(h, LBM_EINVAL, "eps_ref is NULL");
  if (h->staged) return fail(h, LBM_ESTATE, "a staged phi refresh awaits lbm_vanse_commit_epsilon");
  int rc;
  const int next = 1 - h->eps_cur;
  const int dev_f64 = h->field_elem == 8;
  // both fields go to the spare buffers and are checked together with one
  // synchronisation; nothing the lattice uses changes before both passed
  if ((rc = upload_field(h, h->eps_buf[next], eps, 1, is_f64, on_device, false))) return rc;
  if (deps) {
    if ((rc = ensure_deps_buf(h, next))) return rc;
    if ((rc = upload_field(h, h->deps_buf[next], deps, 1, is_f64, on_device, false))) return rc;
  }
  if (!on_device) {
    if ((rc = check_uploaded2(h, h->eps_buf[next], true, "eps_ref", deps ? h->deps_buf[next] : nullptr, false,
                              "deps_dt", h->Ni, dev_f64)))
      return rc;
  }
  return adopt_epsilon(h, next, deps ? 1 : 0, n_ref);
}

extern "C" int lbm_vanse_set_epsilon(lbm_vanse_t h, const float *eps_ref, const float *deps_dt,
                                     long long n_ref, int on_device) {
  return set_epsilon_any(h, eps_ref, deps_dt, n_ref, on_device, 0);
}

extern "C" int lbm_vanse_set_epsilon_f64(lbm_vanse_t h, const double *eps_ref, const double *deps_dt,
                                         long long n_ref, int on_device) {
  return set_epsilon_any(h, eps_ref, deps_dt, n_ref, on_device, 1);
}

// One dense FP32 field into the pitched buffer dst on stream cs, not waited for.
static int copy_field_async(lbm_vanse_t h, void *dst, const float *src, int on_device, cudaStream_t cs) {
  const int nx = h->p.nx, nxp = h->nxp;
  const size_t rows = (size_t)h->p.ny * h->p.nz;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (nx == nxp)
    CUDA_TRY(h, cudaMemcpyAsync(dst, src, (size_t)nx * 4 * rows, kind, cs));
  else
    CUDA_TRY(h, cudaMemcpy2DAsync(dst, (size_t)nxp * 4, src, (size_t)nx * 4, (size_t)nx * 4, rows, kind, cs));
  return LBM_OK;
}

static int stage_epsilon_impl(lbm_vanse_t h, const float *eps, const float *deps, long long n_ref,
                              int on_device) {
  int rc;
  if (!h->copy_stream) {
    CUDA_TRY(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
    CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_order, cudaEventDisableTiming));
    CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_staged, cudaEventDisableTiming));
  }
  const int next = 1 - h->eps_cur;
  if (deps && (rc = ensure_deps_buf(h, next))) return rc;
  // the spare buffers were last read by work already on the handle's stream
  // (the steps before the previous refresh): the copies start after it
  CUDA_TRY(h, cudaEventRecord(h->ev_order, h->stream));
  CUDA_TRY(h, cudaStreamWaitEvent(h->copy_stream, h->ev_order, 0));
  if ((rc = copy_field_async(h, h->eps_buf[next], eps, on_device, h->copy_stream))) return rc;
  if (deps && (rc = copy_field_async(h, h->deps_buf[next], deps, on_device, h->copy_stream))) return rc;
  if (!on_device) {
    // the same scan as set_epsilon's, on the copy stream, into its own slots
    long long *flag = reinterpret_cast<long long *>(h->stats_dev + 56);
    CUDA_TRY(h, cudaMemsetAsync(flag, 0x7f, 2 * sizeof(long long), h->copy_stream));
    CUDA_TRY(h, lbm::launch_validate(h->eps_buf[next], h->Ni, 0, 1, flag, h->copy_stream));
    if (deps) CUDA_TRY(h, lbm::launch_validate(h->deps_buf[next], h->Ni, 0, 0, flag + 1, h->copy_stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->stats_host + 56, flag, 2 * sizeof(long long), cudaMemcpyDeviceToHost,
                                h->copy_stream));
  }
  CUDA_TRY(h, cudaEventRecord(h->ev_staged, h->copy_stream));
  h->staged = 1;
  h->staged_deps = deps ? 1 : 0;
  h->staged_checked = on_device ? 0 : 1;
  h->staged_n_ref = n_ref;
  return LBM_OK;
}

extern "C" int lbm_vanse_stage_epsilon(lbm_vanse_t h, const float *eps_ref, const float *deps_dt,
                                       long long n_ref, int on_device) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!eps_ref) return fail(h, LBM_EINVAL, "eps_ref is NULL");
  if (h->field_elem != 4)
    return fail(h, LBM_EINVAL, "staged phi refreshes need FP32 fields (FP32 or FP16 storage)");
  if (h->staged) return fail(h, LBM_ESTATE, "a staged phi refresh already awaits lbm_vanse_commit_epsilon");
  const int rc = stage_epsilon_impl(h, eps_ref, deps_dt, n_ref, on_device);
  if (rc != LBM_OK && h->copy_stream) {
    // nothing may still write the spare buffers after a failed call
    cudaStreamSynchronize(h->copy_stream);
    h->staged = 0;
  }
  return rc;
}

extern "C" int lbm_vanse_commit_epsilon(lbm_vanse_t h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!h->staged) return fail(h, LBM_ESTATE, "no staged phi refresh to commit");
  h->staged = 0;
  CUDA_TRY(h, cudaEventSynchronize(h->ev_staged));
  if (h->staged_checked) {
    const long long *host = reinterpret_cast<const long long *>(h->stats_host + 56);
    for (int f = 0; f < (h->staged_deps ? 2 : 1); ++f)
      if (host[f] < h->Ni) {
        // the caller's dense index of the stored cell
        const long long i = host[f], row = i / h->nxp, x = i % h->nxp;
        return fail(h, LBM_EINVAL, "%s[%lld] is %s", f == 0 ? "eps_ref" : "deps_dt", row * h->p.nx + x,
                    f == 0 ? "not finite or outside (0, 1]" : "not finite");
      }
  }
  // the handle's stream reads the new fields only after the copies
  CUDA_TRY(h, cudaStreamWaitEvent(h->stream, h->ev_staged, 0));
  return adopt_epsilon(h, 1 - h->eps_cur, h->staged_deps, h->staged_n_ref);
}

static int set_force_any(lbm_vanse_t h, const double *g, const void *field, const void *dfield,
                         long long n_ref, int on_device, int is_f64) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (dfield && !field) return fail(h, LBM_EINVAL, "dfield_dt given without field");
  int rc;
  double gv[3] = {0.0, 0.0, 0.0};
  if (g)
    for (int a = 0; a < 3; ++a) {
      if (!std::isfinite(g[a])) return fail(h, LBM_EINVAL, "g[%d] is not finite", a);
      gv[a] = a < h->D ? g[a] : 0.0;
    }
  const long long n3 = 3 * h->N;
  if (field && !on_device) {
    if (is_f64) {
      if ((rc = check_host_values(h, static_cast<const double *>(field), n3, false, "field"))) return rc;
      if (dfield && (rc = check_host_values(h, static_cast<const double *>(dfield), n3, false, "dfield_dt"))) return rc;
    } else {
      if ((rc = check_host_values(h, static_cast<const float *>(field), n3, false, "field"))) return rc;
      if (dfield && (rc = check_host_values(h, static_cast<const float *>(dfield), n3, false, "dfield_dt"))) return rc;
    }
  }
  if (field) {
    const size_t fbytes = (size_t)3 * h->Ni * h->field_elem;
    if (!h->force) {
      if ((rc = dev_alloc(h, &h->force, fbytes))) return rc;
      CUDA_TRY(h, cudaMemsetAsync(h->force, 0, fbytes, h->stream));
    }
    if ((rc = upload_field(h, h->force, field, 3, is_f64, on_device))) return rc;
    if (dfield) {
      if (!h->dforce) {
        if ((rc = dev_alloc(h, &h->dforce, fbytes))) return rc;
        CUDA_TRY(h, cudaMemsetAsync(h->dforce, 0, fbytes, h->stream));
      }
      if ((rc = upload_field(h, h->dforce, dfield, 3, is_f64, on_device))) return rc;
    }
  }
  for (int a = 0; a < 3; ++a) h->h.g[a] = gv[a];
  h->h.has_force = field ? 1 : 0;
  h->h.has_dforce = dfield ? 1 : 0;
  h->h.n_force = n_ref;
  return push_mirror(h);
}

extern "C" int lbm_vanse_set_force(lbm_vanse_t h, const double *g, const float *field,
                                   const float *dfield_dt, long long n_ref, int on_device) {
  return set_force_any(h, g, field, dfield_dt, n_ref, on_device, 0);
}

extern "C" int lbm_vanse_set_force_f64(lbm_vanse_t h, const double *g, const double *field,
                                       const double *dfield_dt, long long n_ref, int on_device) {
  return set_force_any(h, g, field, dfield_dt, n_ref, on_device, 1);
}

// Upload an optional field as device doubles (temporary buffer).
static int stage_doubles(lbm_vanse_t h, const void *src, long long n, int is_f64, int on_device,
                         double **out) {
  *out = nullptr;
  if (!src) return LBM_OK;
  int rc;
  if ((rc = dev_alloc(h, (void **)out, (size_t)n * sizeof(double)))) return rc;
  if (on_device) {
    if (is_f64) {
      CUDA_TRY(h, cudaMemcpyAsync(*out, src, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CUDA_TRY(h, lbm::launch_convert_f2d(static_cast<const float *>(src), *out, n, h->stream));
    }
  } else {
    std::vector<double> tmp;
    const void *s = src;
    if (!is_f64) {
      tmp.resize(n);
      for (long long i = 0; i < n; ++i) tmp[i] = (double)static_cast<const float *>(src)[i];
      s = tmp.data();
    }
    CUDA_TRY(h, cudaMemcpyAsync(*out, s, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

static int init_any(lbm_vanse_t h, const void *p0, const void *u0, int mode, int on_device, int is_f64) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (mode & ~3) return fail(h, LBM_EINVAL, "mode has unknown bits");
  int rc;
  if (!on_device) {
    if (is_f64) {
      if (p0 && (rc = check_host_values(h, static_cast<const double *>(p0), h->N, false, "p0"))) return rc;
      if (u0 && (rc = check_host_values(h, static_cast<const double *>(u0), 3 * h->N, false, "u0"))) return rc;
    } else {
      if (p0 && (rc = check_host_values(h, static_cast<const float *>(p0), h->N, false, "p0"))) return rc;
      if (u0 && (rc = check_host_values(h, static_cast<const float *>(u0), 3 * h->N, false, "u0"))) return rc;
    }
  }
  double *dp = nullptr, *du = nullptr;
  if ((rc = stage_doubles(h, p0, h->N, is_f64, on_device, &dp)) ||
      (rc = stage_doubles(h, u0, 3 * h->N, is_f64, on_device, &du))) {
    if (dp) cudaFreeAsync(dp, h->stream);
    return rc;
  }
  // the initial state is written with the newest shift
  h->h.sig_rd = h->h.sig_wr;
  h->h.have_prev = 0;
  h->last_check_n = -1;
  if ((rc = push_mirror(h))) return rc;
  cudaError_t e = lbm::launch_init(h->h, h->d, h->h.n, dp, du, mode, h->stream);
  lbm::count_launches(1);
  if (dp) cudaFreeAsync(dp, h->stream);
  if (du) cudaFreeAsync(du, h->stream);
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "init kernel: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" int lbm_vanse_init_equilibrium(lbm_vanse_t h, const float *p0, const float *u0, int mode,
                                          int on_device) {
  return init_any(h, p0, u0, mode, on_device, 0);
}

extern "C" int lbm_vanse_init_equilibrium_f64(lbm_vanse_t h, const double *p0, const double *u0,
                                              int mode, int on_device) {
  return init_any(h, p0, u0, mode, on_device, 1);
}

// ---------------------------------------------------------------- stepping

// Launch `k` plain steps (no check) starting at the mirror's time, then
// advance the device time counter.  k == 0 is a no-op.
static int run_plain_steps(lbm_vanse_t h, int k) {
  for (int j = 0; j < k; ++j)
    CUDA_TRY(h, lbm::launch_step(h->h, h->d, h->h.n, j, 0, h->ls, h->stream));
  if (k > 0) CUDA_TRY(h, lbm::launch_advance(h->d, k, h->stream));
  if (k > 0) lbm::count_launches(k + 1);
  h->h.n += k;
  h->h.sig_rd = h->h.sig_wr;
  return LBM_OK;
}

static int get_graph(lbm_vanse_t h, int parity, int steps, cudaGraphExec_t *out) {
  // the launches depend on whether phi has a time derivative (stage layout)
  auto key = std::make_tuple(parity, steps, h->h.has_deps);
  auto it = h->graphs.find(key);
  if (it != h->graphs.end()) {
    *out = it->second;
    return LBM_OK;
  }
  // capture on a private stream so that the caller's stream is never put in
  // capture mode
  cudaStream_t cs;
  CUDA_TRY(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int j = 0; j < steps && e == cudaSuccess; ++j)
      e = lbm::launch_step(h->h, h->d, parity, j, 0, h->ls, cs);
    if (e == cudaSuccess) e = lbm::launch_advance(h->d, steps, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) {
    cudaGraphExec_t ge;
    e = cudaGraphInstantiate(&ge, g, 0);
    cudaGraphDestroy(g);
    if (e == cudaSuccess) {
      h->graphs[key] = ge;
      *out = ge;
    }
  }
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

// Advance k steps without a check: graph chunks where possible.
static int run_steps(lbm_vanse_t h, long long k) {
  int rc;
  if (k <= 0) return LBM_OK;
  // a pending shift change or an odd start is handled by single steps
  if (h->h.sig_rd != h->h.sig_wr || (h->h.n & 1)) {
    if ((rc = push_mirror(h))) return rc;
    if ((rc = run_plain_steps(h, 1))) return rc;
    --k;
  }
  while (k >= kGraphChunk) {
    cudaGraphExec_t ge;
    if ((rc = get_graph(h, 0, kGraphChunk, &ge))) return rc;
    CUDA_TRY(h, cudaGraphLaunch(ge, h->stream));
    lbm::count_launches(kGraphChunk + 1);
    h->h.n += kGraphChunk;
    k -= kGraphChunk;
  }
  if (k > 0 && (rc = run_plain_steps(h, (int)k))) return rc;
  return LBM_OK;
}

// One check step: fused reductions, finalize, copy the sums to pinned host
// memory (the caller synchronises).
static int run_check_step(lbm_vanse_t h) {
  int rc;
  if ((rc = push_mirror(h))) return rc;
  CUDA_TRY(h, lbm::launch_step(h->h, h->d, h->h.n, 0, 1, h->ls, h->stream));
  CUDA_TRY(h, lbm::launch_advance(h->d, 1, h->stream));
  CUDA_TRY(h, lbm::launch_finalize(h->partials, h->nblocks, h->stats_dev, h->stream));
  lbm::count_launches(3);
  CUDA_TRY(h, cudaMemcpyAsync(h->stats_host, h->stats_dev, lbm::kRedWidth * sizeof(double),
                              cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->stats_host + 32, h->status, sizeof(int), cudaMemcpyDeviceToHost,
                              h->stream));
  h->h.sig_rd = h->h.sig_wr;
  h->h.n += 1;
  return LBM_OK;
}

extern "C" int lbm_vanse_step(lbm_vanse_t h, long long max_steps, double residual_tol, int check_every,
                              lbm_vanse_stats *out) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (max_steps < 0) return fail(h, LBM_EINVAL, "max_steps must be >= 0");
  if (check_every < -1) return fail(h, LBM_EINVAL, "check_every must be >= -1");
  if (!(residual_tol >= 0.0)) return fail(h, LBM_EINVAL, "residual_tol must be >= 0");
  if (check_every == -1 && residual_tol > 0.0)
    return fail(h, LBM_EINVAL, "residual_tol needs check steps (check_every >= 0)");
  int rc;
  lbm_vanse_stats st;
  memset(&st, 0, sizeof(st));
  st.residual = -1.0;
  if (check_every == -1) {
    // plain steps only: no reductions and no synchronisation
    if ((rc = run_steps(h, max_steps))) return rc;
    st.steps_done = h->h.n;
    st.step_of_stats = -1;
    if (out) *out = st;
    return LBM_OK;
  }
  if (max_steps == 0) {
    st.steps_done = h->h.n;
    st.step_of_stats = -1;
    if (out) *out = st;
    return LBM_OK;
  }
  if (residual_tol > 0.0 && !h->u_prev) {
    if ((rc = dev_alloc(h, (void **)&h->u_prev, (size_t)3 * h->Ni * sizeof(float)))) return rc;
    h->h.have_prev = 0;
    h->last_check_n = -1;
  }
  const long long interval = check_every > 0 ? check_every : max_steps;
  long long remaining = max_steps;
  while (remaining > 0) {
    const long long k = remaining < interval ? remaining : interval;
    if ((rc = run_steps(h, k - 1))) return rc;
    const long long n_stats = h->h.n;
    if ((rc = run_check_step(h))) return rc;
    remaining -= k;
    const bool last = remaining == 0;
    if (!(residual_tol > 0.0) && !last) continue;
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    const double *s = h->stats_host;
    if (*reinterpret_cast<const int *>(h->stats_host + 32) != 0) {
      cudaMemsetAsync(h->status, 0, sizeof(int), h->stream);
      *reinterpret_cast<int *>(h->stats_host + 32) = 0;
      return fail(h, LBM_ETIMEOUT, "a bounded wait in the step kernel gave up before step %lld",
                  (long long)h->h.n);
    }
    st.mass = s[0];
    st.momentum[0] = s[1];
    st.momentum[1] = s[2];
    st.momentum[2] = s[3];
    st.u_norm = std::sqrt(s[5]);
    st.force[0] = s[7];
    st.force[1] = s[8];
    st.force[2] = s[9];
    st.step_of_stats = n_stats;
    st.nan_seen = s[6] > 0.0 || !std::isfinite(s[0]) || !std::isfinite(s[5]);
    if (h->u_prev && h->h.have_prev && h->last_check_n >= 0) {
      const double K = (double)(n_stats - h->last_check_n);
      st.residual = s[5] > 0.0 ? std::sqrt(s[4]) / (K * std::sqrt(s[5])) : 0.0;
    } else {
      st.residual = -1.0;
    }
    if (h->u_prev) {
      h->h.have_prev = 1;
      h->last_check_n = n_stats;
    }
    st.steps_done = h->h.n;
    if (st.nan_seen) {
      if (out) *out = st;
      return fail(h, LBM_EUNSTABLE, "NaN or Inf in the moments at step %lld", n_stats);
    }
    if (residual_tol > 0.0 && st.residual >= 0.0 && st.residual <= residual_tol) {
      st.converged = 1;
      break;
    }
  }
  st.steps_done = h->h.n;
  if (out) *out = st;
  return LBM_OK;
}

// ---------------------------------------------------------------- outputs

static int moments_any(lbm_vanse_t h, void *rho, void *p, void *u, int on_device, int is_f64) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  int rc;
  lbm::count_launches(1);
  if ((rc = push_mirror(h))) return rc;
  const long long N = h->N;
  if (on_device) {
    cudaError_t e;
    if (is_f64)
      e = lbm::launch_moments(h->h, h->d, h->h.n, (double *)rho, (double *)p, (double *)u, nullptr,
                              nullptr, nullptr, h->stream);
    else
      e = lbm::launch_moments(h->h, h->d, h->h.n, nullptr, nullptr, nullptr, (float *)rho, (float *)p,
                              (float *)u, h->stream);
    if (e != cudaSuccess) return fail(h, LBM_ECUDA, "moments kernel: %s", cudaGetErrorString(e));
    return LBM_OK;
  }
  const size_t es = is_f64 ? 8 : 4;
  void *buf = nullptr;
  if ((rc = dev_alloc(h, &buf, (size_t)5 * N * es))) return rc;
  char *b = static_cast<char *>(buf);
  void *drho = b, *dp = b + N * es, *du = b + 2 * N * es;
  cudaError_t e;
  if (is_f64)
    e = lbm::launch_moments(h->h, h->d, h->h.n, (double *)drho, (double *)dp, (double *)du, nullptr,
                            nullptr, nullptr, h->stream);
  else
    e = lbm::launch_moments(h->h, h->d, h->h.n, nullptr, nullptr, nullptr, (float *)drho, (float *)dp,
                            (float *)du, h->stream);
  if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, drho, N * es, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, dp, N * es, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, 3 * N * es, cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(buf, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "moments: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" int lbm_vanse_moments(lbm_vanse_t h, float *rho, float *p, float *u, int on_device) {
  return moments_any(h, rho, p, u, on_device, 0);
}

extern "C" int lbm_vanse_moments_f64(lbm_vanse_t h, double *rho, double *p, double *u, int on_device) {
  return moments_any(h, rho, p, u, on_device, 1);
}

extern "C" int lbm_vanse_get_populations(lbm_vanse_t h, double *f_host) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!f_host) return fail(h, LBM_EINVAL, "f_host is NULL");
  int rc;
  if ((rc = push_mirror(h))) return rc;
  const size_t bytes = (size_t)h->N * h->Q * sizeof(double);
  void *buf;
  if ((rc = dev_alloc(h, &buf, bytes))) return rc;
  cudaError_t e = lbm::launch_get_populations(h->h, h->d, h->h.n, static_cast<double *>(buf), h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, buf, bytes, cudaMemcpyDeviceToHost, h->stream);
  cudaFreeAsync(buf, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "get_populations: %s", cudaGetErrorString(e));
  return LBM_OK;
}

extern "C" long long lbm_vanse_steps_done(lbm_vanse_t h) { return h ? h->h.n : -1; }

extern "C" int lbm_vanse_get_params(lbm_vanse_t h, lbm_vanse_params *out) {
  if (!h || !out) return fail(h, LBM_EINVAL, "NULL argument");
  *out = h->p;
  return LBM_OK;
}

// ---------------------------------------------------------------- checkpoint

namespace {
struct StateHeader {
  char magic[8];
  int lattice, storage, nx, ny, nz;
  long long n, n_eps, n_force;
  int has_deps, has_force, has_dforce, reshift_pending;
  double g[3];
  unsigned long long pop_bytes, field_bytes;
};
}  // namespace

extern "C" int lbm_vanse_save_state(lbm_vanse_t h, void *buf, size_t *size) {
  if (!h || !size) return fail(h, LBM_EINVAL, "NULL argument");
  const size_t pop_bytes = (size_t)h->Q * h->h.plane * kElem[h->p.storage];
  const size_t fb = (size_t)h->Ni * h->field_elem;
  const size_t sb = h->p.storage == LBM_FP64 ? 0 : (size_t)h->Ni * 2;
  const size_t total = sizeof(StateHeader) + pop_bytes + sb + 2 * fb + 6 * fb;
  if (!buf) {
    *size = total;
    return LBM_OK;
  }
  if (*size < total) return fail(h, LBM_EINVAL, "buffer too small (%zu < %zu)", *size, total);
  StateHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, "LBMVANSE", 8);
  hd.lattice = h->p.lattice;
  hd.storage = h->p.storage;
  hd.nx = h->p.nx;
  hd.ny = h->p.ny;
  hd.nz = h->p.nz;
  hd.n = h->h.n;
  hd.n_eps = h->h.n_eps;
  hd.n_force = h->h.n_force;
  hd.has_deps = h->h.has_deps;
  hd.has_force = h->h.has_force;
  hd.has_dforce = h->h.has_dforce;
  hd.reshift_pending = h->h.sig_rd != h->h.sig_wr;
  for (int a = 0; a < 3; ++a) hd.g[a] = h->h.g[a];
  hd.pop_bytes = pop_bytes;
  hd.field_bytes = fb;
  char *o = static_cast<char *>(buf);
  memcpy(o, &hd, sizeof(hd));
  o += sizeof(hd);
  CUDA_TRY(h, cudaMemcpyAsync(o, h->pop, pop_bytes, cudaMemcpyDeviceToHost, h->stream));
  o += pop_bytes;
  // phi (current), the shift the data is encoded with, d_t phi
  CUDA_TRY(h, cudaMemcpyAsync(o, h->eps_buf[h->eps_cur], fb, cudaMemcpyDeviceToHost, h->stream));
  o += fb;
  if (sb) CUDA_TRY(h, cudaMemcpyAsync(o, h->h.sig_rd, sb, cudaMemcpyDeviceToHost, h->stream));
  o += sb;
  if (h->h.has_deps)
    CUDA_TRY(h, cudaMemcpyAsync(o, h->deps_buf[h->eps_cur], fb, cudaMemcpyDeviceToHost, h->stream));
  o += fb;
  if (h->h.has_force) CUDA_TRY(h, cudaMemcpyAsync(o, h->force, 3 * fb, cudaMemcpyDeviceToHost, h->stream));
  o += 3 * fb;
  if (h->h.has_dforce) CUDA_TRY(h, cudaMemcpyAsync(o, h->dforce, 3 * fb, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  *size = total;
  return LBM_OK;
}

extern "C" int lbm_vanse_load_state(lbm_vanse_t h, const void *buf, size_t size) {
  if (!h || !buf) return fail(h, LBM_EINVAL, "NULL argument");
  if (size < sizeof(StateHeader)) return fail(h, LBM_EINVAL, "buffer too small");
  if (h->staged) return fail(h, LBM_ESTATE, "a staged phi refresh awaits lbm_vanse_commit_epsilon");
  StateHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  const size_t pop_bytes = (size_t)h->Q * h->h.plane * kElem[h->p.storage];
  const size_t fb = (size_t)h->Ni * h->field_elem;
  if (memcmp(hd.magic, "LBMVANSE", 8) != 0 || hd.lattice != h->p.lattice || hd.storage != h->p.storage ||
      hd.nx != h->p.nx || hd.ny != h->p.ny || hd.nz != h->p.nz || hd.pop_bytes != pop_bytes ||
      hd.field_bytes != fb || size < sizeof(StateHeader) + pop_bytes + (h->p.storage == LBM_FP64 ? 0 : (size_t)h->Ni * 2) + 8 * fb)
    return fail(h, LBM_EINVAL, "state does not match this lattice");
  int rc;
  const char *o = static_cast<const char *>(buf) + sizeof(hd);
  CUDA_TRY(h, cudaMemcpyAsync(h->pop, o, pop_bytes, cudaMemcpyHostToDevice, h->stream));
  o += pop_bytes;
  // the current phi (and its shift) go to buffer 0; the shift the data is
  // encoded with goes to shift buffer 1 when a shift change is pending
  const int cur = 0, other = 1;
  const size_t sb = h->p.storage == LBM_FP64 ? 0 : (size_t)h->Ni * 2;
  CUDA_TRY(h, cudaMemcpyAsync(h->eps_buf[cur], o, fb, cudaMemcpyHostToDevice, h->stream));
  o += fb;
  if (sb) CUDA_TRY(h, cudaMemcpyAsync(h->sig_buf[other], o, sb, cudaMemcpyHostToDevice, h->stream));
  o += sb;
  h->eps_cur = cur;
  if (hd.has_deps) {
    if ((rc = ensure_deps_buf(h, cur))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->deps_buf[cur], o, fb, cudaMemcpyHostToDevice, h->stream));
  }
  o += fb;
  if (hd.has_force) {
    if (!h->force && (rc = dev_alloc(h, &h->force, 3 * fb))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->force, o, 3 * fb, cudaMemcpyHostToDevice, h->stream));
  }
  o += 3 * fb;
  if (hd.has_dforce) {
    if (!h->dforce && (rc = dev_alloc(h, &h->dforce, 3 * fb))) return rc;
    CUDA_TRY(h, cudaMemcpyAsync(h->dforce, o, 3 * fb, cudaMemcpyHostToDevice, h->stream));
  }
  h->h.n = hd.n;
  h->h.n_eps = hd.n_eps;
  h->h.n_force = hd.n_force;
  h->h.has_deps = hd.has_deps;
  h->h.has_force = hd.has_force;
  h->h.has_dforce = hd.has_dforce;
  for (int a = 0; a < 3; ++a) h->h.g[a] = hd.g[a];
  if (h->p.storage != LBM_FP64) {
    CUDA_TRY(h, lbm::launch_shift(h->h, static_cast<const float *>(h->eps_buf[cur]), h->sig_buf[cur],
                                  h->stream));
    h->h.sig_wr = h->sig_buf[cur];
    h->h.sig_rd = hd.reshift_pending ? h->sig_buf[other] : h->h.sig_wr;
  }
  h->h.have_prev = 0;
  h->last_check_n = -1;
  if ((rc = push_mirror(h))) return rc;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

// Accessors for the batch module (same library).
namespace lbm {
LatticeDev *handle_device_desc(lbm_vanse_t h) { return h->d; }
const LatticeDev &handle_mirror(lbm_vanse_t h) { return h->h; }
LatticeDev &handle_mirror_mut(lbm_vanse_t h) { return h->h; }
int handle_push(lbm_vanse_t h) { return push_mirror(h); }
// Upload the descriptor only if it differs from *last (what the device was
// last given); *pushed tells whether it did.
int handle_push_changed(lbm_vanse_t h, LatticeDev *last, int *pushed) {
  sync_mirror_ptrs(h);
  *pushed = 0;
  if (memcmp(&h->h, last, sizeof(LatticeDev)) == 0) return LBM_OK;
  int rc;
  if ((rc = push_mirror(h))) return rc;
  *last = h->h;
  *pushed = 1;
  return LBM_OK;
}
cudaStream_t handle_stream(lbm_vanse_t h) { return h->stream; }
void set_global_error(const char *msg) { g_last_error = msg; }
}  // namespace lbm

extern "C" int lbm_vanse_set_wait_limit(lbm_vanse_t h, unsigned spins, int withhold_copies) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  h->h.wait_limit = spins ? spins : (1u << 22);
  h->h.withhold_copies = withhold_copies ? 1 : 0;
  return push_mirror(h);
}

extern "C" int lbm_vanse_uses_row_kernel(lbm_vanse_t h) { return h ? (h->ls.row ? 1 : 0) : -1; }

extern "C" int lbm_vanse_launch_shape(lbm_vanse_t h, int *shape) {
  if (!h || !shape) return fail(h, LBM_EINVAL, "NULL argument");
  shape[0] = h->ls.row ? 2 : (h->p.storage == LBM_FP64 ? 0 : 1);
  shape[1] = h->ls.row ? h->ls.row_consumers : (int)h->ls.block.x;
  shape[2] = h->ls.row ? h->ls.row_stages : (int)h->ls.block.y;
  shape[3] = h->ls.row ? h->ls.row_grid : (int)(h->ls.grid.x * h->ls.grid.y * h->ls.grid.z);
  return LBM_OK;
}

// ---------------------------------------------------------------- read-back without allocation

namespace {

// The staging array of lbm_vanse_moments_noalloc: reserved with the module on
// every device, shared by all calls on that device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[LBM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the staging array on `dev`, looked up once per device
// with that device current.
int noalloc_scratch(lbm_vanse_t h, int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    int prev = -1;
    CUDA_TRY(h, cudaGetDevice(&prev));
    if (prev != dev) CUDA_TRY(h, cudaSetDevice(dev));
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess || !ptr)
      return fail(h, LBM_ECUDA, "address of the staging array on device %d: %s", dev,
                  cudaGetErrorString(e));
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_vanse_moments_noalloc(lbm_vanse_t h, float *rho, float *p, float *u) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (h->N > LBM_NOALLOC_MAX_CELLS)
    return fail(h, LBM_EINVAL,
                "lattice has %lld cells; lbm_vanse_moments_noalloc takes at most %lld (a staging "
                "array of %zu bytes, 20 bytes per cell)",
                h->N, (long long)LBM_NOALLOC_MAX_CELLS, (size_t)LBM_NOALLOC_SCRATCH_BYTES);
  if (!rho && !p && !u) return LBM_OK;
  // the device that holds the lattice
  cudaPointerAttributes attr;
  CUDA_TRY(h, cudaPointerGetAttributes(&attr, h->pop));
  const int dev = attr.device;
  if (dev < 0 || dev >= kMaxDevices) return fail(h, LBM_ECUDA, "lattice memory on device %d", dev);
  int rc;
  void *scratch = nullptr;
  if ((rc = noalloc_scratch(h, dev, &scratch))) return rc;
  int prev = -1;
  CUDA_TRY(h, cudaGetDevice(&prev));
  if (prev != dev) CUDA_TRY(h, cudaSetDevice(dev));
  // rho at 0, p at N, u at 2N floats; the kernel writes every requested value
  const long long N = h->N;
  float *srho = static_cast<float *>(scratch), *sp = srho + N, *su = srho + 2 * N;
  cudaError_t e = cudaSuccess;
  rc = push_mirror(h);
  if (rc == LBM_OK) {
    lbm::count_launches(1);
    e = lbm::launch_moments(h->h, h->d, h->h.n, nullptr, nullptr, nullptr, rho ? srho : nullptr,
                            p ? sp : nullptr, u ? su : nullptr, h->stream);
    if (e == cudaSuccess && rho)
      e = cudaMemcpyAsync(rho, srho, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && p) e = cudaMemcpyAsync(p, sp, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && u)
      e = cudaMemcpyAsync(u, su, 3 * N * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (prev != dev) cudaSetDevice(prev);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(h, LBM_ECUDA, "moments_noalloc: %s", cudaGetErrorString(e));
  return LBM_OK;
}
