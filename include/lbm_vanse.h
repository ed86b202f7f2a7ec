/*
 * lbm_vanse.h -- C ABI of the GB300 (sm_103a) solver for the consistent
 * lattice Boltzmann scheme of the volume averaged Navier-Stokes equations
 * (VANSE) of Bukreev, Simonis, Kummerlaender, Jessberger and Krause,
 * arXiv 2208.09267.
 *
 * One handle holds one lattice: its populations, its volume fraction phi
 * (the paper's phi^flat, called epsilon here), its force fields and its time
 * counter, all in device memory owned by the library.  Every time step is
 * one fused CUDA kernel (Sec. 2.2): the zeroth and first moments, the
 * quadrature of phi over the cell (eq. (quad), Table "weights"), the
 * effective density (eq. (density)), the pressure-correction force
 * F_PC = c_s^2 rho~ grad(phi) (eq. (pressForce)), the velocity with the Guo
 * half-force shift (eq. (velocity)), the equilibrium with the zeroth moment
 * in place of rho~ phi (eq. (feq)), BGK relaxation with Guo forcing and
 * streaming (eq. (lbe)), with halfway bounce-back at walls.
 *
 * Conventions shared by every entry point:
 *   - Lattice units: dx = dt = 1, c_s^2 = 1/3, nu = (tau - 1/2)/3
 *     (Appendix A, last equation).
 *   - Fields are dense arrays with x fastest: index (z*ny + y)*nx + x.
 *     Vector fields are component-major: component a at offset a*N,
 *     N = nx*ny*nz.  In 2D (D2Q9) nz = 1 and vector fields still have three
 *     components (the third is ignored on input, zero on output).
 *   - `on_device` = 0: pointers are host memory (pageable or pinned); the
 *     call copies them before it returns.  `on_device` = 1: pointers are
 *     device memory of the current device; the call reads/writes them in
 *     stream order on the handle's stream and may return before the copy has
 *     run: keep the buffer alive until the stream has passed that point.
 *   - Inputs are always copied: the library keeps no caller pointer.
 *   - Every call returns an lbm_status; on failure lbm_vanse_last_error()
 *     gives a message.  No call aborts or exits.  A handle is not
 *     thread-safe: serialise calls on one handle.
 *   - All device work of a handle runs on the stream given at creation
 *     (params.cuda_stream, NULL = the legacy default stream).
 */
#ifndef LBM_VANSE_H
#define LBM_VANSE_H

#include <stddef.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_vanse *lbm_vanse_t;
typedef struct lbm_vanse_batch *lbm_vanse_batch_t;

/* Discrete velocity sets: D2Q9 (Table "latt_par"), D3Q27 (Table "latt_3d"),
   D3Q19 (not in the paper; standard textbook weights 1/3, 1/18, 1/36), and
   D1Q3 for one-dimensional problems (Sec. 2.2 names one-dimensional
   stencils beside the 2D and 3D ones; textbook weights 2/3, 1/6; needs
   ny = nz = 1 and is stepped one cell per thread). */
enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2, LBM_D1Q3 = 3 };

/* Population storage.  LBM_FP64: f_i stored and collided in double, in the
   canonical evaluation order, bit-identical to the FP64 reference.
   LBM_FP32: the deviation f_i/w_i - rho0*sigma stored in float, collided in
   float.  LBM_FP16_SHIFTED: the same deviation times 2^k stored in IEEE
   half, collided in float.  sigma is a per-cell shift, the quadrature
   int phi_ref dV of eq. (quad) rounded to half: f_i/w_i of the rest state,
   so that the stored deviations carry the flow signal and not the
   varpi grad^2 phi part of the zeroth moment.  A value is stored against
   the shift of the cell whose memory holds it. */
enum lbm_storage { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_SHIFTED = 2 };

enum lbm_status {
  LBM_OK = 0,
  LBM_EINVAL = -1,     /* bad argument or field value */
  LBM_ENOMEM = -2,     /* device allocation failed or HBM budget exceeded */
  LBM_ECUDA = -3,      /* a CUDA runtime call failed */
  LBM_EUNSTABLE = -4,  /* a check step saw NaN/Inf in the moments */
  LBM_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
  LBM_ESTATE = -6      /* call not valid in the handle's current state */
};

/* Bits of lbm_vanse_params.walls / quad_axes: axis x = 1, y = 2, z = 4. */
enum { LBM_AXIS_X = 1u, LBM_AXIS_Y = 2u, LBM_AXIS_Z = 4u };

typedef struct {
  int lattice;              /* enum lbm_lattice */
  int storage;              /* enum lbm_storage */
  int nx, ny, nz;           /* cells per axis, >= 1; nz must be 1 for D2Q9,
                               ny = nz = 1 for D1Q3 */
  double tau;               /* BGK relaxation time, eq. (lbe); > 0.5 */
  double rho0;              /* reference density; p = c_s^2 (rho~ - rho0) */
  int quad_dim;             /* row of Table "weights" (1, 2, 3); 0 = number
                               of bits in quad_axes; -1 = pointwise density
                               rho~ = M0 / phi(x) (varpi_0 = 1, the other
                               weights 0): the zeroth-moment reading of the
                               earlier scheme that Sec. 1 says misses the
                               pressure, for comparison only */
  unsigned quad_axes;       /* axes whose face neighbours enter eq. (quad);
                               0 = every lattice axis.  The paper picks the
                               D1Q3/D2Q5/D3Q7 rule by the number of
                               directions in which phi varies (Sec. 2.2). */
  unsigned walls;           /* axes whose first and last layer are solid
                               (halfway bounce-back); other axes periodic */
  int fp16_scale_log2;      /* k of LBM_FP16_SHIFTED (stored = dev * 2^k);
                               ignored for the other storages */
  void *cuda_stream;        /* cudaStream_t for all device work, or NULL */
  size_t hbm_budget_bytes;  /* 0 = unlimited; create fails with LBM_ENOMEM
                               when the handle would need more */
  int block_x, block_y;     /* thread-block shape of the one-cell-per-thread
                               step kernel; 0 = library default */
  int kernel;               /* step kernel: 0 = automatic (row-staged where
                               it fits and nx >= 32, else one cell per
                               thread), 1 = one cell per thread, 2 =
                               row-staged (tiles of whole x-rows staged in
                               shared memory by TMA bulk copies; needs
                               8 <= nx <= 512, FP32 or FP16 storage and no
                               walls on x; LBM_EINVAL otherwise) */
  int fp16_rounding;        /* LBM_FP16_SHIFTED stores: 0 = stochastic
                               rounding (unbiased; random bits from a
                               counter-based hash of cell and step, so runs
                               are reproducible), 1 = round to nearest */
  int quad_auto;            /* 1 = choose the quadrature rule from phi (Sec.
                               2.2: D1Q3, D2Q5 or D3Q7 according to how many
                               axes phi varies along): every
                               set_epsilon / commit_epsilon scans phi_ref and
                               d_t phi on the device and sets quad_axes to the
                               axes along which a value differs from its
                               neighbour's (every lattice axis when phi is
                               uniform) and quad_dim to their number; the scan
                               synchronises the handle's stream.  0 = use
                               quad_axes and quad_dim as given. */
  int drag_model;           /* phase-interaction drag in the force sum (Sec.
                               2.2 lists drag among the forces F_k; the
                               Conclusion names interaction forces):
                               0 = none; 1 = Ergun-type law of a fixed bed of
                               particles, F_D = -(b_lin + b_q |u|) u with
                               b_lin = rho~ c1 (1 - phi)^2 nu / (phi d^2),
                               b_q = rho~ c2 (1 - phi) / d, taken implicitly
                               in eq. (velocity) (u and the force sum stay
                               consistent with the Guo scheme).  Needs
                               0 < phi <= 1 everywhere (phi = 1: no drag). */
  double drag_c1, drag_c2;  /* Ergun coefficients (150 and 1.75 in Ergun's
                               correlation), >= 0 */
  double drag_d;            /* particle diameter, lattice units, > 0 */
  double les_cs;            /* Smagorinsky constant C >= 0 (the Conclusion
                               names LES): tau is replaced per cell by
                               (tau + sqrt(tau^2 + 18 sqrt(2) C^2 |Pi^neq| /
                               M0)) / 2, Pi^neq the non-equilibrium momentum
                               flux, filter width one cell; 0 = BGK.
                               drag_model or les_cs > 0 select the
                               one-cell-per-thread kernel (kernel = 2 then
                               fails with LBM_EINVAL). */
  int row_consumers;        /* row-staged kernel: consumer warps per block
                               (0 = the compiled default; values above the
                               compiled maximum fall back to it) */
  int row_stages;           /* row-staged kernel: rows staged in flight per
                               block (0 = default; 2 .. compiled maximum).
                               Neither changes the arithmetic, only the
                               launch shape; the autotuner picks them. */
} lbm_vanse_params;

/* Global sums of the state at time n (pre-collision), taken on a check step
   in FP64 on the device.  mass = sum M0, momentum = sum (J + F/2), residual =
   ||u^n - u^{n-K}||_2 / (K ||u^n||_2) over the cells, K = steps since the
   previous check (-1 when there is no previous check or residual tracking
   is off).  On a periodic lattice the Guo scheme gives sum J(n+1) -
   sum J(n) = force, so consecutive checks also pin the momentum input. */
typedef struct {
  double mass;
  double momentum[3];
  double residual;
  double u_norm;            /* ||u^n||_2 */
  double force[3];          /* sum of the force sum_k F_k over the cells */
  long long steps_done;     /* time counter n after the call */
  long long step_of_stats;  /* the n the sums describe */
  int nan_seen;             /* 1 if a check saw NaN or Inf */
  int converged;            /* 1 if the residual reached residual_tol */
} lbm_vanse_stats;

/* Library version string; never NULL. */
LBM_API const char *lbm_vanse_version(void);

/* Message of the last failed call on h (h may be NULL: last failure of
   any handle on this thread).  Never NULL; valid until the next call. */
LBM_API const char *lbm_vanse_last_error(lbm_vanse_t h);

/* Fill p with defaults: D3Q19, FP32, 32^3, tau 0.6, rho0 1, quad on every
   axis, no walls, k = 10, default stream, no budget, default block. */
LBM_API int lbm_vanse_params_default(lbm_vanse_params *p);

/* Device bytes a handle with these parameters allocates (populations,
   phi double buffer, shift double buffer, and with_deps / with_force_field:
   the d_t phi double buffer and the force fields, which are allocated
   lazily; plus the moment and reduction scratch).  Used for admission by
   HBM budget. */
LBM_API size_t lbm_vanse_device_bytes(const lbm_vanse_params *p, int with_deps, int with_force_field);

/* Create a lattice in the rest state u = 0, p = 0 with phi = 1 everywhere:
   f_i = w_i rho0 (eq. (equilibrium) with u = 0).  Errors: LBM_EINVAL for
   bad parameters, LBM_ENOMEM if allocation fails or exceeds the budget,
   LBM_ECUDA.  *out is NULL on failure. */
LBM_API int lbm_vanse_create(const lbm_vanse_params *p, lbm_vanse_t *out);

/* Release every device allocation of h (stream-ordered) and h itself.
   NULL is accepted. */
LBM_API void lbm_vanse_destroy(lbm_vanse_t h);

/* Set the volume fraction phi(x, t) = eps_ref(x) + (t - n_ref) deps_dt(x)
   (Sec. 2.2: phi varies in space and time; the pair is refreshed by the
   caller, and is exact at t = n_ref).  eps_ref: N values in (0, 1];
   deps_dt: N values or NULL for a static field.  The shift sigma of the
   reduced-precision storages is recomputed from eps_ref: the next step
   decodes with the previous sigma and encodes with the new one, so no extra
   pass over the populations runs.
   Errors: LBM_EINVAL if a host-side eps_ref value is not in (0, 1] or not
   finite, or a host-side deps_dt value is not finite (device-side inputs
   are not validated); a failed call leaves both fields as they were.
   LBM_ESTATE while a staged refresh awaits its commit (below).  The FP64
   twin takes doubles; on FP32/FP16 handles it rounds them to float. */
LBM_API int lbm_vanse_set_epsilon(lbm_vanse_t h, const float *eps_ref, const float *deps_dt,
                          long long n_ref, int on_device);
LBM_API int lbm_vanse_set_epsilon_f64(lbm_vanse_t h, const double *eps_ref, const double *deps_dt,
                              long long n_ref, int on_device);

/* The same refresh of phi(x, t) = eps_ref(x) + (t - n_ref) deps_dt(x)
   (Sec. 2.2) in two calls, so that its upload overlaps the steps between
   them.  lbm_vanse_stage_epsilon starts copying eps_ref and deps_dt (FP32,
   N values each, dense, x fastest; deps_dt NULL = static phi; on_device as
   in lbm_vanse_set_epsilon) into the handle's spare phi buffers on a copy
   stream of its own and returns without waiting; host values are then
   scanned there.  Steps issued meanwhile use the current phi.
   lbm_vanse_commit_epsilon waits for the copy and, if the values passed,
   makes them current: the state afterwards is bit for bit the one that
   lbm_vanse_set_epsilon(h, eps_ref, deps_dt, n_ref, on_device) called at
   the commit gives.
   Ownership: the caller's buffers are read asynchronously and must stay
   valid and unchanged until lbm_vanse_commit_epsilon returns (pinned host
   memory lets the copy overlap the steps).
   Errors: stage: LBM_EINVAL (NULL handle or eps_ref, FP64 storage),
   LBM_ESTATE (a staged refresh already awaits its commit), LBM_ENOMEM,
   LBM_ECUDA.  commit: LBM_ESTATE (nothing staged), LBM_EINVAL (a host value
   of eps_ref is not in (0, 1] or not finite, or one of deps_dt is not
   finite: the refresh is dropped and the lattice is unchanged), LBM_ECUDA.
   While a refresh is staged, lbm_vanse_set_epsilon, its FP64 twin and
   lbm_vanse_load_state return LBM_ESTATE. */
LBM_API int lbm_vanse_stage_epsilon(lbm_vanse_t h, const float *eps_ref, const float *deps_dt,
                            long long n_ref, int on_device);
LBM_API int lbm_vanse_commit_epsilon(lbm_vanse_t h);

/* External force density: sum_k F_k = g + field(x) + (t - n_ref) dfield_dt(x)
   + F_PC (Sec. 2.2 eq. (pressForce); Sec. 3, force sum of the manufactured
   examples).  g: three doubles (NULL = 0).  field, dfield_dt: 3*N values or
   NULL.  Errors: LBM_EINVAL for non-finite host values. */
LBM_API int lbm_vanse_set_force(lbm_vanse_t h, const double *g, const float *field,
                        const float *dfield_dt, long long n_ref, int on_device);
LBM_API int lbm_vanse_set_force_f64(lbm_vanse_t h, const double *g, const double *field,
                            const double *dfield_dt, long long n_ref, int on_device);

/* Initial populations at the current time n (eq. (equilibrium)):
   f_i = w_i rho~0 m(x) poly_i(u_eq) with rho~0 = rho0 + p0/c_s^2 and
   m = phi(x, n).  mode bit 1: m = int phi dV of eq. (quad) (the paper's
   form after the first step, eq. (feq)); bit 2: u_eq = u0 - F/(2 M0) so that
   eq. (velocity) returns u0 at time n.  p0: N values or NULL (0); u0: 3*N or
   NULL (0).  Solid cells are left empty. */
LBM_API int lbm_vanse_init_equilibrium(lbm_vanse_t h, const float *p0, const float *u0, int mode,
                               int on_device);
LBM_API int lbm_vanse_init_equilibrium_f64(lbm_vanse_t h, const double *p0, const double *u0,
                                   int mode, int on_device);

/* Advance up to max_steps time steps (eq. (lbe)), each one fused kernel
   launch (chunks of steps are replayed as a captured CUDA graph).  Every
   check_every steps (0 = only the last step) and on the last step, a check
   step also reduces mass, momentum and the velocity residual in FP64; when
   residual_tol > 0 and the residual falls to it, the call stops early.
   out (may be NULL) receives the last check's sums.  Synchronises with the
   stream once per check when residual_tol > 0, else once at the end.
   check_every = -1: no check step at all; the steps are only enqueued on
   the stream (no synchronisation), out gets steps_done and
   step_of_stats = -1, and residual_tol must be 0 (a wait-limit timeout in
   these steps is reported by the next call that checks).
   Errors: LBM_EUNSTABLE when a check saw NaN/Inf (the state is left as it
   is); LBM_ECUDA. */
LBM_API int lbm_vanse_step(lbm_vanse_t h, long long max_steps, double residual_tol, int check_every,
                   lbm_vanse_stats *out);

/* Macroscopic fields at the current time n from the pre-collision state:
   rho~ (eq. (density)), p = c_s^2 (rho~ - rho0), u (eq. (velocity)).
   rho, p: N values; u: 3*N values; any may be NULL.  Solid cells get 0. */
LBM_API int lbm_vanse_moments(lbm_vanse_t h, float *rho, float *p, float *u, int on_device);
LBM_API int lbm_vanse_moments_f64(lbm_vanse_t h, double *rho, double *p, double *u, int on_device);

/* Host copies of rho, p and u, the same values as lbm_vanse_moments with
   on_device = 0, read back without allocating any device memory.  The paper
   has no counterpart: this is a library service.

   lbm_vanse_moments stages host outputs in a temporary device buffer.  Some
   callers cannot allocate one: a server that has handed its whole device
   memory budget to resident lattices (a temporary buffer could fail with
   out-of-memory, or hold memory the budget gave to another lattice), or a
   thread that must not call into the CUDA allocator while other threads use
   the same memory pool.  This call stages the fields instead in one fixed
   device array of LBM_NOALLOC_SCRATCH_BYTES that the library reserves when
   it is loaded on a device.  Each cell needs 20 bytes, so lattices of at
   most LBM_NOALLOC_MAX_CELLS cells (nx*ny*nz) are accepted; larger ones
   fail with LBM_EINVAL and a message naming the limit.

   All calls on a device share that array: calls that overlap in time (from
   several host threads) race on it and may return each other's values, so
   callers must serialise them.  The call needs nothing in the array to start
   at zero (every staged value is written before it is read) and returns
   after the copies to the host have completed.  The first call on a device
   looks up the array's address there (cudaGetSymbolAddress, with that device
   current); when that set-up happens in the first call, make that call
   before any stream capture begins.  The address is kept for the rest of
   the process: it assumes that the device's primary context lives as long
   as the process (a cudaDeviceReset, or a primary context torn down and
   created again, leaves a stale address: do not call this entry point
   after either).  rho, p: N values; u: 3*N values; any
   may be NULL.  Errors: LBM_EINVAL (NULL handle, lattice too large),
   LBM_ECUDA. */
#define LBM_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
#define LBM_NOALLOC_MAX_CELLS ((long long)(LBM_NOALLOC_SCRATCH_BYTES / 20))
LBM_API int lbm_vanse_moments_noalloc(lbm_vanse_t h, float *rho, float *p, float *u);

/* Decoded populations f_i(x, n) in double, natural (not AA-swapped) order,
   array of structures f[cell*Q + i]; host memory.  For checks and dumps. */
LBM_API int lbm_vanse_get_populations(lbm_vanse_t h, double *f_host);

/* Number of kernels this library has launched in this process so far (a
   replayed graph counts each of its kernel nodes).  Diagnostic. */
LBM_API long long lbm_vanse_launch_count(void);

/* Iteration limit of the row-staged kernel's waits for its staged rows
   (0 = the default of 2^22 polls).  A wait that runs out makes the step
   return LBM_ETIMEOUT after the kernel has drained the copies it had in
   flight; the state of that step is then incomplete.  withhold_copies = 1
   (testing the timeout path only) makes the kernel issue no copies, so its
   first wait runs out on a barrier that nothing completes. */
LBM_API int lbm_vanse_set_wait_limit(lbm_vanse_t h, unsigned spins, int withhold_copies);

/* 1 if the handle's step runs the row-staged kernel, 0 for the one-cell-per-
   thread kernel, -1 for a NULL handle. */
LBM_API int lbm_vanse_uses_row_kernel(lbm_vanse_t h);

/* Launch shape of the handle's step (not in the paper; what the autotuner
   and the benchmark record): shape[0] = kernel (0 FP64 one cell per
   thread, 1 FP32/FP16 one cell per thread, 2 row-staged), then for the
   row-staged kernel consumer warps, staged rows and grid blocks, for the
   others block x, block y and grid blocks.  shape: 4 ints, caller-owned. */
LBM_API int lbm_vanse_launch_shape(lbm_vanse_t h, int *shape);

/* Time counter n and lattice description. */
LBM_API long long lbm_vanse_steps_done(lbm_vanse_t h);
LBM_API int lbm_vanse_get_params(lbm_vanse_t h, lbm_vanse_params *out);

/* Checkpoint: raw device state (populations in storage format, time counter,
   parity, phi, d_t phi, force fields, shift) to a host buffer.  Call with
   buf = NULL to get the size in *size.  Restoring into a handle created with
   the same parameters continues bit-identically. */
LBM_API int lbm_vanse_save_state(lbm_vanse_t h, void *buf, size_t *size);
LBM_API int lbm_vanse_load_state(lbm_vanse_t h, const void *buf, size_t size);

/* ---------------------------------------------------------------------- */
/* Batched stepping (many independent lattices advanced by persistent,    */
/* graph-captured kernels over one device work table of tiles).  Not in   */
/* the paper: the paper's Sec. 2.2 update is applied to each member.      */
/* ---------------------------------------------------------------------- */

/* Create an empty batch on `stream` (cudaStream_t or NULL) holding at most
   max_members lattices and max_tiles tiles; tile_cells is the number of
   stored cells one tile covers (0 = library default).  A member holds
   ceil(nxp*ny*nz / tile_cells) tiles, nxp being nx rounded up to a multiple
   of 8 (the stored row pitch).  Members must use FP32 or FP16 storage. */
LBM_API int lbm_vanse_batch_create(int max_members, int max_tiles, int tile_cells, void *stream,
                           lbm_vanse_batch_t *out);
LBM_API void lbm_vanse_batch_destroy(lbm_vanse_batch_t b);

/* Add lattice h with a budget of max_steps further steps; the handle stays
   owned by the caller and must outlive its membership.  Returns the member
   slot (>= 0) or an error (LBM_ENOMEM when the table is full). */
LBM_API int lbm_vanse_batch_add(lbm_vanse_batch_t b, lbm_vanse_t h, long long max_steps);
LBM_API int lbm_vanse_batch_remove(lbm_vanse_batch_t b, lbm_vanse_t h);

/* Advance every member by min(k, its remaining budget) steps in one graph
   replay of k fused steps per lattice type (k even).  With check = 1 the
   last step of the replay also reduces each member's statistics (read them
   with lbm_vanse_batch_stats after the call; the call synchronises).
   A member whose budget is spent idles. */
LBM_API int lbm_vanse_batch_step(lbm_vanse_batch_t b, int k, int check);
LBM_API int lbm_vanse_batch_stats(lbm_vanse_batch_t b, lbm_vanse_t h, lbm_vanse_stats *out);
LBM_API int lbm_vanse_batch_size(lbm_vanse_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_VANSE_H */
