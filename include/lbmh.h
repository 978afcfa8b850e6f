/*
 * lbmh — C ABI of a B300 (sm_103a) implementation of the lattice Boltzmann
 * method with adaptive relaxation parameter and Lax-Friedrichs-type
 * equilibrium for hyperbolic systems with source terms (Zhang, Lin, Zhao,
 * Zhao, arXiv 2609.18177).
 *
 * One call of lbmh_step advances the whole lattice by one collide-and-stream
 * step of Eq. (2.2) in the implementation form of Section 2.1:
 *   U = sum_k f_k (2.3); abar_j = max_x max_r |lambda_r(dF_j/dU)| (2.19);
 *   dt = CFL dx / sum_j abar_j, lambda = dx/dt (2.21);
 *   Lax-Friedrichs-type equilibrium (2.20); characteristic smoothness
 *   indicator (2.13)-(2.14), smoothed over the 3^d box (2.15), omega (2.16);
 *   collision plus half the source at x - e_k, pull streaming, the implicit
 *   moment (2.8) and the second half of the source at x.
 *
 * Conventions
 *   - Every function returns LBMH_OK (0) or a negative LBMH_ERR_* code.  The
 *     message of the last error of a handle is kept until the next call on
 *     that handle (lbmh_last_error).
 *   - The library owns the device memory of a handle (distributions, scratch,
 *     control block); the caller owns every array it passes in.
 *   - Work is enqueued on the CUDA stream given in the problem (NULL = the
 *     legacy default stream).  lbmh_step and lbmh_advance_to are asynchronous
 *     except where stated; lbmh_moments, lbmh_get_f, lbmh_omega and lbmh_info
 *     synchronise the stream.
 *   - A handle is not thread-safe.  Handles are independent.
 *   - Layouts: conservative state U is SoA FP64 [m][ny][nx] (x fastest;
 *     [m][nz][ny][nx] in 3D); distributions f are FP64 [Q][m][ny][nx]
 *     ([Q][m][nz][ny][nx] in 3D) with k = 0..2d in the order e_0 = 0,
 *     e_j = unit vector j, e_{j+d} = -e_j (Section 2.3).  In 1D, ny = 1.
 *     Nodes sit at cell centres x_i = x0 + (i + 1/2) dx.
 */
#ifndef LBMH_H
#define LBMH_H

#include <stdint.h>

#if defined(__GNUC__)
#define LBMH_API __attribute__((visibility("default")))
#else
#define LBMH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define LBMH_OK 0
#define LBMH_ERR_INVALID_ARG (-1)  /* bad problem description, pointer or size */
#define LBMH_ERR_OOM (-2)          /* device allocation failed */
#define LBMH_ERR_NONPHYSICAL (-3)  /* a step produced NaN/inf, rho<=0 or p<=0 */
#define LBMH_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up */
#define LBMH_ERR_CUDA (-5)         /* a CUDA runtime call failed */
#define LBMH_ERR_UNSUPPORTED (-6)  /* valid request this build does not provide */
#define LBMH_ERR_BOUNDS (-7)       /* bounds-checked build only: an index left its array (it was clamped) */

/* Physical systems, Section 5: scalar advection u_t + a.grad u = 0; Euler
 * (gamma-law gas); shallow water (g) with optional Gaussian bed-slope source;
 * reactive Euler with one-step Arrhenius kinetics.  LBMH_LINEAR (constant
 * symmetric matrices, Section 4) is accepted by the oracle only. */
typedef enum {
  LBMH_ADVECTION = 0,
  LBMH_EULER = 1,
  LBMH_SWE = 2,
  LBMH_REACTIVE_EULER = 3,
  LBMH_LINEAR = 4
} lbmh_system;

/* Boundary of each side (Section 5; the reading of each in the lattice is a
 * read of f^n at ghost nodes beyond the side):
 *   PERIODIC  wrapped node (must pair with the opposite side);
 *   OUTFLOW   zero gradient: the nearest interior node;
 *   REFLECT   reflecting wall (Example 5.13, y = +-15): the mirror node's
 *             distributions with the velocities normal to the wall exchanged
 *             and the normal momentum negated (needs >= 4 nodes across);
 *   INFLOW    fixed state (Example 5.13, x = 40): f^eq(u_in) with the step's
 *             alpha and lambda.
 * REFLECT and INFLOW are implemented by the fused kernels (and the batch
 * engine); the unfused path and lbmh_step_static return
 * LBMH_ERR_UNSUPPORTED for them. */
typedef enum { LBMH_BC_PERIODIC = 0, LBMH_BC_OUTFLOW = 1, LBMH_BC_REFLECT = 2, LBMH_BC_INFLOW = 3 } lbmh_bc;

/* LBMH_FP64: distributions stored and collided in FP64.
 * LBMH_FP32: distributions stored and collided in FP32; the step control and
 * the conservation sums stay in FP64; the Arrhenius root of Eq. (2.8) is found
 * in FP32 (it is stored in FP32) and in FP64 where that does not converge. */
typedef enum { LBMH_FP64 = 0, LBMH_FP32 = 1 } lbmh_precision;

typedef enum { LBMH_OMEGA_ADAPTIVE = 0, LBMH_OMEGA_FIXED = 1 } lbmh_omega_mode;

/* Step implementation: the fused single-pass kernel (default where
 * available) or the unfused four-kernel reference path. */
typedef enum { LBMH_KERNEL_AUTO = 0, LBMH_KERNEL_FUSED = 1, LBMH_KERNEL_UNFUSED = 2 } lbmh_kernel;

/* Statement of the balance law (2.1) and its discretisation.  Field names
 * follow the paper: cfl of (2.21), eps of alpha_j = abar_j + eps (Section 5
 * uses 1e-10), omega from (2.16) unless omega_mode is FIXED. */
typedef struct lbmh_problem {
  int system;          /* lbmh_system */
  int dim;             /* 1, 2 or 3; the lattice is DdQ(2d+1) */
  int nx, ny;          /* nodes per direction (ny ignored in 1D) */
  double x0, x1, y0, y1; /* domain; 2D requires (x1-x0)/nx == (y1-y0)/ny */
  int bc[4];           /* lbmh_bc at x-lo, x-hi, y-lo, y-hi; periodic must pair */
  double cfl, eps;
  double adv[2];       /* advection velocity a */
  double gamma, g;     /* Euler ratio of specific heats; gravity */
  double bed_amp, bed_w2, bed_xc, bed_yc; /* bed b = amp exp(-((x-xc)^2+(y-yc)^2)/w2) */
  double K, Ti, q;     /* Arrhenius rate constant, activation temperature, heat release */
  int m_linear;        /* LBMH_LINEAR only */
  const double *A;     /* LBMH_LINEAR only */
  int omega_mode;      /* lbmh_omega_mode */
  double omega_fixed;
  double h_dry;        /* shallow water: h < h_dry is dry (u = v = 0); 1e-5 if 0 */
  int precision;       /* lbmh_precision */
  int kernel;          /* lbmh_kernel */
  void *cuda_stream;   /* cudaStream_t to enqueue on */
  double sponge_width; /* > 0: sponge layer over [x0, x0 + sponge_width] (Example 5.13): omega is
                          blended toward 1, omega' = 1 + (omega - 1)(1 - sigma(x)),
                          sigma = (1 + cos(pi (x - x0) / sponge_width)) / 2; 0: none */
  double u_in[8];      /* conservative state (first m entries) held by INFLOW sides */
  /* 3D (dim = 3, the D3Q7 lattice; the paper names 3D as future work):
   * advection, Euler and reactive Euler, periodic or outflow sides;
   * KERNEL_AUTO takes the fused z-marching kernel in FP32 and the four-kernel
   * path (KERNEL_UNFUSED) in FP64; dx == dy == dz required.  U and f are
   * laid out [..][nz][ny][nx]. */
  int nz;
  double z0, z1;
  int bc_z[2];         /* lbmh_bc at z-lo, z-hi */
  double adv_z;        /* advection velocity along z */
} lbmh_problem;

typedef struct lbmh_handle lbmh_handle;

/* Diagnostics of the current state (after the last enqueued step). */
typedef struct lbmh_info {
  double t;            /* simulated time */
  int64_t steps;       /* steps executed */
  double abar[2];      /* speed bound of the current state (2.19) */
  double last_dt, last_lambda; /* of the last executed step */
  double sum_U[8];     /* FP64 sum over nodes of U after the last executed step */
  uint32_t status;     /* bit 0: non-physical state (NaN/inf, rho<=0, p<=0); bit 1: reaction
                          root not converged; bit 2: a bounded device wait gave up; bit 3:
                          negative depth h < -1e-12 (reported only: the scheme is not
                          positivity preserving at wet-dry fronts); bit 4: an index left its
                          array (bounds-checked build only) */
  int m, Q;            /* fields and velocities */
  int kernel;          /* implementation in use: LBMH_KERNEL_FUSED or _UNFUSED */
  int64_t device_bytes; /* device memory owned by the handle */
  double abar_z;       /* 3D: speed bound along z of the current state (2.19); 0 in 1D/2D */
  /* slabs (lbmh_create_slab); zero for other handles */
  int64_t halo_bytes;  /* bytes of one block of three halo rows (lbmh_halo_get / _set) */
  int halo_rows[2];    /* halo rows below and above the rows the slab writes (0 or 3) */
  int row0;            /* global row index of the slab's local row 0 */
} lbmh_info;

/* Validate the problem and allocate device memory for it.  *out receives a
 * handle (NULL on error).  The state is undefined until lbmh_set_state. */
LBMH_API int lbmh_create(const lbmh_problem *p, lbmh_handle **out);

/* Set t = 0 and f_k := f_k^eq(U) with alpha and lambda from U (Eq. 2.20).
 * U: FP64 [m][ny][nx]; a device pointer when on_device != 0, else host.
 * Enqueued on the handle's stream; a host U is copied before returning. */
LBMH_API int lbmh_set_state(lbmh_handle *h, const double *U, int on_device);

/* Enqueue n time steps (n >= 0).  Asynchronous; no host synchronisation. */
LBMH_API int lbmh_step(lbmh_handle *h, int64_t n);

/* Step until t >= T (the step that crosses T is taken whole; there is no
 * clipped final step) or max_steps steps were taken.  Synchronises the
 * stream every few dozen steps to test t. */
LBMH_API int lbmh_advance_to(lbmh_handle *h, double T, int64_t max_steps);

/* U = sum_k f_k of the current state into U_out (FP64 [m][ny][nx], device
 * pointer if on_device).  Synchronises.  t and steps may be NULL.  Returns
 * LBMH_ERR_NONPHYSICAL if a step flagged a non-physical state. */
LBMH_API int lbmh_moments(lbmh_handle *h, double *U_out, int on_device, double *t, int64_t *steps);

/* Checkpoint: copy the distributions out (FP64 [Q][m][ny][nx], host or
 * device), or replace them together with the time and step count.  A
 * restored handle continues bitwise-identically. */
LBMH_API int lbmh_get_f(lbmh_handle *h, double *f_out, int on_device, double *t, int64_t *steps);
LBMH_API int lbmh_set_f(lbmh_handle *h, const double *f_in, int on_device, double t, int64_t steps);

/* omega of every node that the next step will use (Eq. 2.16), FP64 [ny][nx]. */
LBMH_API int lbmh_omega(lbmh_handle *h, double *out, int on_device);

/* Fill *out; synchronises. */
LBMH_API int lbmh_get_info(lbmh_handle *h, lbmh_info *out);

/* Free everything owned by the handle.  NULL is accepted. */
LBMH_API int lbmh_destroy(lbmh_handle *h);

/* Message of the last error on h (or, when h is NULL, of the calling host
 * thread's last failure without a handle: lbmh_create, lbmh_step_static).
 * Never NULL. */
LBMH_API const char *lbmh_last_error(const lbmh_handle *h);

/* ------------------------------------------------------------------------
 * Slabs: one 2D lattice decomposed along y into row ranges, one handle per
 * range (one per GPU, the paper's "parallel multidimensional computations",
 * Section 6).  The step of Eq. (2.2) needs f^n up to three nodes away, and its
 * only global quantity is the speed bound abar_j of Eq. (2.19), a maximum
 * over all nodes.  So a slab stores its rows plus three halo rows on each
 * side that borders another slab, writes only its own rows, and per step:
 *   1. the caller takes the maximum over the slabs of lbmh_get_speed_bound
 *      and hands it to every slab with lbmh_set_speed_bound;
 *   2. lbmh_step(h, 1) on every slab;
 *   3. lbmh_halo_get of each side with a neighbour is passed to that
 *      neighbour's lbmh_halo_set of the facing side.
 * The initial state: each slab computes lbmh_state_speed_bound of its U0
 * rows, the caller takes the maximum and calls lbmh_set_state_bound.  Node
 * positions follow global rows and every node runs the arithmetic of the
 * single-lattice step, so the slabs' rows hold the bits of the whole lattice
 * stepped as one.  Slabs run the fused kernel (FP32 or FP64).
 * ------------------------------------------------------------------------ */

/* Create the slab holding rows [row_begin, row_end) (at least 3) of the 2D
 * lattice `global`.  Its local lattice has (row_end - row_begin) rows plus 3
 * halo rows on each side that borders another slab (a y-periodic lattice cut
 * into several slabs: both sides); lbmh_get_info reports them.  U, f and
 * moments of the handle cover the local lattice, halo rows included (their
 * values after a step are those of the last lbmh_halo_set). */
LBMH_API int lbmh_create_slab(const lbmh_problem *global, int row_begin, int row_end, lbmh_handle **out);

/* Speed bound (Eq. 2.19) of a conservative state U (layout of
 * lbmh_set_state) over the handle's nodes into abar_out[0..d-1].  The
 * handle's state is unchanged.  Synchronises.  1D and 2D. */
LBMH_API int lbmh_state_speed_bound(lbmh_handle *h, const double *U, int on_device, double *abar_out);

/* As lbmh_set_state, with alpha^0 and lambda^0 of the initial equilibrium
 * (Eq. 2.20, 2.21) taken from abar[0..d-1] (positive, finite) instead of U's
 * own speed bound: a slab passes the maximum over all slabs.  1D and 2D. */
LBMH_API int lbmh_set_state_bound(lbmh_handle *h, const double *U, int on_device, const double *abar);

/* The speed bound the next step will use (Eq. 2.19: the side output of the
 * previous step, over the nodes this handle writes) into abar_out[0..d-1].
 * Synchronises. */
LBMH_API int lbmh_get_speed_bound(lbmh_handle *h, double *abar_out);

/* Replace the speed bound the next step uses to form dt, lambda and alpha_j
 * (Eq. 2.19-2.21) by abar[0..d-1] (non-negative).  Enqueued on the handle's
 * stream.  1D and 2D. */
LBMH_API int lbmh_set_speed_bound(lbmh_handle *h, const double *abar);

/* Slabs: the three rows of the current state next to side `side` (0: low y,
 * 1: high y) among the rows the slab writes -- the rows the neighbour across
 * that side keeps as its halo -- copied into `rows` (lbmh_info.halo_bytes
 * bytes: all Q*m planes, three whole padded rows each, in the storage
 * precision; host or device).  A host copy synchronises.
 * LBMH_ERR_INVALID_ARG on a side without a neighbour. */
LBMH_API int lbmh_halo_get(lbmh_handle *h, int side, void *rows, int on_device);

/* Slabs: store a neighbour's lbmh_halo_get block as the halo rows beyond side
 * `side`.  Synchronises. */
LBMH_API int lbmh_halo_set(lbmh_handle *h, int side, const void *rows, int on_device);

/* ------------------------------------------------------------------------
 * Batches: many 2D lattices of one system and precision, of uneven sizes,
 * advanced together by one persistent kernel launch per step (replayed from
 * a captured CUDA graph three steps at a time); the resident CTAs take
 * segments of rows from a shared counter, so lattices that finish early free
 * their share of the GPU at once.  Each lattice keeps its own
 * time step (Eq. 2.21 from its own speed bound), time and step count, and
 * stops by itself at its step target or end time.  Lattices live in a device
 * arena of fixed capacity allocated at creation; lbmh_batch_add admits a
 * lattice only if its footprint fits (first-fit), so a caller can queue work
 * by HBM footprint.  Not thread-safe; batches are independent.
 * ------------------------------------------------------------------------ */
typedef struct lbmh_batch lbmh_batch;

/* Create an empty batch of `system` (2D only) in `precision` with a device
 * arena of capacity_bytes and room for max_instances lattices. */
LBMH_API int lbmh_batch_create(int system, int precision, int64_t capacity_bytes, int max_instances,
                               void *cuda_stream, lbmh_batch **out);

/* Device bytes one lattice of problem p occupies in a batch arena (two
 * distribution copies), or -1 for an invalid problem. */
LBMH_API int64_t lbmh_batch_footprint(const lbmh_problem *p);

/* Admit a lattice: f := f^eq(U0) (U0 FP64 [m][ny][nx], host or device).  It
 * stops after max_steps steps (if > 0) or once t >= T (if T > 0).  *slot
 * receives its index.  LBMH_ERR_OOM when the arena or the slots are full.
 * Synchronises the stream. */
LBMH_API int lbmh_batch_add(lbmh_batch *b, const lbmh_problem *p, const double *U0, int on_device,
                            int64_t max_steps, double T, int *slot);

/* Free a lattice's slot and arena space.  Synchronises. */
LBMH_API int lbmh_batch_remove(lbmh_batch *b, int slot);

/* Enqueue n batched steps (lattices that reached their target are skipped). */
LBMH_API int lbmh_batch_step(lbmh_batch *b, int64_t n);

/* Time each kernel variant (ring depth 1 or 2 rows ahead; segments of 64,
 * 128, 256 or 512 rows) on the live batch for steps_per_candidate steps and
 * keep the fastest.  Every timed launch is a real step of the batch.
 * *best_ms (may be NULL) receives the chosen variant's time per step. */
LBMH_API int lbmh_batch_autotune(lbmh_batch *b, int steps_per_candidate, double *best_ms);

/* Per slot (arrays of max_instances, any may be NULL): done = 1 finished
 * (target reached or non-physical), 0 running, -1 free; time; steps; status
 * bits.  Synchronises. */
LBMH_API int lbmh_batch_poll(lbmh_batch *b, int *done, double *t, int64_t *steps, uint32_t *status);

/* U = sum_k f_k of one lattice into U_out (FP64 [m][ny][nx]).  Synchronises
 * when U_out is a host array. */
LBMH_API int lbmh_batch_moments(lbmh_batch *b, int slot, double *U_out, int on_device);

/* Arena use, capacity, live lattices, grid size and the chosen variant
 * (1000 * rows ahead + rows per segment). */
LBMH_API int lbmh_batch_info(lbmh_batch *b, int64_t *used_bytes, int64_t *capacity_bytes, int *active, int *grid,
                             int *variant);

LBMH_API int lbmh_batch_destroy(lbmh_batch *b);
LBMH_API const char *lbmh_batch_last_error(const lbmh_batch *b);

/* One time step that allocates no device memory (the paper has no
 * counterpart: this is a deployment entry point).  Meant for callers that
 * cannot call cudaMalloc: code inside a host callback or a CUDA-graph node
 * where allocation is illegal, runtimes that only hand out memory from a
 * frozen pool, or real-time loops that cannot afford the implicit device
 * synchronisation an allocation may cause.  No handle is needed.
 *
 * f_in, f_out: distinct, non-overlapping device arrays of exactly
 * Q*m*ny*nx doubles each, FP64 [Q][m][ny][nx] (the layout of lbmh_get_f;
 * ny = 1 in 1D), on the current device; the step reads f_in and writes f_out.
 * The library cannot check their sizes: a smaller array makes the kernels
 * read or write past it.  dt, lambda and the speed bound are computed from
 * f_in exactly as lbmh_step computes them for a handle's state.
 * dt_out, status_out: NULL, or host pointers that receive the step's dt and
 * its status bits (those of lbmh_info.status: non-physical state, reaction
 * root not converged, negative depth); when either is given the call
 * synchronises the stream and returns LBMH_ERR_NONPHYSICAL if the new state
 * is non-physical.  Only LBMH_FP64 is accepted.
 *
 * The intermediate arrays live in one static device array of 16 MiB that
 * every GPU loading this library holds until the process exits; grids whose
 * ghost-extended scratch does not fit ((nx+6)(ny+6)(m+2) doubles plus a few
 * KB) are rejected with LBMH_ERR_INVALID_ARG.  Outside a stream capture each
 * call looks the array's device address up (cudaGetSymbolAddress); under a
 * capture the address found by an earlier call on the same device is used,
 * so make one call on each device before capturing.  All calls share the
 * array and each call clears the part that must start from zero: calls that
 * may overlap on the GPU (other streams, other host threads) race with each
 * other and must be serialised by the caller.  Errors are reported through
 * lbmh_last_error(NULL), which keeps one message per host thread. */
LBMH_API int lbmh_step_static(const lbmh_problem *p, const double *f_in, double *f_out, double *dt_out,
                              uint32_t *status_out);

/* Library version string. */
LBMH_API const char *lbmh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBMH_H */
