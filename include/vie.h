/*
 * libvie -- GB300-native circulant-preconditioned voxel VIE solver (C ABI).
 *
 * Problem (Groth, Polimeridis, Tambova, White, "Circulant preconditioning in
 * the volume integral equation method for silicon photonics", Sec. 2,
 * Eqs. JVIE and discrete_form): on a uniform grid of nx*ny*nz cubic voxels of
 * edge h, solve
 *
 *      (I - M N) w = M e_inc,        M = (eps_r - 1)/eps_r  per voxel,
 *
 * for the normalised polarisation current w = j / (j omega eps0).  eps_r is
 * the permittivity relative to the background eps_bg (Table 1, "Si in SiO2"),
 * N = I + G is the Galerkin JVIE operator with the background wavenumber
 * k_b = k0 sqrt(eps_bg), time dependence exp(+j omega t), eps = eps' - j eps''.
 * G's entries: one-point rule between distinct voxels and the equal-volume
 * sphere self term (the paper does not print its singular integrals).
 *
 * Layouts (all arrays C-ordered, x fastest):
 *   scalar voxel field   [nz][ny][nx]           complex (double2: re, im)
 *   vector voxel field   [3][nz][ny][nx]        components x, y, z
 *
 * Ownership: every pointer argument marked "device" must point to memory of
 * the device that is current when the plan is created, allocated and freed by
 * the caller.  "host" pointers are ordinary (preferably pinned) host memory.
 * The library owns everything inside a plan (generator spectra, material
 * arrays, preconditioner blocks, Krylov workspace); it allocates device
 * memory in vie_plan_create, vie_build_preconditioner, the first vie_solve of
 * a plan (Krylov workspace), the first vie_solve_host of a plan (its three
 * staging buffers), the first FP64 fallback of a mixed solve (see
 * vie_solve) and the vie_server_* calls, and never inside vie_matvec /
 * vie_precond_apply or later solves of the same plan.
 *
 * Streams: every call enqueues its GPU work on the stream given at plan
 * creation (NULL = legacy default stream).  vie_matvec and vie_precond_apply
 * return without synchronising; vie_build_preconditioner and vie_solve
 * synchronise that stream before returning.
 *
 * Errors: every call returns a vie_status.  Negative values are hard errors
 * (the message is available from vie_last_error() on the calling thread);
 * VIE_ENOCONV (1) means the solver stopped at its iteration limit and the
 * best iterate was written.  No call throws or aborts.
 */
#ifndef LIBVIE_VIE_H
#define LIBVIE_VIE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VIE_OK = 0,
  VIE_ENOCONV = 1,      /* iteration limit reached; best iterate returned     */
  VIE_PENDING = 2,      /* vie_server_poll: request not finished yet          */
  VIE_EINVAL = -1,      /* invalid argument or unsupported size               */
  VIE_ENOMEM = -2,      /* device or host allocation failed                   */
  VIE_ECUDA = -3,       /* CUDA runtime error                                 */
  VIE_ETIMEOUT = -4,    /* a bounded wait ran out                             */
  VIE_EREJECTED = -5,   /* server admission refused the request               */
  VIE_ESTATE = -6       /* call out of order (e.g. solve before permittivity)  */
} vie_status;

typedef enum { VIE_FP64 = 0, VIE_MIXED = 1 } vie_precision;

/* Homogenisation of M for the preconditioner, Sec. 5.2 (three variants). */
typedef enum { VIE_HOM_MODE = 1, VIE_HOM_MEAN = 2, VIE_HOM_REALMEAN = 3 } vie_homog;

/* Preconditioner: none (identity) or the 1-level circulant of Sec. 4. */
typedef enum { VIE_PREC_NONE = 0, VIE_PREC_CIRCULANT = 1 } vie_precond_kind;

/* Axis-aligned partition box in voxel indices (Sec. 5.3).  levels selects the
 * circulant approximation of the box: 1 (or 0) the 1-level preconditioner of
 * Sec. 4 (blocks of m = 3 ny nz per x-frequency, memory reduction allowed);
 * 2 the 2-level (Chan-Olkin) preconditioner of the paragraph after the C_B^-1
 * display (blocks of 3 nz per (x, y) frequency pair, M homogenised over each
 * z-plane, no memory reduction; nz <= 32). */
typedef struct { int x0, y0, z0, nx, ny, nz, levels; } vie_box;

typedef struct {
  int restart;            /* GMRES restart length (default 50)                      */
  double tol;             /* stop at ||b - A w||_2 / ||b||_2 <= tol (FP64 residual) */
  int max_iter;           /* cap on total GMRES iterations (all restarts/refinements)*/
  double inner_tol;       /* mixed: floor of each inner c64 cycle's relative target */
  int max_refine;         /* mixed: cap on FP64 iterative-refinement steps          */
  int precision;          /* vie_precision                                          */
  int precond;            /* vie_precond_kind                                       */
  int homog;              /* vie_homog                                              */
  double reduce_tol;      /* memory reduction threshold tau (Sec. 5.1.1); 0 = off   */
  const vie_box* boxes;   /* partition boxes (copied at plan creation); NULL = one  */
  int nboxes;             /*   box covering the whole grid                          */
  int inner_restart;      /* mixed: length of each complex-FP32 GMRES cycle; 0 =   */
                          /*   min(2 restart, 128), the FP64 GMRES(restart) basis  */
                          /*   bytes in complex FP32                                */
} vie_opts;

typedef struct {
  int iters_inner;        /* total GMRES iterations                                  */
  int iters_outer;        /* FP64 refinement steps (1 for VIE_FP64)                  */
  double relres;          /* final ||b - A w|| / ||b|| computed in FP64              */
  size_t precond_bytes;   /* device bytes held by the preconditioner blocks          */
  double kept_fraction;   /* kept blocks / total frequencies over all boxes          */
  float t_setup_ms;       /* preconditioner build time of the last build             */
  float t_solve_ms;       /* wall time of the last solve                             */
  long long precond_blocks;    /* stored (inverted) blocks over all boxes: the kept
                                  frequencies f <= n/2 plus one representative each  */
  long long precond_discarded; /* frequencies applied with the representative block
                                  (the discarded ones, Sec. 5.1.1), over all boxes    */
  int reorth_passes;           /* Arnoldi steps that took the second Gram-Schmidt pass */
  int iters_fp64_fallback;     /* mixed: GMRES iterations run in FP64 after the
                                  refinement stalled (a correction that raised the
                                  FP64 residual, or three steps under 1% gain); 0
                                  when the complex-FP32 inner solves sufficed.
                                  Included in iters_inner.                        */
} vie_info;

typedef struct vie_plan_s* vie_plan_t;

/* Fill *opts with the defaults: restart 50, tol 1e-9, max_iter 5000,
 * inner_tol 1e-6, max_refine 1000, VIE_MIXED, VIE_PREC_CIRCULANT,
 * VIE_HOM_REALMEAN, reduce_tol 1e-3, whole-grid box, inner_restart 0. */
void vie_default_opts(vie_opts* opts);

/* Create a plan for an nx*ny*nz grid of voxel edge h (same length unit as
 * 1/k0), free-space wavenumber k0 and background permittivity eps_bg (Sec. 2;
 * Eq. sys_mat).  Assembles the 6 unique Green's generators in FP64 and
 * stores their circulant-embedding spectra (the O(6n) storage of the remark
 * after Eq. sys_mat).  cuda_stream: a cudaStream_t or NULL.  opts may be
 * NULL (defaults).  Boxes must lie inside the grid and not overlap.
 * Cross-sections whose embedding Py x Pz exceeds 4096 points take the y and z
 * transforms of the matvec as separate line passes (one more work array).
 * The x-embedding is 2 smooth(nx) (smooth: the next 2-3-5-7-smooth integer),
 * or 8 smooth(ceil(nx/4)) where the complex-FP32 x pass splits over a
 * cluster of CTAs (every L >= 2 nx - 1 gives the same product).
 * Errors: VIE_EINVAL for non-positive sizes, h, k0 or eps_bg, boxes out of
 * range / overlapping, box levels outside 0..2, 3*nx*ny*nz >= 2^31 - 64, an
 * embedding or box length beyond the transform limits, and, when a
 * preconditioner is requested, a 1-level box with 3 ny nz > 864 or a 2-level
 * box with nz > 32 or (nx/2+1)(ny/2+1) > 65535; VIE_ENOMEM if device memory
 * runs out. */
vie_status vie_plan_create(int nx, int ny, int nz, double h, double k0, double eps_bg,
                           const vie_opts* opts, void* cuda_stream, vie_plan_t* out);

/* Release every device and host resource of the plan (NULL is ignored). */
void vie_plan_destroy(vie_plan_t plan);

/* Set the relative permittivity eps_r = eps' - j eps'' (device, double2,
 * [nz][ny][nx], relative to vacuum; eps' > 0).  Computes M (Sec. 2) on the
 * device.  Invalidates a previously built preconditioner. */
vie_status vie_set_permittivity(vie_plan_t plan, const void* eps_dev);

/* Build the block-diagonal 1-level circulant preconditioner of Sec. 4 / 5.3:
 * per box, homogenise M (Sec. 5.2), form the Chan eigenvalues (Eq. Chan and
 * the diagonalisation C = F^-1 Lambda F), assemble the per-frequency blocks
 * D_f (Eq. Di), select the kept blocks (Eqs. proxy1-proxy2) when
 * reduce_tol > 0, and factor every kept block by LU with partial pivoting
 * (complex FP64 for VIE_FP64; complex FP32, from the FP64-assembled blocks,
 * for VIE_MIXED); the explicit inverse is stored in the solve's precision.
 * Synchronises the plan stream.  No-op for VIE_PREC_NONE. */
vie_status vie_build_preconditioner(vie_plan_t plan);

/* y = A x = x - M (x + G x) (Eq. discrete_form) for device vectors x, y
 * ([3][nz][ny][nx] double2; may not alias).  precision VIE_FP64 computes in
 * complex FP64; VIE_MIXED rounds x to complex FP32, applies the FP32 operator
 * and widens the result.  Asynchronous on the plan stream. */
vie_status vie_matvec(vie_plan_t plan, const void* x_dev, void* y_dev, int precision);

/* z = P^{-1} r with the built preconditioner (identity outside the boxes),
 * device vectors [3][nz][ny][nx] double2 (no aliasing).  precision as for
 * vie_matvec.  VIE_ESTATE if the preconditioner was not built. */
vie_status vie_precond_apply(vie_plan_t plan, const void* r_dev, void* z_dev, int precision);

/* Solve (I - M N) w = M e_inc (Sec. 2) with right-preconditioned GMRES
 * (restart opts.restart).  VIE_FP64: complex FP64 throughout.  VIE_MIXED:
 * FP64 iterative refinement whose every step runs one complex-FP32 GMRES
 * cycle on the scaled FP64 residual (stopped early at the relative target
 * max(inner_tol, tol ||b|| / (2 ||r||))), so GMRES restarts from FP64
 * residuals.  When a correction raises the FP64 residual (it is taken back)
 * or three steps in a row gain less than 1%, the solve goes on as FP64
 * GMRES(restart) from its iterate: the first time, this builds the
 * complex-FP64 inverses of the preconditioner and allocates the FP64 basis
 * (as for VIE_FP64); info->iters_fp64_fallback counts those iterations.
 * e_inc and w_out are
 * device [3][nz][ny][nx] double2.  Builds the preconditioner if needed.
 * info may be NULL.  Synchronises the plan stream. */
vie_status vie_solve(vie_plan_t plan, const void* e_inc_dev, void* w_out_dev, vie_info* info);

/* As vie_set_permittivity + vie_solve, with host buffers: copies eps and
 * e_inc to the device, solves and copies w back (host, double2 arrays).
 * The first call on a plan allocates three device staging buffers (eps,
 * e_inc and w: 7 N complex FP64 values); the plan keeps them for later
 * calls and frees them in vie_plan_destroy. */
vie_status vie_solve_host(vie_plan_t plan, const void* eps_host, const void* e_inc_host,
                          void* w_out_host, vie_info* info);

/* Solve n independent problems (each plan already has its permittivity; all
 * plans on the current device, each at most once) in lockstep: their GMRES
 * runs advance together, one captured step graph per set of plans holds
 * each plan's preconditioner and matvec as parallel branches and then the
 * Arnoldi step kernels as single launches over a work-list of all plans of
 * a precision, so plans of different lengths, cross-sections, precisions
 * and options batch together.  A plan's host-side work between cycles runs
 * on its own stream.  Each result is bitwise the result of vie_solve on that
 * plan alone.  e_inc[i], w_out[i] are device pointers; info may be NULL or
 * an array of n.  Returns the most severe status. */
vie_status vie_solve_batch(vie_plan_t* plans, int n, const void* const* e_inc_dev,
                           void* const* w_out_dev, vie_info* info);

/* Continuous-batching server.  Requests are admitted in arrival order while
 * their estimated device footprint fits in budget_bytes and fewer than
 * max_inflight (1..256) are admitted.  Up to four worker threads prepare
 * admitted requests (plan, upload, preconditioner); one driver thread keeps
 * all prepared requests in one lockstep set (as vie_solve_batch), which
 * requests join between chunks of steps as they become ready and leave as
 * they finish.  Each result equals the request's vie_solve result bitwise.
 * A request that can never fit is rejected (VIE_EREJECTED). */
typedef struct vie_server_s* vie_server_t;

vie_status vie_server_create(size_t budget_bytes, int max_inflight, vie_server_t* out);

/* Submit one solve: grid/physics as in vie_plan_create, permittivity and
 * incident field as HOST double2 arrays (copied before return), result to
 * the HOST array w_out (written before the request reports VIE_OK).
 * *ticket receives the request id. */
vie_status vie_server_submit(vie_server_t srv, int nx, int ny, int nz, double h, double k0,
                             double eps_bg, const vie_opts* opts, const void* eps_host,
                             const void* e_inc_host, void* w_out_host, int64_t* ticket);

/* VIE_OK (finished, *info filled), VIE_PENDING, or the request's error. */
vie_status vie_server_poll(vie_server_t srv, int64_t ticket, vie_info* info);

/* Block until every submitted request has finished or timeout_ms elapses
 * (VIE_ETIMEOUT). */
vie_status vie_server_drain(vie_server_t srv, double timeout_ms);

/* Bytes currently reserved by admitted requests. */
size_t vie_server_reserved_bytes(vie_server_t srv);

/* Estimated device bytes of a plan with these sizes and options (used by
 * admission control). */
size_t vie_estimate_bytes(int nx, int ny, int nz, const vie_opts* opts);

void vie_server_destroy(vie_server_t srv);

/* Allocation-free matvec.  The paper has no counterpart: this entry point
 * exists for callers that may not allocate device memory at all (a host
 * framework that owns every byte of the GPU through its own pool, a
 * real-time loop with a fixed budget), and so cannot create a plan.
 * Computes the same y = x - M (x + G x) in complex FP64 as
 * vie_matvec(plan, x, y, VIE_FP64) for a plan with this grid, voxel size,
 * wavenumber, background and permittivity, from the caller's buffers only:
 * eps_dev [nz][ny][nx], x_dev and y_dev [3][nz][ny][nx] (device, double2;
 * y may not overlap x or eps in any byte: VIE_EINVAL), cuda_stream a
 * cudaStream_t or NULL.  Every temporary lives in one file-scope device
 * array of 64 MiB inside libvie (held by each GPU from the first call -- or
 * from context creation under eager module loading -- until the process
 * exits); grids that need more, or whose x-embedding exceeds 4266 points
 * (nx > 2130) or whose Py*Pz exceeds 4096, are rejected with VIE_EINVAL and
 * a message.  Every call looks up the array's device address on the current
 * device (cudaGetSymbolAddress); under lazy module loading the first call on
 * a device also loads libvie's device code there, so make that first call
 * before any stream capture.  All calls share the array: calls whose GPU
 * work overlaps (other streams or threads) race and corrupt each other's
 * results.  Calls no cudaMalloc / cudaFree.  Asynchronous on cuda_stream. */
vie_status vie_matvec_static(int nx, int ny, int nz, double h, double k0, double eps_bg, const void* eps_dev,
                             const void* x_dev, void* y_dev, void* cuda_stream);

/* The autotuner's report for the plan: per tuned kernel the shape, each
 * candidate launch variant with its measured device time (ms) and the
 * choice -- the matvec's yz passes (x-columns per CTA of the register or of
 * the generic kernels) and its x pass (compile-time radix-16 kernel, the
 * generic Stockham kernel with one of three radix orders, or the kernel split
 * over a cluster of CTAs, per precision), timed at plan
 * creation, and each box's kept-block product (1, 2, 4 or 8 CTAs per
 * block) and tensor-core representative-block product (N tile of 64 or 32
 * columns), timed at preconditioner build.  Choices are cached per process and
 * shape; VIE_AUTOTUNE=0 in the environment keeps the default rules, and a
 * file named by VIE_TUNE_FILE keeps the choices across processes (read at
 * the first lookup, appended to by each new choice).  The
 * string belongs to the plan (valid until it is destroyed or rebuilt). */
const char* vie_plan_tuning(vie_plan_t plan);

/* Test hook: override one of the autotuner's choices for this plan.  kernel
 * "x_pass_c64" / "x_pass_c128" with choice -1 (default rule), 0 (three-pass
 * compile-time kernel, complex FP32, L = 2048 or 4096), 1..3 (generic
 * Stockham kernel with radix order 1..3), 4 (four-pass compile-time kernel,
 * complex FP32, L = 4096 or 8192) or 5, 6, 7 (complex FP32: the x pass split
 * over a cluster of 2, 4 or 8 CTAs, for embeddings whose three lines do not
 * fit one CTA's shared memory; at least the smallest split that fits); "yz_passes_c64" with 16, 8 or 4 x-columns
 * per CTA of the register yz passes; "yz_generic_c64" with 1, 2, 4, 8 or 16
 * x-columns per CTA of the generic yz passes (as shared memory allows);
 * "block_gemv" with 1, 2, 4 or 8 CTAs per kept block, "rep_gemm_tc" with
 * an N tile of 64 or 32 columns for the complex-FP32 representative-block
 * product (both set on the built preconditioner; a rebuild tunes again).  VIE_EINVAL for a variant that
 * does not exist for the plan's shape. */
vie_status vie_plan_set_tuning(vie_plan_t plan, const char* kernel, int choice);

/* Message of the last error on the calling thread ("" if none). */
const char* vie_last_error(void);

/* Number of kernels this library has launched in this process (all plans);
 * used to report launch counts.  Launches inside a replayed CUDA graph are
 * counted once per replay and kernel. */
int64_t vie_kernel_launches(void);

/* Per-kernel device timing, a benchmark and test hook.  While enabled
 * (on != 0), solves launch their Arnoldi steps eagerly instead of through a
 * CUDA graph and every library kernel launch is bracketed by two CUDA events
 * on its stream.  vie_profile_query sums, for one kernel name (e.g. "mv_x",
 * "block_lu", "arnoldi_update"), the launches recorded since the last
 * vie_profile_reset and their total device time in ms (it synchronises on
 * the recorded events).  vie_profile_kernels writes up to cap distinct
 * recorded names into names (static strings) and returns how many exist. */
void vie_profile_enable(int on);
void vie_profile_reset(void);
vie_status vie_profile_query(const char* kernel, int64_t* launches, double* total_ms);
int vie_profile_kernels(const char** names, int cap);

#ifdef __cplusplus
}
#endif

#endif /* LIBVIE_VIE_H */
