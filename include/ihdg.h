/*
 * libihdg -- the element-parallel iHDG sweep on one GB300 (sm_103a), behind a C ABI.
 *
 * The method (Muralikrishnan, Tran, Bui-Thanh, "iHDG: An Iterative HDG Framework for
 * Partial Differential Equations"):
 *   * Section 2, Eqs. (HDGlocal), (HDGeqn), (RiemannFluxBoth): upwind HDG for
 *     sum_k d_k(A_k u) + C u = f on a mesh of elements K with skeleton E_h.
 *   * Section 2, Eqs. (iHDGlocal), (iHDGtrace), Algorithm 1: the iteration.  Every element
 *     solves its local equation with the weighted trace of iterate k, independently of all
 *     others; the weighted trace of iterate k+1 is then formed face by face; the loop stops
 *     when ||u^{k+1} - u^k||_{L2} < tol (Section 5.1, Eq. (tolerancecriteriarelerror)).
 *   * Section 3: scalar transport (Eqs. transportLocalk1, transportLocale) and linearized
 *     shallow water with backward Euler (Eq. localSolverDD and the trace formula below it).
 *   * Section 4.1: convection-diffusion in first-order form (Eqs. ErrorDDMCD1, ErrorDDMCD2,
 *     the flux general_flux_convdiff with gamma = 1, alpha = sqrt((beta.n)^2 + 4)).
 *
 * Discretisation choices where the paper is silent: uniform box meshes of congruent
 * elements; tensor-product Q^p (p = 1..4) with a Gauss-Lobatto-Legendre (GLL) nodal basis;
 * Gauss-Legendre quadrature with q = p+2 points per direction for the forcing and the
 * boundary data; Dirichlet traces are the L2 projection of g onto each boundary face.
 *
 * Conventions used by every call:
 *   * Elements are numbered lexicographically, x index fastest.  Inside an element, nodes
 *     (GLL, (p+1)^d) and quadrature points (Gauss, q^d) are lexicographic, x fastest.
 *   * Faces: all x-normal faces first (i + (nx+1)*(j + ny*k)), then y-normal
 *     (i + nx*(j + (ny+1)*k)), then z-normal (i + nx*(j + ny*k)).  Points on a face are
 *     lexicographic over the tangential axes in increasing axis order.  Boundary faces are
 *     numbered in global face order.
 *   * Volume components: transport (u); convection-diffusion (sigma_1..sigma_d, u);
 *     shallow water (phi, u, v).  One scalar trace per face node: u_hat, u_hat, phi_hat.
 *   * Host pointers are owned by the caller, read during the call only, and outputs are
 *     written only when the returned status is IHDG_OK, IHDG_NOT_CONVERGED or
 *     IHDG_DIVERGED.  A context is not thread-safe: use one per thread.
 *   * Every call returns a status; ihdg_last_error() gives a one-line reason.
 *   * No call falls back to the CPU.  Without a usable GPU, ihdg_create() fails with
 *     IHDG_ERR_CUDA.
 */
#ifndef IHDG_H
#define IHDG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IHDG_OK = 0,
  IHDG_ERR_INVALID = 1,      /* bad argument: null pointer, size, coefficient */
  IHDG_ERR_NOMEM = 2,        /* workspace too small or device allocation failed */
  IHDG_ERR_CUDA = 3,         /* a CUDA call failed; see ihdg_last_error() */
  IHDG_NOT_CONVERGED = 4,    /* max_iters sweeps ran without meeting tol (outputs valid) */
  IHDG_DIVERGED = 5,         /* residual non-finite or grew by diverge_factor (outputs valid) */
  IHDG_ERR_BUSY = 6,         /* serving: request not finished / no room admitted */
  IHDG_ERR_TIMEOUT = 7,      /* a bounded device wait ran out; the context stays usable */
  IHDG_ERR_UNSUPPORTED = 8   /* (pde, dim, p, precision) combination not built */
} ihdg_status;

typedef enum { IHDG_TRANSPORT = 0, IHDG_CONVDIFF = 1, IHDG_SWE = 2 } ihdg_pde;

/* Numerical flux of the transport equation (Section 3).  IHDG_FLUX_UPWIND: the upwind HDG
 * flux, tau = |beta.n| with the weighted trace of Eq. transportLocale.  IHDG_FLUX_NPC: the
 * flux of Eq. Ntaub, tau = |beta.n|(1 + sgn(beta.n))/2 - beta.n (0 on outflow faces), no
 * weight on the trace; the iteration then terminates after as many sweeps as there are
 * element layers along the flow (Theorem iHDG-NPC).  Both make the trace the upwind value and
 * have the same fixed point.  Convection-diffusion and shallow water take only the upwind
 * flux (the paper gives NPC's tau for transport only). */
typedef enum { IHDG_FLUX_UPWIND = 0, IHDG_FLUX_NPC = 1 } ihdg_flux;

/* Time rule of the shallow-water steps.  BACKWARD_EULER: the local problem of Section 3 (Eq.
 * localSolverDD) with M/dt.  CRANK_NICOLSON: the rule of the paper's shallow-water experiments
 * (Section 5, linearized shallow water): (M/dt)(q^{m+1} - q^m) = -(N(q^{m+1}) + N(q^m))/2, N
 * the HDG spatial residual.  The system is linear and autonomous, so the step is computed as
 * q^{m+1} = 2 q^{m+1/2} - q^m with q^{m+1/2} the backward-Euler step of size dt/2, iterated
 * from q^m to tolerance tol/2: its iterates map one to one onto the Crank-Nicolson iterates
 * (k-th iterate 2 q^{m+1/2,k} - q^m, increments twice as large), so the iteration count and
 * the stopping decision are the Crank-Nicolson iteration's.  Other PDEs: must be 0. */
typedef enum { IHDG_BACKWARD_EULER = 0, IHDG_CRANK_NICOLSON = 1 } ihdg_time_scheme;

/* Arithmetic of the sweep.  FP64: every step in float64.  MIXED_*: defect correction --
 * float64 outer sweeps form the residual r = S(E) - E and its float64 norm; inner sweeps on
 * the correction equation e = r + G(e) run in float32 (CUDA cores), TF32 or BF16 (tcgen05
 * tensor cores, float32 accumulation); E += e; repeat until the float64 norm < tol. */
typedef enum {
  IHDG_FP64 = 0,
  IHDG_MIXED_FP32 = 1,
  IHDG_MIXED_TF32 = 2,
  IHDG_MIXED_BF16 = 3
} ihdg_precision;

/* Inner-sweep kernel of the mixed path.  AUTO: tensor cores for bf16, tf32 and 3D float32,
 * the CUDA-core kernel for 2D float32, temporally blocked (opts.sweeps_per_sync) -- or what
 * ihdg_autotune chose for the problem on this context.  TENSOR_CORES: tcgen05 local apply wherever the element shape
 * fits (n_in <= 64, n_exp <= 32), else the CUDA-core kernels.  CUDA_CORES: register- or
 * shared-memory-resident state.  GLOBAL: global-memory state (any size). */
typedef enum {
  IHDG_KERNEL_AUTO = 0,
  IHDG_KERNEL_TENSOR_CORES = 1,
  IHDG_KERNEL_CUDA_CORES = 2,
  IHDG_KERNEL_GLOBAL = 3
} ihdg_inner_kernel;

/* Uniform box mesh of n[0] x n[1] (x n[2]) congruent elements on [lo, hi], order p. */
typedef struct {
  int dim;          /* 2 or 3 (shallow water: 2) */
  int n[3];         /* elements per direction, >= 1 (n[2] ignored when dim = 2) */
  double lo[3], hi[3];
  int p;            /* polynomial order, 1..4 */
} ihdg_mesh;

typedef struct {
  ihdg_pde pde;
  double beta[3];       /* transport / convection-diffusion velocity (constant) */
  double kappa;         /* convection-diffusion diffusivity, > 0 */
  double nu;            /* reaction nu (u, v)_K in the local equation, >= 0 (transport and
                           convection-diffusion).  A backward-Euler step of the time-dependent
                           equation is a solve with nu + 1/dt and the forcing f + u^m/dt, warm-
                           started from u^m (opts.u0): the remarks on time-dependent transport
                           (after Theorem 1) and convection-diffusion (Section 4.1) */
  double Phi;           /* shallow water mean geopotential, > 0 */
  double coriolis_f;    /* shallow water Coriolis parameter (constant) */
  double friction;      /* shallow water bottom friction gamma >= 0 */
  double dt;            /* shallow water backward-Euler step, > 0 */
  ihdg_flux flux;       /* transport: IHDG_FLUX_UPWIND (0, the default) or IHDG_FLUX_NPC;
                           other PDEs: must be IHDG_FLUX_UPWIND (else IHDG_ERR_UNSUPPORTED) */
  double tau_gamma;     /* convection-diffusion stabilisation: 0 = the upwind tau^+- =
                           (alpha - beta.n^+-)/2 (the default); > 0 = the mesh-dependent
                           tau = tau_gamma (p+1)(p+2)/h on both sides of every face, h the
                           element size along the face normal, which the paper takes for the
                           diffusion-dominated limit (Section 4.2); other PDEs: must be 0 */
  ihdg_time_scheme time_scheme;   /* shallow water: BACKWARD_EULER (0, the default) or
                                     CRANK_NICOLSON; other PDEs: must be 0 (else
                                     IHDG_ERR_UNSUPPORTED) */
} ihdg_coeffs;

typedef struct {
  double tol;              /* stop when ||u^k - u^{k-1}||_{L2} < tol (absolute) */
  int max_iters;           /* sweep budget (default 2000 when <= 0) */
  ihdg_precision prec;
  double diverge_factor;   /* DIVERGED when residual > factor * its running minimum;
                              <= 0 disables the check (default 1e6 when == 0) */
  int inner_max;           /* mixed: inner sweeps per outer step cap (0 = automatic: 400;
                              32 for shallow-water steps, whose warm-started inner loops
                              stall above their stopping ratio) */
  double inner_rtol;       /* mixed: inner stop when step norm <= inner_rtol * ||r||
                              (0 = auto: 2e-3 float32, 1e-2 tf32, 0.2 bf16, or the autotuned value) */
  const double* u0;        /* optional initial guess, volume layout (host for ihdg_solve,
                              device for ihdg_solve_device); NULL = zero */
  int profile;             /* 1: time every sweep launch with CUDA events (one launch per
                              host check, so slower overall) and report the averages below */
  ihdg_inner_kernel inner_kernel;   /* mixed: inner-sweep kernel (AUTO = 0) */
  int sweeps_per_sync;     /* mixed, 2D CUDA-core inner kernel: inner sweeps between two grid
                              barriers.  1: one barrier per sweep (register-resident kernel);
                              H >= 2: temporal blocking, every block sweeps its tile plus a halo
                              of H elements H times in shared memory (the same iterates; halo
                              work recomputed); 0: automatic (the autotuned value, else 4) */
  int tile_shape;          /* mixed, temporally blocked 2D kernel: which tile shape, counted
                              in order of increasing tile + halo area over at most one tile per
                              SM (1: the smallest area, the automatic rule; 2, 3, ...: the
                              next ones; past the last: the last); 0: automatic (the autotuned
                              value, else 1) */
  int krylov_restart;      /* 0: Algorithm 1 (the plain iteration).  m >= 1: GMRES(m) on the
                              fixed-point system (I - T) E = F of one float64 sweep E -> T E + F
                              (the iHDG sweep as preconditioner, Section 4.2, closing remark):
                              restarted every m steps, at most max_iters steps in all (one
                              homogeneous sweep each); tol bounds the residual relative to the
                              initial one, ||F - (I - T) E||_2 <= tol ||F - (I - T) E^0||_2, in
                              the export space.  float64 only (prec must be IHDG_FP64), m <= 4096;
                              the workspace grows by (m + 1) export vectors.  result.residual is
                              the true relative residual of the returned solution.  Taken by
                              ihdg_solve*, ihdg_swe_steps*; the grouped, served and
                              variable-coefficient calls return IHDG_ERR_UNSUPPORTED. */
} ihdg_options;

typedef struct {
  int iterations;          /* sweeps executed (plain: the paper's count K; mixed: all) */
  int fp64_sweeps;         /* of which float64 */
  int lowp_sweeps;         /* of which low precision */
  double residual;         /* last float64 ||u^k - u^{k-1}|| */
  ihdg_status status;
  double setup_ms;         /* host operator build + uploads (0 when cached) */
  double solve_ms;         /* device time of the sweep loop and reconstruction */
  double fp64_sweep_ms;    /* profile: mean device time of one float64 launch (plain sweep;
                              mixed: outer sweep or residual check) */
  double lowp_sweep_ms;    /* profile: device time of the persistent low-precision inner
                              loop per sweep it ran */
  int fp64_launches;       /* profile: float64 sweep launches timed */
  int lowp_launches;       /* profile: low-precision sweep launches timed */
  int kernel_launches;     /* CUDA kernels this call launched (including sweeps that found
                              the loop already stopped and returned at once) */
  double latency_ms;       /* serving: submit -> results on the host */
  double queue_ms;         /* serving: submit -> admitted to a slot */
  int inner_kernel_used;   /* mixed: the kernel that ran the inner sweeps (0 none or not
                              recorded, 1 tensor cores k_inner_tc, 2 temporally blocked
                              k_inner_blk, 3 register-resident k_inner_reg, 4 shared-memory
                              tile k_inner_tile, 5 global state k_inner_persist, 6 tensor
                              cores with TMA-staged gathers k_inner_tcs) */
} ihdg_result;

typedef struct {
  long long n_el;          /* elements */
  int nvol;                /* volume values per element = ncomp * (p+1)^dim */
  int ncomp;               /* volume components */
  int nqv;                 /* forcing values per element (q^dim, q = p+2); 0 for SWE */
  long long n_bface;       /* boundary faces */
  int nqf;                 /* boundary values per boundary face (q^(dim-1)); 0 for SWE */
  long long n_face;        /* all faces */
  int nface_nodes;         /* trace values per face ((p+1)^(dim-1)) */
  int n_exp;               /* exported trace values per element (device state) */
  int n_in;                /* gathered trace inputs per element */
} ihdg_sizes;

typedef struct ihdg_ctx ihdg_ctx;

/* Create a context bound to CUDA device `device`.  Fails with IHDG_ERR_CUDA when no such
 * device exists or it is not sm_103.  *out receives the context (caller destroys it).
 * No counterpart in the paper: the context holds device state (operator images, scratch,
 * the pinned loop-state readback) across calls.  ihdg_destroy frees it; NULL is ignored. */
ihdg_status ihdg_create(ihdg_ctx** out, int device);
void ihdg_destroy(ihdg_ctx* ctx);
/* One-line description of the last failure on this context ("" when none).  Never NULL.
 * No counterpart in the paper (error reporting of this library). */
const char* ihdg_last_error(const ihdg_ctx* ctx);

/* Sizes of every array for this problem (host-only; validates mesh and coefficients).  The
 * spaces are those of Section 2 (volume space V_h, trace space M_h on the skeleton) with the
 * Q^p / GLL reading given at the top of this file; n_exp and n_in describe this library's
 * export-state form of the local solve (Section 2, Eq. iHDGlocal). */
ihdg_status ihdg_problem_sizes(const ihdg_mesh* mesh, const ihdg_coeffs* coeffs, ihdg_sizes* out);

/* Physical coordinates of the quadrature points where the caller samples f and g
 * (host-only; the paper does not fix the rule: Gauss-Legendre, p+2 points per direction).  vol_xyz: [n_el][nqv][dim]; bnd_xyz: [n_bface][nqf][dim]; either may be
 * NULL.  The library samples nothing itself: the forcing and boundary data are inputs. */
ihdg_status ihdg_quadrature_points(const ihdg_mesh* mesh, double* vol_xyz, double* bnd_xyz);

/* Physical coordinates of the GLL nodes, [n_el][(p+1)^dim][dim] (host-only): where the
 * volume solution of every solve is reported (the nodal basis of V_h, Section 2). */
ihdg_status ihdg_node_points(const ihdg_mesh* mesh, double* xyz);

/* Steady solve (transport, convection-diffusion) by the iHDG iteration, host buffers:
 * Algorithm 1 (Section 2, Eqs. iHDGlocal and iHDGtrace) on the equations of Section 3
 * (transport) or Section 4.1 (convection-diffusion), stopped by the test of Section 5.1.
 *   f_qp      [n_el][nqv]        forcing f at the quadrature points
 *   g_qp      [n_bface][nqf]     Dirichlet / inflow data g at boundary quadrature points
 *                                (transport reads it on inflow faces only)
 *   u_out     [n_el][nvol]       volume solution u^K at the GLL nodes
 *   trace_out [n_face][nface_nodes] trace u_hat^K at the face GLL nodes (NULL = skip)
 * Copies inputs to the device, runs, copies outputs back (all inside the call). */
ihdg_status ihdg_solve(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                       const double* f_qp, const double* g_qp, const ihdg_options* opts,
                       double* u_out, double* trace_out, ihdg_result* res);

/* Device workspace the device-pointer calls need for this problem and precision.  No
 * counterpart in the paper (memory sizing of ihdg_solve_device / ihdg_swe_steps_device). */
ihdg_status ihdg_workspace_bytes(const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                                 const ihdg_options* opts, size_t* bytes);

/* As ihdg_solve (Algorithm 1, same citations), but every array (including opts->u0) is
 * DEVICE memory of the context's
 * device, workspace is caller-allocated device memory of at least ihdg_workspace_bytes(),
 * 256-byte aligned, and all work is ordered on `stream` (a cudaStream_t; NULL = legacy
 * default stream).  Returns after the solve has finished on the device. */
ihdg_status ihdg_solve_device(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                              const double* d_f_qp, const double* d_g_qp,
                              const ihdg_options* opts, double* d_u_out, double* d_trace_out,
                              void* d_workspace, size_t workspace_bytes, void* stream,
                              ihdg_result* res);

/* As ihdg_solve_device, for callers that cannot allocate device memory: code embedded in
 * a host application whose allocator owns all of the GPU's memory, or in a pipeline where a
 * cudaMalloc/cudaFree (which synchronise the device) is not allowed.  The paper has no
 * counterpart: this is a deployment variant of the same solve.  It allocates nothing: the
 * operator image and the whole solve workspace live in one file-scope device array of
 * IHDG_STATIC_SCRATCH_BYTES that every GPU which loads the library holds until exit.  The
 * caller passes inputs and outputs (device memory, as for ihdg_solve_device).  Problems
 * whose scratch exceeds the array fail with IHDG_ERR_NOMEM and a message giving the size.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array and it keeps
 * the last call's contents: calls whose GPU work overlaps (other streams or host threads)
 * race, so serialise them. */
#define IHDG_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
ihdg_status ihdg_solve_device_static(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                                     const double* d_f_qp, const double* d_g_qp,
                                     const ihdg_options* opts, double* d_u_out, double* d_trace_out,
                                     void* stream, ihdg_result* res);

/* No counterpart in the paper (it has no precision or kernel choice).
 * Autotuner of the mixed path: times complete solves of the caller's problem (host inputs as
 * for ihdg_solve) for every inner-kernel choice, a ladder of inner stopping ratios
 * (float32/tf32: 5e-4 .. 1e-2; bf16: 2e-2 .. 0.3) and, for the CUDA-core kernel on 2D
 * meshes, 1..4 sweeps per grid barrier; keeps the fastest that converges, and returns it in
 * *tuned (a copy of *opts with inner_kernel, inner_rtol and sweeps_per_sync set) with its
 * device time in *best_ms.  The choice is also cached in the context for this problem shape
 * (pde, flux, dim, n, p, precision): later solves on the context whose inner_kernel is AUTO,
 * inner_rtol 0 and sweeps_per_sync 0 use it.  Serving slots do not (their results must not depend on timing).
 * FP64 options have nothing to tune: *tuned = *opts.  Errors as for ihdg_solve; a problem
 * that converges under no candidate returns IHDG_NOT_CONVERGED. */
ihdg_status ihdg_autotune(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                          const double* f_qp, const double* g_qp, const ihdg_options* opts,
                          ihdg_options* tuned, double* best_ms);

/* Grouped float64 solves of many steady problems (no counterpart in the paper; every
 * problem's sweeps are independent, Algorithm 1, so problems can share the GPU): n problems of
 * any mesh sizes, orders and PDEs (transport, convection-diffusion; shallow water is stepped
 * by ihdg_swe_steps*) solved in one call.  Problems of one element shape (dimension, nodes per
 * face) run their whole loops in one cooperative launch as far as their blocks are
 * co-resident, each exactly as in its own launch (bitwise the result, iteration count and
 * status of ihdg_solve_device); larger ones run one by one; one readback at the end.
 * opts->prec must be IHDG_FP64 (else IHDG_ERR_UNSUPPORTED) and opts->u0 NULL (zero initial
 * guess).  d_f[i], d_g[i]: device forcing and boundary data of problem i (layouts of
 * ihdg_solve); d_u[i]: device volume output [n_el][nvol]; d_tr: NULL, or per problem a device
 * trace output or NULL.  d_workspace: 256-byte aligned device memory of at least
 * ihdg_group_workspace_bytes(), owned by the caller.  res: n results (or NULL).  Errors as for
 * ihdg_solve_device; host arrays are read during the call only. */
ihdg_status ihdg_group_workspace_bytes(int n, const ihdg_mesh* meshes, const ihdg_coeffs* coeffs,
                                       const ihdg_options* opts, size_t* bytes);
ihdg_status ihdg_solve_group_device(ihdg_ctx* ctx, int n, const ihdg_mesh* meshes, const ihdg_coeffs* coeffs,
                                    const double* const* d_f, const double* const* d_g, const ihdg_options* opts,
                                    double* const* d_u, double* const* d_tr, void* d_workspace,
                                    size_t workspace_bytes, void* stream, ihdg_result* res);

/* Linearized shallow water (Section 3, Eq. localSolverDD), walls on the whole boundary:
 * advance q (in/out, [n_el][3][(p+1)^2] volume layout (phi, u, v), host) by nsteps steps of
 * coeffs->dt with coeffs->time_scheme (backward Euler, or the Crank-Nicolson rule of the
 * paper's shallow-water experiments, Section 5); each step runs the iHDG iteration
 * warm-started from the previous step.  iters_per_step (host, length nsteps) may be NULL.
 * res reports the totals and the status of the worst step. */
ihdg_status ihdg_swe_steps(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                           double* q_inout, int nsteps, const ihdg_options* opts,
                           int* iters_per_step, ihdg_result* res);

/* Device-pointer form of ihdg_swe_steps (Section 3, Eq. localSolverDD; the same steps):
 * q is device memory; iters_per_step stays a host array. */
ihdg_status ihdg_swe_steps_device(ihdg_ctx* ctx, const ihdg_mesh* mesh,
                                  const ihdg_coeffs* coeffs, double* d_q_inout, int nsteps,
                                  const ihdg_options* opts, int* iters_per_step,
                                  void* d_workspace, size_t workspace_bytes, void* stream,
                                  ihdg_result* res);

/* Host-only inspection of the float64 per-element operators this library builds for a
 * problem (no device needed), i.e. the precomputed local solve of Section 2, Eq. iHDGlocal:
 * which = 0 L_E (n_exp x n_in), 1 Q (n_in x n_in), 2 L_vol (nvol x n_in), 3 R (n_exp x
 * nvol), 4 forcing-to-export (n_exp x nqv), 5 forcing-to-volume (nvol x nqv).  Row-major
 * into data (may be NULL to query rows/cols only). */
ihdg_status ihdg_host_operator(const ihdg_mesh* mesh, const ihdg_coeffs* coeffs, int which,
                               int* rows, int* cols, double* data);

/* Serving: continuous batching of independent steady solves (transport or
 * convection-diffusion) on one GPU.  ihdg_server_start allocates one device arena of
 * hbm_budget_bytes and starts `slots` worker threads, each with its own CUDA stream.
 * ihdg_submit copies the request's inputs (host arrays as for ihdg_solve), prepares its
 * operators on the calling thread, and queues it; it fails with IHDG_ERR_NOMEM when the
 * request's footprint (operators, workspace, inputs, outputs) exceeds the whole budget.  A
 * free slot admits the first queued request whose footprint fits in the arena's free space,
 * so requests arriving while others run start as soon as a slot and memory free up, and the
 * slots' GPU work overlaps.  Traces and all solve state stay on the device until the slot
 * copies u and the trace back.  ihdg_poll returns IHDG_ERR_BUSY until the request is done,
 * then its result (status, sweeps, latency_ms from submit to completion, queue_ms);
 * ihdg_fetch copies u (and the trace unless NULL) and releases the ticket.  A request's
 * launch configuration depends only on its own size, so its result is the same alone and in
 * any mix.  The paper solves one problem at a time; this is a deployment interface around
 * the same solve.  ihdg_server_stop waits for running requests and frees the arena. */
typedef long long ihdg_ticket;
ihdg_status ihdg_server_start(ihdg_ctx* ctx, size_t hbm_budget_bytes, int slots);
ihdg_status ihdg_server_stop(ihdg_ctx* ctx);
ihdg_status ihdg_submit(ihdg_ctx* ctx, const ihdg_mesh* mesh, const ihdg_coeffs* coeffs,
                        const double* f_qp, const double* g_qp, const ihdg_options* opts,
                        ihdg_ticket* out);
ihdg_status ihdg_poll(ihdg_ctx* ctx, ihdg_ticket ticket, ihdg_result* res);
ihdg_status ihdg_fetch(ihdg_ctx* ctx, ihdg_ticket ticket, double* u_out, double* trace_out);

/* Transport with a velocity field that varies in space (Section 3: beta.grad u = f with beta
 * continuous across the skeleton; the paper's transport experiments of Section 5.1, Table 1,
 * use such fields).  Every element has its own local matrix A_K, so the local solves of
 * Algorithm 1 are factorised once per field into a plan: float64 LU on the host (threads over
 * elements), and L_K = A_K^{-1} G_K (the trace coupling) and A_K^{-1} kept in device memory in
 * float64 with float32 and bf16 copies of L_K.  A sweep is then u_K^{k+1} = A_K^{-1} b_K +
 * L_K t_K(u^k) for every element: the device streams each element's own operator (a batched
 * GEMV), so it is bound by HBM bandwidth.  The local equation is (transportLocalk1) in its
 * integrated-by-parts form (beta.grad u, v)_K + <|beta.n| (u - u_hat^k), v>_dK = (f, v)_K
 * (equal to the printed form under exact integration; beta, not div beta, is sampled), with
 * the upwind trace of Eq. transportLocale.
 *
 * ihdg_face_quadrature_points: the Gauss points of EVERY global face (global face order),
 * [n_face][nqf][dim] (host-only), where the caller samples beta on the skeleton.
 *
 * ihdg_var_plan_create: beta_vol [n_el][nqv][dim] at the volume quadrature points of
 * ihdg_quadrature_points, beta_face [n_face][nqf][dim] at the points above (host arrays, read
 * during the call).  Each beta component must keep one sign (or vanish) over all faces
 * normal to its axis, so that each element face is an inflow or an outflow face as a whole
 * (true for the paper's fields); otherwise IHDG_ERR_UNSUPPORTED.  Built for 2D p = 1..4 and
 * 3D p = 1..2.  The plan allocates its device memory on the context's device
 * (ihdg_var_plan_info reports how much) and is freed by ihdg_var_plan_destroy.
 *
 * ihdg_var_solve: f_qp [n_el][nqv] (forcing at the volume quadrature points), g_qp
 * [n_bface][nqf] (inflow data at the boundary quadrature points, read on inflow faces only),
 * options as for ihdg_solve with prec FP64, MIXED_FP32 or MIXED_BF16 (float32 / bf16 inner
 * sweeps with float32 accumulation on the correction equation, float64 outer sweeps and
 * stopping norm) and opts->u0 an optional initial guess [n_el][(p+1)^dim]; u_out
 * [n_el][(p+1)^dim], trace_out [n_face][(p+1)^(dim-1)] (NULL = skip).  Host buffers, copies
 * inside the call.  ihdg_var_solve_device: the same with device arrays, ordered on `stream`;
 * returns after the solve has finished.  Errors as for ihdg_solve; IHDG_ERR_INVALID when the
 * plan belongs to another context's device. */
typedef struct ihdg_var_plan ihdg_var_plan;
ihdg_status ihdg_face_quadrature_points(const ihdg_mesh* mesh, double* xyz);
ihdg_status ihdg_var_plan_create(ihdg_ctx* ctx, const ihdg_mesh* mesh, const double* beta_vol,
                                 const double* beta_face, ihdg_var_plan** out);
void ihdg_var_plan_destroy(ihdg_var_plan* plan);
ihdg_status ihdg_var_plan_info(const ihdg_var_plan* plan, size_t* device_bytes, double* setup_ms);
ihdg_status ihdg_var_solve(ihdg_ctx* ctx, ihdg_var_plan* plan, const double* f_qp, const double* g_qp,
                           const ihdg_options* opts, double* u_out, double* trace_out, ihdg_result* res);
ihdg_status ihdg_var_solve_device(ihdg_ctx* ctx, ihdg_var_plan* plan, const double* d_f_qp,
                                  const double* d_g_qp, const ihdg_options* opts, double* d_u_out,
                                  double* d_trace_out, void* stream, ihdg_result* res);
/* Several plans solved together (the paper solves one problem at a time; no counterpart):
 * every sweep step is one grouped launch per (dim, p) class covering all the class's plans,
 * so problems of uneven size and order share launches, and small problems that could not fill
 * the GPU alone fill it together.  Each block of a grouped launch works for one plan exactly as
 * that block of the plan's own launch would (same grid, element mapping, fixed-order
 * reductions, loop decisions), so every plan's u, trace, iteration count and status are
 * bitwise those of ihdg_var_solve_device with the same options; the plans advance through
 * their float64 / mixed phases independently and stop on their own tolerance.  n plans of
 * the context's device (1..64; distinct plans), device arrays d_f_qp[i], d_g_qp[i],
 * d_u_out[i] (and d_trace_out[i] unless d_trace_out or the entry is NULL) laid out as for
 * ihdg_var_solve_device; opts is shared (opts->u0 must be NULL); res: n results (solve_ms is
 * the whole group's device time).  Allocates a few KB of device descriptors per call.  Errors
 * as for ihdg_var_solve_device. */
ihdg_status ihdg_var_solve_group(ihdg_ctx* ctx, int n, ihdg_var_plan* const* plans,
                                 const double* const* d_f_qp, const double* const* d_g_qp,
                                 const ihdg_options* opts, double* const* d_u_out,
                                 double* const* d_trace_out, void* stream, ihdg_result* res);
/* Host-only inspection of one element's float64 local solve as the plan builds it (no device
 * needed): which = 0 L_K = A_K^{-1} G_K (nvol x n_in; column f*nf + r is face f's node r),
 * 1 A_K^{-1} (nvol x nvol).  Row-major into data (NULL: query rows/cols only). */
ihdg_status ihdg_var_host_operator(const ihdg_mesh* mesh, const double* beta_vol, const double* beta_face,
                                   long long element, int which, int* rows, int* cols, double* data);

/* Device peak rates that bound the sweep kernels where neither HBM bandwidth nor the bf16
 * tensor rate does.  No counterpart in the paper: these are roofline denominators.  Each is
 * the best of five timed launches of one probe kernel (after a warm-up launch) on `device`:
 * float64 and float32 FMA rates (8 independent FMA chains per thread, 2 flops per FMA, full
 * occupancy) and the L2 read bandwidth (ld.global.cg over a 48 MB buffer resident in L2).
 * Allocates and frees its own device memory (a few MB).  Errors: IHDG_ERR_INVALID (null
 * out), IHDG_ERR_CUDA (no such device, launch failure), IHDG_ERR_NOMEM. */
typedef struct {
  double fp64_fma_tflops;
  double fp32_fma_tflops;
  double l2_read_gbs;
  int sms;
} ihdg_peaks;
ihdg_status ihdg_measure_peaks(int device, ihdg_peaks* out);

/* Sizes in bytes of the public structs, for bindings that mirror them (no counterpart in the
 * paper): out[0..5] = sizeof(ihdg_mesh), sizeof(ihdg_coeffs), sizeof(ihdg_options),
 * sizeof(ihdg_result), sizeof(ihdg_sizes), sizeof(ihdg_peaks); the first min(n, 6) are
 * written into the caller's host array.  Host only, no device work.  IHDG_ERR_INVALID when
 * out is NULL or n < 0. */
ihdg_status ihdg_abi_sizes(size_t* out, int n);

#ifdef __cplusplus
}
#endif
#endif /* IHDG_H */
