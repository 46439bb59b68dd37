/*
 * reg.h - C ABI of the GB300 semi-Lagrangian Gauss-Newton-Krylov registration
 * library (libregnk.so).
 *
 * Method: Mang & Biros, "A semi-Lagrangian two-level preconditioned
 * Newton-Krylov solver for constrained diffeomorphic image registration"
 * (arXiv 1604.02153). The library minimises, over a stationary velocity v,
 *     J[v] = 1/2 ||m_1 - m_R||^2_L2 + beta/2 <v, A v>_L2          (eq. varopt:objective)
 * subject to the transport equation d_t m + grad m . v = 0, m(0) = m_T, with
 * periodic boundary conditions on the 2-torus [0, 2 pi)^2 (§2): compressible
 * (no divergence constraint, K = I, the default) or incompressible (div v = 0
 * with w = 0, K the Leray projection; reg_options.incompressible).
 *
 * Conventions shared by every call
 * --------------------------------
 * Grid     n1 x n2 nodes, h_i = 2 pi / n_i, node (i, j) at (i h_1, j h_2).
 *          n1, n2 are 2^k in [32, 2048] or 3 * 2^k in [96, 1536]; with the
 *          two-level preconditioner n1/2 and n2/2 must be such sizes too. (§3.2)
 * Layout   a scalar field is n1*n2 contiguous float32, row-major with x_1
 *          fastest: u[j*n1 + i]. A vector field (v, v~, g, H v~) is two
 *          scalar fields back to back (structure of arrays): component 1 at
 *          offset 0, component 2 at offset n1*n2.
 * Memory   every float pointer is a DEVICE pointer on the context's device
 *          unless its comment says "host". The caller owns all field buffers;
 *          the library copies what it keeps and never frees caller memory.
 *          Device buffers must start on a 16-byte boundary (torch
 *          allocations do); a call given one that does not returns REG_EINVAL.
 * Streams  every call runs on the stream set by reg_set_stream (default: the
 *          legacy default stream). Calls that return a host scalar or a
 *          status that depends on device data synchronise that stream;
 *          the others are asynchronous with respect to the host.
 * Errors   every call returns a reg_status. REG_EINVAL leaves the context
 *          unchanged. After REG_ECUDA or REG_ENOMEM the context must be
 *          destroyed. reg_last_error() gives a human-readable message.
 * Threads  a context is not thread-safe; use one context per host thread.
 * CPU      there is no CPU fallback: if the CUDA runtime or an sm_103a device
 *          is missing, reg_create returns REG_ECUDA.
 */
#ifndef REGNK_REG_H
#define REGNK_REG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct reg_ctx reg_ctx;

typedef enum {
  REG_OK = 0,
  REG_EINVAL = 1,       /* bad argument (size, null pointer, option value)      */
  REG_ENOMEM = 2,       /* device allocation failed                             */
  REG_ECUDA = 3,        /* CUDA runtime or kernel launch error                  */
  REG_ESTATE = 4,       /* call order violated (e.g. no images set)             */
  REG_ENOTCONV = 5,     /* reg_solve hit max_newton before the tolerance        */
  REG_ELINESEARCH = 6,  /* Armijo backtracking exhausted (§3.4.1)               */
  REG_ENEGCURV = 7,     /* PCG met p^T H p <= 0 and kept the last iterate       */
  REG_ENONFINITE = 8,   /* a NaN/Inf reached a reduction                        */
  REG_ETIMEOUT = 9      /* a bounded device wait gave up                        */
} reg_status;

/* Regularisation seminorm, eq. varopt:regv / eq. diffopregv:
 * A = -Lap (H1), Lap^2 (H2), -Lap^3 (H3); spectral weights |k|^(2p). */
enum { REG_H1 = 1, REG_H2 = 2, REG_H3 = 3 };
/* Interpolation model (§3.5 "Interpolation"): C2 periodic cubic B-spline
 * (the paper's model, default) or cubic Lagrange on raw samples (variant). */
enum { REG_INTERP_SPLINE = 0, REG_INTERP_LAGRANGE = 1 };
/* Preconditioner (§3.4.2): spectral P_REG = beta A, or two-level P_2L. */
enum { REG_PC_REG = 0, REG_PC_2L = 1 };
/* Coarse solver of P_2L (§3.4.2): CHEB(k) or nested PCG(eps). */
enum { REG_PCSOLVER_CHEB = 0, REG_PCSOLVER_PCG = 1 };
/* reg_options.hessian */
enum { REG_HESSIAN_GN = 0, REG_HESSIAN_FULL = 1 };
/* reg_options.precision */
enum { REG_PRECISION_FP64 = 0, REG_PRECISION_FP32 = 1 };

typedef struct { int n1, n2; } reg_grid;

typedef struct {
  int reg_norm;            /* REG_H1 (default) | REG_H2 | REG_H3                     */
  int interp;              /* REG_INTERP_SPLINE (default) | REG_INTERP_LAGRANGE     */
  int precond;             /* REG_PC_2L (default) | REG_PC_REG                       */
  int pc_solver;           /* REG_PCSOLVER_CHEB (default) | REG_PCSOLVER_PCG         */
  int cheb_iters;          /* k of CHEB(k), default 10 (§4.2.2)                      */
  double pc_eps;           /* eps of PCG(eps), default 0.1 (§4.2.2)                  */
  double gabs;             /* absolute ||g||_inf stop, default 1e-5 (§3.4.1)         */
  int max_newton;          /* default 50                                             */
  int max_pcg;             /* outer and nested PCG iteration cap, default 100        */
  int lanczos_steps;       /* Lanczos steps for e_max, default 30 (§4.2.1)           */
  double emax_safety;      /* e_max = largest Ritz value * this, default 1.05        */
  unsigned long long lanczos_seed; /* SplitMix64 seed of the Lanczos start vector   */
  int max_backtracks;      /* Armijo halvings, default 10                            */
  double armijo_c1;        /* Armijo constant, default 1e-4                          */
  int persistent_matvec;   /* 0 (default): one launch per transport step; 1: the GN
                              data term runs as one persistent cooperative kernel   */
  int inject_barrier_timeout; /* failure injection for tests, default 0: if 1, the
                              persistent kernel's first grid barrier (or the
                              flow kernel's first tile wait, see flow_matvec)
                              waits for an arrival that never comes; every block
                              gives up after its bounded wait (~0.5 s) and the
                              call returns REG_ETIMEOUT with the context still
                              usable                                            */
  int programmatic_launch; /* 1 (default): kernels launched directly on the stream
                              carry programmatic stream serialisation, so a
                              kernel's blocks may be scheduled while its
                              predecessor finishes (each waits for the
                              predecessor's completion before touching memory:
                              results are identical); kernels inside the
                              library's CUDA graphs are plain launches either
                              way. 0: plain launches everywhere                */
  int fused_transport;     /* 1 (default): with the spline model, every transport
                              step (state, adjoint, incremental state and adjoint,
                              and the gathers of div v at Y_D and of the gradient
                              history) computes the spline coefficients it gathers
                              from inside the step kernel (a 48^2 or 64^2
                              coefficient box per 32^2 tile) whenever the
                              velocity's displacements fit the box's halo (<= 6 or
                              <= 14 cells); results are those of the separate
                              prefilter kernel up to FP32 rounding order.
                              0: always a separate prefilter kernel             */
  int coarse_nt;           /* time steps of the coarse-grid problem of P_2L; 0
                              (default): the problem's nt. §3.4.2 expects the
                              preconditioner's PDE solves to need little
                              accuracy; nt / 2 keeps the displacement per step
                              in coarse cells equal to the fine grid's         */
  int coarse_interp;       /* interpolation model of P_2L's coarse problem: -1
                              (default) the problem's model, or REG_INTERP_SPLINE
                              / REG_INTERP_LAGRANGE (cubic Lagrange needs no
                              prefilter; §3.4.2 expects the preconditioner's PDE
                              solves to need little accuracy)                  */
  int step_tile;           /* tile shape of the adjoint and incremental-state step
                              kernels where they run unfused (cubic Lagrange,
                              or displacements beyond the fused kernels' box):
                              k = 1..9 is 128 << ((k-1)/3) threads per block,
                              1 << ((k-1)%3) adjacent points per thread; 0: the
                              built-in shape (k = 5, 256 x 2); -1 (default):
                              reg_create times the nine shapes on each grid
                              level, once per grid and interpolation model in
                              the process, and keeps the fastest. Results do
                              not depend on the shape                          */
  int incompressible;      /* 0 (default): K = I in the gradient and the Hessian
                              (eq. control-elim, eq. hessian-matvec). 1: the
                              incompressible problem, div v = 0 with w = 0 (§2):
                              K = the Leray projection -grad Lap^-1 div + I of
                              §3.1, applied spectrally (the derivative
                              wavenumbers of REG_SPEC_GRAD/DIV, identity where
                              |k| = 0); reg_solve and reg_warm_start project
                              the velocity onto divergence-free fields first,
                              and P_2L's coarse operator and Lanczos start
                              vector carry K as well                          */
  int hessian;             /* REG_HESSIAN_GN (default): the Gauss-Newton matvec
                              (every lambda term of eq. hessian-matvec and
                              eq. inc-adj-pde-elim dropped, §3.4.1 footnote).
                              REG_HESSIAN_FULL: eq. hessian-matvec as written,
                              K[int lambda~ grad m + lambda grad m~ dt] with the
                              div(lambda v~) source in the incremental adjoint;
                              the gradient then keeps the adjoint history
                              (nt+1 fields) and the matvec needs it at the same
                              velocity (recomputed if missing). Problem grid
                              only: P_2L's coarse operator stays Gauss-Newton.
                              The full Hessian may be indefinite: PCG stops at
                              negative curvature (REG_ENEGCURV in kkt_solve).
                              Needs persistent_matvec = 0                     */
  int precision;           /* accumulation of inner products, squared norms and
                              the objective: REG_PRECISION_FP64 (default):
                              error-free FP32 products and sums per thread,
                              FP64 across threads (FP64 accuracy, bitwise
                              reproducible); REG_PRECISION_FP32: plain FP32 at
                              every level (the "plain FP32" comparison form;
                              the Armijo test and the Krylov scalars then carry
                              FP32 rounding). Fields are FP32 either way       */
  int use_graphs;          /* 1 (default): fixed launch sequences (the fine
                              matvec inside PCG, P_2L with CHEB) are replayed
                              as CUDA graphs after their first two calls;
                              0: every launch is issued from the host. Results
                              are identical                                    */
  int flow_matvec;         /* 1: on a grid level with the cubic
                              Lagrange model and nt >= 2 whose 32 x 16 point
                              tiles all fit the GPU at once (e.g. the 512^2
                              coarse grid of P_2L), the GN data term of a matvec
                              (eq. inc-state-slm forward, eq. inc-adj-slm
                              backward, int lambda~ grad m dt) is one launch:
                              each block keeps its tile for all 2 nt steps and
                              waits only for the neighbouring tiles its
                              stencils reach (bounded waits: REG_ETIMEOUT after
                              ~0.5 s, context usable). Results are bitwise those
                              of the per-step kernels. 0 (default): one launch
                              per step (faster on this GPU: 78 against 130 us
                              per 512^2 matvec, nt = 4). Ignored with
                              persistent_matvec = 1. Two contexts
                              whose flow kernels can run at the same time on
                              one GPU (different streams) must not both use it:
                              each launch needs all its blocks resident, so
                              their waits could run out (reg_batch_create
                              turns it off for its problems)                 */
  double beta_w;           /* 0 (default): no mass source. > 0: the near-
                              incompressible problem of §2: the mass source
                              w = div v (eq. icconstraint) carries the H1 norm
                              of eq. varopt:regw with weight beta_w, so J adds
                              beta_w/2 ||div v||^2_H1. Eliminating w and its
                              multiplier p from the control equations
                              (Appendix A, eq. control-v, eq. control-w:
                              p = -beta_w (I - Lap) w) gives the reduced
                              gradient g = beta A v + K[b] and Hessian
                              beta A v~ + K[b~] of eq. control-elim and
                              eq. hessian-matvec with K = beta A M^-1,
                              M = beta A - beta_w grad (I - Lap) div: per
                              wavenumber I - c kd kd^T/|kd|^2 with
                              c = beta_w (1+|k|^2)|kd|^2 / (beta |k|^2p +
                              beta_w (1+|k|^2)|kd|^2) in [0, 1) (kd the
                              derivative wavenumbers), a bounded 2 -> 2
                              multiplier like the Leray projection it tends to
                              as beta_w grows. P_REG and P_2L keep beta A (the
                              coarse operator carries K). Not with
                              incompressible = 1; reg_set_beta changes beta
                              only                                            */
  int graph_pdl;           /* launches captured into the library's CUDA graphs:
                              0 (default) plain kernel-to-kernel edges; 1 the
                              coarse grid's launches carry programmatic stream
                              serialisation (see programmatic_launch), so a
                              kernel's blocks are scheduled while its
                              predecessor drains; 2 every launch does. Results
                              are identical                                   */
} reg_options;

typedef struct {
  int newton_iters;        /* accepted Newton steps                                  */
  int pcg_iters;           /* outer PCG iterations, summed                           */
  int matvecs;             /* fine-grid GN Hessian matvecs                           */
  int coarse_matvecs;      /* coarse-grid GN data-term matvecs inside P_2L           */
  int line_search_steps;   /* objective evaluations in Armijo backtracking           */
  double J0, J;            /* objective at the initial guess and at the result       */
  double gnorm_rel;        /* ||g||_inf / ||g_ref||_inf at the result                */
  double gnorm_inf;        /* ||g||_inf at the result                                */
  double gref_inf;         /* ||g(v = 0)||_inf, the reference of the relative test   */
  double seconds;          /* host wall time of the call                             */
  int status;              /* reg_status of the solve                                */
} reg_info;

/* Fills *opt with the defaults listed above. */
reg_status reg_default_options(reg_options* opt);

/* Creates a context for one registration problem on `grid` with nt
 * semi-Lagrangian time steps (h_t = 1/nt, §3.2) and regularisation weight
 * beta > 0, on the current CUDA device. opt may be NULL (defaults). The
 * context allocates its workspace (fields, time histories, FFT buffers, the
 * coarse grid of P_2L) on the device; *out receives the handle. */
reg_status reg_create(reg_grid grid, int nt, double beta, const reg_options* opt,
                      reg_ctx** out);

/* Frees the context and its device workspace. NULL is accepted. */
reg_status reg_destroy(reg_ctx* ctx);

/* Sets the cudaStream_t (passed as void*) that later calls run on. */
reg_status reg_set_stream(reg_ctx* ctx, void* cuda_stream);

/* Copies the reference image m_R and the template image m_T (n1*n2 floats
 * each, device) into the context (eq. varopt:objective). Invalidates every
 * cached velocity-dependent quantity. */
reg_status reg_set_images(reg_ctx* ctx, const float* m_R, const float* m_T);

/* Changes beta (continuation). Chebyshev bounds are rescaled as
 * (e - 1) * beta_old / beta_new, not recomputed (§3.4.2, §4.2.1). */
reg_status reg_set_beta(reg_ctx* ctx, double beta);

/* Semi-Lagrangian state solve (eq. state-pde-elim, §3.3.2): transports m0
 * (n1*n2, device) by the stationary velocity v (2*n1*n2, device) from t = 0
 * to t = 1 and writes m(1) to m1 (n1*n2, device). RK2 characteristic, cubic
 * interpolation. Needs no images. */
reg_status reg_transport(reg_ctx* ctx, const float* v, const float* m0, float* m1);

/* Deformation map of the velocity v (§2: m_1 = m_T o y, computed from v in
 * a post-processing step): u = y - x (2*n1*n2 floats, physical units,
 * component 1 then 2), the composition of the nt semi-Lagrangian departure
 * maps of the context (u_j = u_{j-1}(X_D) + X_D - x, interpolation model of
 * the context), and, if det is not NULL, det grad y = (1 + d1 u1)(1 + d2 u2)
 * - d2 u1 d1 u2 with spectral derivatives (n1*n2 floats; the quantity that
 * §4 bounds when choosing beta, 1 for divergence-free v). Device buffers;
 * needs no images; allocates 10*n1*n2 floats of workspace on first use. */
reg_status reg_deformation_map(reg_ctx* ctx, const float* v, float* u, float* det);

/* RK2A comparator (§3.3.1, Appendix "RK2A derivation"): the state equation
 * in antisymmetric form d_t m + 1/2 (grad m . v + div(m v) - m div v) = 0,
 * solved from m0 to m1 = m(1) with nt Heun steps and pseudospectral
 * derivatives (FFT-heavy Eulerian transport, 12 FFTs per step), and its
 * adjoint -d_t lam - 1/2 (div(lam v) + grad lam . v + lam div v) = 0 from
 * lam1 = lam(1) back to lam0 = lam(0), whose Heun step is the transpose of
 * the state's. The scheme is stable only for small CFL numbers (the paper
 * uses 0.2: nt >= max|v_i| / (0.2 h_i)). All fields n1*n2 floats (v: 2*n1*n2),
 * device; needs no images; allocates 9*n1*n2 floats of workspace on first
 * use. */
reg_status reg_transport_rk2a(reg_ctx* ctx, const float* v, const float* m0, float* m1, int nt);
reg_status reg_adjoint_rk2a(reg_ctx* ctx, const float* v, const float* lam1, float* lam0, int nt);

/* Departure points of one time step (§3.3.2 "Tracing the Characteristic",
 * Heun): X_D = x - h_t/2 (v(x) + v(x - h_t v(x))) for the forward-in-time
 * equations and Y_D = x + h_t/2 (v(x) + v(x + h_t v(x))) for the backward
 * ones. Written as displacements in cell units, (X_D - x)/h, to dX and dY
 * (2*n1*n2 each, device, component 1 then 2). Either output may be NULL. */
reg_status reg_departure_points(reg_ctx* ctx, const float* v, float* dX, float* dY);

/* Periodic cubic interpolation (§3.5): out[x] = u(x + disp[x] * h), where
 * disp (2*n1*n2, device) is in cell units and u (n1*n2, device) holds
 * samples at the nodes. Uses the context's interpolation model. */
reg_status reg_interpolate(reg_ctx* ctx, const float* u, const float* disp, float* out);

/* Pseudospectral operators (§3.2, eq. diffopregv, eq. reg-precond, §3.4.2).
 * `op` selects (in -> out, sizes in fields of n1*n2 floats):
 *   REG_SPEC_GRAD     scalar -> vector   grad u (Nyquist zeroed)
 *   REG_SPEC_DIV      vector -> scalar   div v  (Nyquist zeroed)
 *   REG_SPEC_REG      vector -> vector   beta A v
 *   REG_SPEC_REGPOW   vector -> vector   (beta A)^s v, k = 0 weight -> 1 (s < 0 or s = 1/2)
 *   REG_SPEC_LOWPASS  vector -> vector   keep |k_i| < n_i/4
 *   REG_SPEC_HIGHPASS vector -> vector   remove |k_i| < n_i/4
 *   REG_SPEC_PREFILTER scalar -> scalar  periodic cubic B-spline coefficients
 *   REG_SPEC_LERAY    vector -> vector   K = -grad Lap^-1 div + I (§3.1, w = 0):
 *                                        the divergence-free part
 *   REG_SPEC_REGOP    vector -> vector   R^s for the regularisation of J: beta A, or
 *                     R = beta A - beta_w grad (I - Lap) div with
 *                     reg_options.beta_w > 0 (J = ... + 1/2 <v, R v>), k = 0
 *                     weight -> 1 unless s = 1
 *   REG_SPEC_K        vector -> vector   the context's K of eq. control-elim: identity,
 *                     Leray projection (incompressible) or the
 *                     near-incompressible K (beta_w > 0)
 * `s` is used by REG_SPEC_REGPOW and REG_SPEC_REGOP. in and out must not alias. */
enum { REG_SPEC_GRAD = 0, REG_SPEC_DIV = 1, REG_SPEC_REG = 2, REG_SPEC_REGPOW = 3,
       REG_SPEC_LOWPASS = 4, REG_SPEC_HIGHPASS = 5, REG_SPEC_PREFILTER = 6, REG_SPEC_LERAY = 7,
       REG_SPEC_REGOP = 8, REG_SPEC_K = 9 };
reg_status reg_spectral(reg_ctx* ctx, int op, double s, const float* in, float* out);

/* Spectral restriction of a vector field from the context grid to the grid
 * (n1/2, n2/2), two-level contexts only, (cut-off filter at |k_i| < n_i/4 included) and prolongation
 * back by zero padding (§3.4.2 "Restriction/Prolongation", "Filters").
 * fine: 2*n1*n2 floats, coarse: 2*(n1/2)*(n2/2) floats, device. */
reg_status reg_restrict(reg_ctx* ctx, const float* fine, float* coarse);
reg_status reg_prolong(reg_ctx* ctx, const float* coarse, float* fine);

/* Objective J (host double) and reduced gradient g = beta A v +
 * K[int_0^1 lambda grad m dt] (eq. control-elim) at v (device). g
 * (2*n1*n2, device) may be NULL. Caches the state, adjoint characteristics
 * and the time history of grad m for later Hessian matvecs at the same v.
 * Synchronises the stream (returns a host scalar). */
reg_status reg_objective_gradient(reg_ctx* ctx, const float* v, double* J, float* g);

/* Objective only (state solve plus regularisation); *J is host. */
reg_status reg_objective(reg_ctx* ctx, const float* v, double* J);

/* Gauss-Newton Hessian matvec Hvt = H(v) vt = beta A vt + K[int_0^1 lambda~ grad m dt]
 * (eq. hessian-matvec with every lambda term dropped, §3.4.1 footnote, §3.5
 * "Hessian"): incremental state solve forward, incremental adjoint solve
 * backward, all device pointers of 2*n1*n2 floats. If v differs from the
 * velocity cached by the last objective/gradient call (compared on the
 * device), the velocity-dependent cache is rebuilt first; a stale result is
 * never returned. Synchronises the stream for that comparison. */
reg_status reg_hessian_matvec(reg_ctx* ctx, const float* v, const float* vt, float* Hvt);

/* Applies the configured preconditioner inverse (P_REG^-1 or P_2L^-1,
 * §3.4.2) at the cached velocity: z = P^-1 r (2*n1*n2 floats each, device).
 * Requires a previous reg_objective_gradient. */
reg_status reg_precond_apply(reg_ctx* ctx, const float* r, float* z);

/* Solves H(v) x = rhs with PCG (§3.4.1; relative residual rtol, at most
 * maxit iterations, zero initial guess) and the configured preconditioner
 * at the velocity v. x, rhs: 2*n1*n2 floats, device. info (host) may be
 * NULL; it receives pcg_iters, matvecs, coarse_matvecs and status. */
reg_status reg_kkt_solve(reg_ctx* ctx, const float* v, const float* rhs, double rtol,
                         int maxit, float* x, reg_info* info);

/* Chebyshev bounds of P_2L's coarse split operator at v = 0 (§3.4.2
 * "Eigenvalue Estimates"): e_max from Lanczos, e_min analytic. Host doubles.
 * Computed on first use and cached; this call forces the estimate. */
reg_status reg_eigen_bounds(reg_ctx* ctx, double* emin, double* emax);

/* Inexact Gauss-Newton-Krylov solve (§3.4, §3.5): starting from v (device,
 * 2*n1*n2, overwritten with the result), iterate until
 * ||g||_inf / ||g(0)||_inf <= gtol or ||g||_inf <= gabs, PCG with forcing
 * eta_k = min(0.5, ||g_k|| / ||g(0)||), Armijo backtracking. info (host)
 * may be NULL. Returns REG_OK on convergence, REG_ENOTCONV or
 * REG_ELINESEARCH otherwise (v then holds the last accepted iterate). */
reg_status reg_solve(reg_ctx* ctx, float* v, double gtol, reg_info* info);

/* ---- Batches of independent problems --------------------------------------
 * B problems, each with its own grid (any grid reg_create accepts), nt,
 * beta[i] and the shared options, solved concurrently: every problem gets
 * its own context and CUDA stream (non-blocking, created by the batch), and
 * a pool of host threads drives the solves, so that the small kernels of
 * different problems overlap on the GPU. Each problem's result equals a
 * solve of that problem alone. Arrays of pointers are host arrays of B
 * device pointers with the per-problem layout of the single-problem calls.
 * The calls use the current CUDA device of the creating thread. */
typedef struct reg_batch reg_batch;
reg_status reg_batch_create(const reg_grid* grids, int B, int nt, const double* beta,
                            const reg_options* opt, reg_batch** out);
reg_status reg_batch_destroy(reg_batch* batch);
/* Copies every problem's images (synchronises the batch's streams). */
reg_status reg_batch_set_images(reg_batch* batch, const float* const* m_R,
                                const float* const* m_T);
/* Changes beta of every problem (beta: host array of B values). */
reg_status reg_batch_set_beta(reg_batch* batch, const double* beta);
/* reg_solve on every problem with up to `threads` host threads (<= 0: half
 * the host's hardware threads). v[i] is the initial guess and receives the result. infos (host, B
 * entries) may be NULL. Returns REG_OK if every problem converged, else the
 * first hard error, or REG_ENOTCONV / REG_ELINESEARCH if those were the only
 * failures (see infos[i].status). */
reg_status reg_batch_solve(reg_batch* batch, float* const* v, double gtol, int threads,
                           reg_info* infos);
/* reg_hessian_matvec on every problem (synchronises on return). */
reg_status reg_batch_hessian_matvec(reg_batch* batch, const float* const* v,
                                    const float* const* vt, float* const* Hvt);
const char* reg_batch_last_error(const reg_batch* batch);

/* ---- 3D grids ------------------------------------------------------------
 * The registration problem on an n1 x n2 x n3 periodic grid (d = 3 in the
 * formulation of §2-§3; the paper's experiments are 2D and name 3D as the
 * next step): RK2 departure points, periodic tricubic interpolation (cubic
 * B-spline with a separable recursive prefilter, or cubic Lagrange), the
 * semi-Lagrangian state, adjoint, incremental state and Gauss-Newton
 * incremental adjoint steps of §3.3.2, pseudospectral grad, div and
 * (beta A)^s by 3D FFTs, J (eq. varopt:objective), the reduced gradient
 * (eq. control-elim, K = I) and the GN Hessian matvec (eq. hessian-matvec).
 * Fields are float32 with x_1 fastest, then x_2, then x_3; vector fields
 * are their three components back to back (3 n1 n2 n3 floats); device
 * pointers, 16-byte aligned, owned by the caller. n_i in {32, 64, 128, 256,
 * 96, 192}. Options as reg_create: precond REG_PC_REG (the spectral
 * preconditioner) or REG_PC_2L (the two-level preconditioner of §3.4.2 with
 * CHEB(cheb_iters) or PCG(pc_eps * eta) coarse solves, eta the Newton step's
 * forcing term (0.5 outside a solve); every n_i / 2 must be a supported size,
 * the coarse problem has the same nt and interpolation model), compressible,
 * Gauss-Newton; anything else REG_EINVAL. Calls run on the stream of reg3_set_stream (default stream
 * otherwise). reg3_create allocates (74 + 7 nt) n1 n2 n3 floats of device
 * memory (6.8 GB at 256^3, nt = 4), with P_2L also a coarse-grid context
 * (one eighth of that) and 3 n1 n2 n3 floats of coarse work vectors, freed
 * by reg3_destroy. fused_transport 1
 * (default) gathers from shared-memory boxes around 32 x 8 x 8 tiles when the
 * displacements of the velocity fit one (halo ceil(max |d|) + 2 cells per
 * axis, at most 112 KB), from global memory otherwise; 0 always from global
 * memory. Both forms compute every point with the same arithmetic.
 * Errors: REG_EINVAL for a NULL or unaligned pointer or an unknown op,
 * REG_ESTATE when reg3_set_images has not been called, REG_ENOMEM or
 * REG_ECUDA from the CUDA runtime (the message in reg3_last_error); the
 * solve returns REG_ENOTCONV, REG_ELINESEARCH or REG_ENONFINITE as
 * reg_solve does, with v holding the last accepted iterate. */
typedef struct reg3_ctx reg3_ctx;
reg_status reg3_create(int n1, int n2, int n3, int nt, double beta, const reg_options* opt,
                       reg3_ctx** out);
reg_status reg3_destroy(reg3_ctx* ctx);
reg_status reg3_set_stream(reg3_ctx* ctx, void* cuda_stream);
reg_status reg3_set_images(reg3_ctx* ctx, const float* m_R, const float* m_T);
/* m1 = the state solve of eq. state-slm from m0 with velocity v (3 fields) */
reg_status reg3_transport(reg3_ctx* ctx, const float* v, const float* m0, float* m1);
/* Deformation map of v (§2: m_1 = m_T o y, from v after the solve): u = y - x
 * (3 fields, physical units), the composition of the nt departure maps
 * (u_j = u_{j-1}(X_D) + X_D - x, the context's interpolation model), and,
 * if det is not NULL, det grad y = det(I + grad u) with spectral derivatives
 * (one field; the quantity §4 bounds when choosing beta). u and det must not
 * overlap (REG_EINVAL). The next call at a velocity rebuilds its state. */
reg_status reg3_deformation_map(reg3_ctx* ctx, const float* v, float* u, float* det);
/* REG_SPEC_GRAD (1 -> 3 fields), REG_SPEC_DIV (3 -> 1), REG_SPEC_REGPOW
 * (3 -> 3, (beta A)^s; for s != 1 the zero entry of A's symbol is one, so
 * the mean is scaled by beta^s, eq. reg-precond) on the 3D grid; other ops
 * REG_EINVAL */
reg_status reg3_spectral(reg3_ctx* ctx, int op, double s, const float* in, float* out);
/* *J (host) and, if g is not NULL, the reduced gradient (3 fields) at v;
 * synchronises */
reg_status reg3_objective_gradient(reg3_ctx* ctx, const float* v, double* J, float* g);
/* Hvt = H(v) vt, the Gauss-Newton matvec; synchronises */
reg_status reg3_hessian_matvec(reg3_ctx* ctx, const float* v, const float* vt, float* Hvt);
/* the inexact Newton-Krylov solve of reg_solve (§3.4.1) with PCG and P_REG;
 * v is the initial guess and receives the result; info may be NULL */
reg_status reg3_solve(reg3_ctx* ctx, float* v, double gtol, reg_info* info);
/* z = P^-1 r with the context's preconditioner (3 fields each; P_2L at the
 * velocity v: its coarse problem is restricted from v, and the Chebyshev
 * bounds are estimated on first use); synchronises */
reg_status reg3_precond_apply(reg3_ctx* ctx, const float* v, const float* r, float* z);
/* Chebyshev bounds of P_2L's coarse split operator at v = 0 (§3.4.2
 * "Eigenvalue Estimates"; e_max from Lanczos, e_min analytic), estimated by
 * this call; REG_EINVAL for a P_REG context */
reg_status reg3_eigen_bounds(reg3_ctx* ctx, double* emin, double* emax);
const char* reg3_last_error(const reg3_ctx* ctx);

/* ---- Lockstep batches: one launch per step over every problem ------------
 * B independent problems (any grids reg_create accepts, nt shared, beta[i]
 * per problem) held in one set of device arrays with a table of (n1, n2,
 * offset) per problem. Every semi-Lagrangian step (departure points, state,
 * adjoint, incremental state and incremental adjoint steps, the gathers of
 * div v and of the gradient history; eq. state-slm, eq. adj-slm,
 * eq. inc-state-slm, eq. inc-adj-slm) is ONE kernel launch over the 32 x 32
 * tiles of all problems; every FFT pass is one launch per run of problems
 * with the same grid and beta (the batch orders the problems so that such
 * runs are contiguous); every per-problem inner product and norm is one
 * segmented reduction launch with an FP64 result per problem; the
 * Gauss-Newton matvec is captured once as a CUDA graph and replayed by every
 * PCG iteration. The Newton-Krylov method (§3.4.1) runs in lockstep: each
 * problem follows its own iteration (gradient test, forcing term, PCG stop,
 * Armijo step) and a device mask lets the kernels skip the problems that do
 * not take part in a phase. Each problem's results are bitwise those of the
 * one-problem calls on a context with the same options (the same kernels'
 * arithmetic, the same reduction partition and order).
 * Options: the defaults of reg_default_options except precond = REG_PC_REG
 * (required: P_REG, §3.4.2); interp must be REG_INTERP_SPLINE, hessian GN,
 * precision FP64, incompressible 0, beta_w 0, fused_transport 1,
 * persistent_matvec 0; anything else returns REG_EINVAL. The steps run the
 * fused prefilter+step kernels only: a velocity whose displacement per step
 * exceeds their 64^2 box (14 cells) makes objective_gradient and
 * hessian_matvec return REG_EINVAL, and inside reg_lockstep_solve an Armijo
 * trial with such a displacement counts as a rejected trial (J = +inf),
 * where a one-problem context would take the separate prefilter instead.
 * Pointer arrays are host arrays of B device pointers, 16-byte aligned, with
 * the per-problem layout of the single-problem calls. The batch runs on its
 * own non-blocking stream; every call returns after synchronising it. */
typedef struct reg_lockstep reg_lockstep;
reg_status reg_lockstep_create(const reg_grid* grids, int B, int nt, const double* beta,
                               const reg_options* opt, reg_lockstep** out);
reg_status reg_lockstep_destroy(reg_lockstep* batch);
/* Orders the batch's work after what is queued on cuda_stream so far. */
reg_status reg_lockstep_set_stream(reg_lockstep* batch, void* cuda_stream);
reg_status reg_lockstep_set_images(reg_lockstep* batch, const float* const* m_R,
                                   const float* const* m_T);
/* J[i] (host, B entries) and, if g is not NULL, g[i] for every problem. */
reg_status reg_lockstep_objective_gradient(reg_lockstep* batch, const float* const* v, double* J,
                                           float* const* g);
reg_status reg_lockstep_hessian_matvec(reg_lockstep* batch, const float* const* v,
                                       const float* const* vt, float* const* Hvt);
/* reg_solve of every problem in lockstep; v[i] is the initial guess and
 * receives the result; infos (host, B entries) may be NULL (seconds is the
 * whole batch's wall time). Returns as reg_batch_solve. */
reg_status reg_lockstep_solve(reg_lockstep* batch, float* const* v, double gtol, reg_info* infos);
/* Diagnostics: replays the matvec graph of the last reg_lockstep_hessian_matvec
 * `reps` times between two CUDA events on the batch's stream (every problem
 * active, the cached velocities) and returns the mean device time per
 * matvec in *ms (REG_ESTATE before that graph exists: two matvec calls). */
reg_status reg_lockstep_matvec_time(reg_lockstep* batch, int reps, double* ms);
/* The batch's total grid points, 32 x 32 tiles and the kernels in one
 * replay of the solver's matvec graph (0 before its capture); NULL outputs
 * are skipped. */
reg_status reg_lockstep_info(const reg_lockstep* batch, long long* points, int* tiles,
                             int* launches);
const char* reg_lockstep_last_error(const reg_lockstep* batch);

/* ---- Learned warm start (no counterpart in the paper) --------------------
 * A U-Net maps an image pair (m_R, m_T) on an S x S grid to a stationary
 * velocity v_0 from which reg_solve starts; the solve runs to the same
 * gradient tolerance and decides the result (reg_warm_start keeps
 * v_0 only if J(v_0) < J(0)). Architecture: 4 levels with 32, 64, 128, 256
 * channels, two periodic 3x3 convolutions + bias + ReLU per level, 2x2
 * average pooling down, nearest-neighbour 2x upsampling up, skip
 * concatenation [upsampled, encoder output], a last periodic 3x3
 * convolution to the 2 velocity components. Forward, backward and Adam run
 * in the library's kernels: convolutions are implicit GEMMs on the BF16
 * tensor cores with FP32 accumulation; activations and their gradients are
 * BF16, master weights, weight gradients and Adam moments FP32.
 *
 * Parameter layout (host float arrays of reg_unet_param_count() values): for
 * each layer in the order enc0a (2->32), enc0b (32->32), enc1a (32->64),
 * enc1b, enc2a (64->128), enc2b, enc3a (128->256), enc3b, dec2a (384->128),
 * dec2b, dec1a (192->64), dec1b, dec0a (96->32), dec0b, out (32->2): the
 * weights W[co][t][ci] with tap t = 3a + b reading the input at offset
 * (a - 1, b - 1) in (row, column), then the biases b[co].
 *
 * Images and velocities use the single-problem layouts: a batch of B images
 * is B*S*S floats, a batch of velocities B*2*S*S (per problem component 1
 * then 2). `idx` (device int32, B entries, may be NULL for 0..B-1) selects
 * the problems of a batch from larger arrays. Device buffers start on a
 * 16-byte boundary. Calls run on the stream set by reg_unet_set_stream. */
typedef struct reg_unet reg_unet;
long long reg_unet_param_count(void);
/* S: multiple of 32 in [32, 1024]; batch_max * S * S <= 2^26. Parameters
 * start at zero: set them before use. */
reg_status reg_unet_create(int S, int batch_max, reg_unet** out);
reg_status reg_unet_destroy(reg_unet* net);
int reg_unet_size(const reg_unet* net);
reg_status reg_unet_set_stream(reg_unet* net, void* cuda_stream);
/* host parameters in, Adam moments and step count reset; synchronises */
reg_status reg_unet_set_params(reg_unet* net, const float* host_params);
reg_status reg_unet_get_params(reg_unet* net, float* host_params);
/* v = net(m_R, m_T) for B problems (v: B*2*S*S, device) */
reg_status reg_unet_forward(reg_unet* net, int B, const int* idx, const float* m_R,
                            const float* m_T, float* v);
/* mean squared error L = mean (net(m_R, m_T) - v_target)^2 over all B*2*S*S
 * values (*loss, host; may be NULL) and its gradient dL/dparams copied to
 * host_grad (parameter layout; may be NULL). Parameters are not changed. */
reg_status reg_unet_gradients(reg_unet* net, int B, const int* idx, const float* m_R,
                              const float* m_T, const float* v_target, float* host_grad,
                              double* loss);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, learning
 * rate lr) on the loss of reg_unet_gradients; *loss (host, may be NULL) is
 * the loss before the step */
reg_status reg_unet_train_step(reg_unet* net, int B, const int* idx, const float* m_R,
                               const float* m_T, const float* v_target, float lr, double* loss);
/* Tensor-core path of the forward and data-gradient 3x3 convolutions (no
 * counterpart in the paper): 0 (default) BF16 mma.sync implicit GEMMs in
 * registers; 1 the fifth-generation tensor cores (tcgen05.mma, BF16 operands
 * staged in shared memory, the FP32 accumulator in tensor memory). Both
 * accumulate in FP32; the results differ by accumulation order only. With
 * path 1, forward, gradients and train_step synchronise once more to read
 * the kernels' error flag: a convolution whose bounded wait for its MMAs ran
 * out returns REG_ETIMEOUT (network still usable). The weight-gradient
 * GEMMs stay on mma.sync. REG_EINVAL for other values. */
reg_status reg_unet_set_conv_path(reg_unet* net, int path);
const char* reg_unet_last_error(const reg_unet* net);

/* Warm start for the context's images: restricts m_R, m_T spectrally to the
 * network's grid (the problem grid must be square with S, 2S or 4S points
 * per axis), evaluates the network, prolongs v_0 spectrally to the problem
 * grid and writes it to v (device, 2*n1*n2) if J(v_0) < J(0), else writes
 * v = 0. *accepted (host, may be NULL) = 1 if v_0 was kept. Uses the
 * context's stream for the network too. */
reg_status reg_warm_start(reg_ctx* ctx, reg_unet* net, float* v, int* accepted);

/* ---- Allocation-free interpolation (no counterpart in the paper) ---------
 * For callers that must not allocate device memory while they run: code
 * whose device memory belongs to another framework's caching allocator (a
 * cudaMalloc next to it can fail or fragment that pool) and latency-bound
 * loops that cannot pay for cudaMalloc/cudaFree, which may block the host and
 * synchronise the device. Needs no reg_ctx.
 *
 * Computes the same result as reg_interpolate with the spline model:
 * out[x] = u(x + disp[x] * h), the periodic C2 cubic B-spline interpolant of
 * the samples u (n1*n2 floats, device) evaluated at displacements disp
 * (2*n1*n2 floats in cell units, component 1 then 2, device), written to out
 * (n1*n2 floats, device), on `cuda_stream` (cudaStream_t as void*, NULL for
 * the legacy default stream). n1, n2 are grid sizes reg_create accepts and
 * n1*n2 <= REG_STATIC_MAX_POINTS; anything else returns REG_EINVAL.
 *
 * The spline coefficients go to one fixed device array of
 * REG_STATIC_MAX_POINTS floats (4 MiB) inside the library, which each GPU
 * that loads the library holds until the process exits. The call allocates
 * nothing. All calls share that array, and it keeps the last call's
 * contents (every call overwrites the part it reads before reading it):
 * calls that can overlap on the GPU (different streams, or different host
 * threads on one device) race on it, so issue them on one stream or order
 * them. The first call on a device looks up the array's device address with
 * that device current; make that first call before any stream capture.
 * Returns REG_ECUDA if that look-up or one of its own launches fails (a
 * launch error pending from earlier work is cleared first, not reported). */
#define REG_STATIC_MAX_POINTS (1024 * 1024)
reg_status reg_interpolate_static(int n1, int n2, const float* u, const float* disp,
                                  float* out, void* cuda_stream);

/* Euclidean inner product of two float32 device vectors of length n (any
 * alignment; n = 0 gives 0 and allows NULL), accumulated to float64 accuracy
 * like the Krylov and line-search reductions: each thread sums exact
 * products with compensated FP32 pairs, threads and blocks are summed in
 * FP64. *out host. */
reg_status reg_dot(reg_ctx* ctx, const float* a, const float* b, long long n, double* out);

/* Message of the last error on this context (never NULL). */
const char* reg_last_error(const reg_ctx* ctx);

/* ---- Diagnostics (no counterpart in the paper) ----------------------------
 * Per-kernel-class device time for roofline reporting. While profiling is
 * enabled every launch of a class is bracketed by CUDA events on the
 * context's stream; reg_profile_read synchronises that stream and returns the
 * summed device time (ms), the number of bracketed launch groups and the
 * algorithmic bytes those launches move (inputs read once, outputs written
 * once; see the kernel sources for the per-point figures). */
enum { REG_KC_FFT_ROWS = 0,       /* row FFT passes (forward and inverse)       */
       REG_KC_FFT_COLS = 1,       /* column FFT pass with the spectral symbol    */
       REG_KC_PREFILTER = 2,      /* cubic B-spline prefilter (x and y passes)   */
       REG_KC_DEPARTURE = 3,      /* RK2 departure points                        */
       REG_KC_GATHER = 4,         /* state steps and other 4x4 gathers           */
       REG_KC_ADJOINT_STEP = 5,   /* adjoint / incremental adjoint steps         */
       REG_KC_INCSTATE_STEP = 6,  /* incremental state steps                     */
       REG_KC_REDUCE = 7,         /* FP64 inner products and norms               */
       REG_KC_VECTOR = 8,         /* Krylov vector updates                       */
       REG_KC_MATVEC = 9,         /* persistent GN data-term matvec (one launch) */
       REG_KC_COUNT = 10 };
/* enable != 0 starts profiling and clears the totals; 0 stops it. Launch
 * sequences that are replayed as CUDA graphs (the fine matvec inside PCG,
 * the P_2L application with CHEB) are then captured with an event pair
 * around every kernel and the stream is synchronised after each replay to
 * read them, so their kernel times carry no host launch gaps. */
reg_status reg_profile_enable(reg_ctx* ctx, int enable);
/* Totals of one kernel class on one grid level (0: the problem grid, 1: the
 * coarse grid of P_2L) since the last reg_profile_enable(ctx, 1); ms,
 * launches and bytes are host pointers (any may be NULL). */
reg_status reg_profile_read(reg_ctx* ctx, int level, int kclass, double* ms, long long* launches,
                            double* bytes);
/* Kernels launched by the library in this process so far (all contexts),
 * counting every kernel node of every CUDA graph replay. */
long long reg_launch_count(void);
/* Tile shapes the context's step kernels use (see reg_options.step_tile):
 * tiles[0..3] = adjoint and incremental-state step on the problem grid, then
 * on the coarse grid of P_2L (0 without one). tiles: 4 ints, host. */
reg_status reg_step_tiles(const reg_ctx* ctx, int* tiles);

#ifdef __cplusplus
}
#endif
#endif /* REGNK_REG_H */
