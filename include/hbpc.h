/*
 * hbpc.h -- C-ABI of libhbpc, a GB300 (sm_103a) implementation of the implicit
 * two-derivative deferred-correction time discretisation HBPC(q, k_max) for the
 * discontinuous Galerkin spectral element method (Zeifang & Schuetz, "Two-
 * derivative deferred correction time discretization for the discontinuous
 * Galerkin method").
 *
 * Conventions
 *  - Every function returns hbpc_status (0 = HBPC_OK) and never aborts or exits;
 *    hbpc_last_error() returns a message for the last failure of a context.
 *  - State layout (host and device): canonical FP64 array w[e][v][k][j][i] --
 *    element e = ex + nx*(ey + ny*ez), variable v, node indices (only the last
 *    `dim` of k, j, i exist), i fastest.  n_dof = n_E * n_var * (N+1)^dim.
 *  - Pointers documented as "device" must be device memory of the context's
 *    device (cudaMalloc, cudaMallocManaged or a framework allocator); "host"
 *    pointers are ordinary host memory.  The caller owns every buffer it passes;
 *    the library copies what it keeps.  All device work is enqueued on the
 *    stream given at creation (NULL = legacy default stream) and the calls
 *    return after that stream has finished the call's work.
 *  - Meshes are uniform and Cartesian.  A context is created periodic in
 *    every direction (hbpc_mesh.periodic must be 1); hbpc_set_boundary then
 *    replaces the periodic connection of a direction by two boundaries
 *    (constant Dirichlet states, Euler slip walls, Navier-Stokes no-slip
 *    walls).
 *  - Invalid arguments are rejected before anything is allocated or launched.
 */
#ifndef HBPC_H
#define HBPC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HBPC_OK = 0,
  HBPC_ERR_INVALID_ARG = 1,    /* bad parameter; nothing was done */
  HBPC_ERR_OOM = 2,            /* a device allocation failed */
  HBPC_ERR_CUDA = 3,           /* a CUDA call failed (message has the CUDA error) */
  HBPC_ERR_NO_CONVERGENCE = 4, /* Newton or GMRES iteration cap reached */
  HBPC_ERR_NONFINITE = 5,      /* a residual or update norm is NaN or Inf */
  HBPC_ERR_TIMEOUT = 6,        /* a bounded wait for the device gave up
                                  (hbpc_set_wait_limit), or a bounded
                                  wait inside the tensor-core block apply
                                  ran out (its outputs are then NaN) */
  HBPC_ERR_UNSUPPORTED = 7     /* valid request that this build does not cover */
} hbpc_status;

/* Conservation laws.  ADVECTION: w_t + div(a w) = 0 (Sec. 4.1.1).
 * BURGERS: w_t + div((w^2/2)(1,..,1)) = 0 (inviscid part of the Burgers workload).
 * EULER: compressible Euler with reference Mach number eps (Eq. 21). */
typedef enum {
  HBPC_LAW_ADVECTION = 0,
  HBPC_LAW_BURGERS = 1,
  HBPC_LAW_EULER = 2,
  /* Euler flux plus the Navier-Stokes viscous flux of Sec. 5 (Eq. 25: stress
     tensor with constant dynamic viscosity mu = nu, heat flux lambda grad T,
     lambda = c_p mu / Pr, R = 1/(gamma eps^2)), discretised with the BR2
     lifting of the gradient variables (v, T) (Sec. 5.1.1) and its
     linearisation for R^(2) (Sec. 5.1.2).  Compiled for dim 2 and 3. */
  HBPC_LAW_NAVIER_STOKES = 3
} hbpc_law;

/* Numerical flux of Eq. 13: f* = 1/2 (F(wL) + F(wR)) . n + kappa (wL - wR).
 * GLOBAL_LF: kappa is a global constant per variable, lf_scale times the paper's
 *   lambda: |a.n| (advection), 1 (Burgers), diag(1/eps, 1, .., 1, 1/eps) (Euler).
 * RUSANOV: kappa = 1/2 max(|v_n| + c) over the two traces (frozen, i.e. not
 *   differentiated, in R2 and in the linearised operator). */
typedef enum { HBPC_FLUX_GLOBAL_LF = 0, HBPC_FLUX_RUSANOV = 1 } hbpc_flux;

/* Node family of the 1-D basis (Sec. 3.1.1). */
typedef enum { HBPC_NODES_LOBATTO = 0, HBPC_NODES_GAUSS = 1 } hbpc_nodes;

/* Preconditioner of the extended linear system (Sec. 3.2.3).  NONE: plain
 * GMRES.  BJEXT: the BJ_ext block preconditioner, right preconditioning; needs
 * n_var (N+1)^dim <= 160 and 2 n_E (n_var (N+1)^dim)^2 doubles of device memory.
 * LEARNED: the BJ_ext structure with the block inverse (I - c1 J + c2 J^2)^-1
 * replaced by a learned per-element network (hbpc_pc_* below; no counterpart in
 * the paper).  BJEXT_H: the BJ^H_ext preconditioner of Sec. 3.2.3, BJ_ext with
 * the element Hessian block H_i = dR2/dW|_i (at the current sigma, neighbours
 * frozen, the Rusanov kappa not differentiated) kept in A_i, so that
 * M_i = (I - c1 J_i + c2 H_i + c2 J_i^2)^-1 and P^-1 (w, s) = (u, J u + s) with
 * u = M (w - c2 J s); the same size limit and memory as BJEXT.  For a linear
 * flux H = 0 and BJEXT_H is BJEXT; Navier-Stokes is HBPC_ERR_UNSUPPORTED (the
 * paper also drops the Hessian there).  With hbpc_set_schur the D block of
 * either preconditions the Schur system.  The preconditioner never changes the
 * answer, only the GMRES iteration count: Newton stops on the same FP64
 * residual. */
typedef enum { HBPC_PC_NONE = 0, HBPC_PC_BJEXT = 1, HBPC_PC_LEARNED = 2, HBPC_PC_BJEXT_H = 3 } hbpc_pc;

/* Arithmetic of the Krylov loop.  FP64: everything in FP64, Jv by the
 * difference quotients of Eq. 23 (Eq. 24 for a linear flux).  MIXED: the
 * Newton residual, the update and the stage logic stay FP64; the Krylov basis
 * and the Jacobian-vector products use FP32 with the analytic linearised
 * operator dR1/dw v = R2(w, v) (Sec. 3.2.1). */
typedef enum { HBPC_PREC_FP64 = 0, HBPC_PREC_MIXED = 1 } hbpc_precision;

typedef struct {
  int dim;          /* 1, 2 or 3 */
  int n[3];         /* elements per direction (n[m] >= 1 for m < dim) */
  double lo[3];     /* domain [lo, hi] per direction */
  double hi[3];
  int periodic;     /* 1: periodic in every direction (the connectivity at
                       creation; hbpc_set_boundary bounds a direction later);
                       0 is HBPC_ERR_UNSUPPORTED, any other value
                       HBPC_ERR_INVALID_ARG */
} hbpc_mesh;

typedef struct {
  int law;          /* hbpc_law */
  int flux;         /* hbpc_flux */
  double a[3];      /* advection velocity */
  double gamma;     /* ratio of specific heats (Euler) */
  double eps;       /* reference Mach number eps (Euler, Eq. 21); also enters
                       eps_FD of Eq. 23 for every law (use 1 for advection) */
  double lf_scale;  /* multiplies the global-LF lambda; 1 = Eq. 13 as printed */
  double nu;        /* viscosity: nu of a term nu Laplace(w) added to a scalar
                       law (advection or Burgers), discretised by the BR2
                       lifting of Sec. 5.1.1 (Eqs. 26-30 with F^v = nu grad w,
                       central face fluxes, face-local liftings), or the dynamic
                       viscosity mu of HBPC_LAW_NAVIER_STOKES.  0 = inviscid;
                       < 0 is HBPC_ERR_INVALID_ARG; > 0 with Euler is
                       HBPC_ERR_UNSUPPORTED (use the Navier-Stokes law). */
  double eta_br2;   /* BR2 stabilisation factor of the face-local liftings (the
                       paper leaves its value open); <= 0 selects 2 * dim, the
                       number of faces of an element */
  double prandtl;   /* Prandtl number of the Navier-Stokes heat flux; <= 0
                       selects 0.72, the paper's value.  Ignored by other laws. */
} hbpc_physics;

typedef struct {
  int q;                 /* order of the quadrature: 4, 6 or 8 (Eq. A.1-A.3) */
  int kmax;              /* corrector sweeps, >= 0 */
  double dt;             /* time step, > 0 */
  double tol_newton_rel; /* ||G(X^r)|| <= tol * ||G(X^0)|| (Sec. 3.2.1) */
  double tol_newton_abs; /* or ||dW||_2 <= tol_abs (Sec. 5.2); 0 disables */
  double tol_gmres_rel;  /* GMRES relative tolerance */
  int gmres_restart;     /* Krylov dimension per cycle, 1..1000 */
  int gmres_max_iter;    /* GMRES iterations per Newton step (cap), >= 1 */
  int newton_max_iter;   /* Newton iterations per stage solve (cap), >= 1 */
  int pc;                /* hbpc_pc */
  int precision;         /* hbpc_precision */
  double t_end;          /* final time T_end of the problem (Algorithm 1), used
                            by hbpc_run; 0 = not given; < 0 or not finite is
                            HBPC_ERR_INVALID_ARG */
} hbpc_solver;

typedef struct {
  long long steps;        /* HBPC steps taken */
  long long newton_solves;
  long long newton_its;
  long long gmres_its;
  long long r1_evals;     /* full-mesh operator passes (R1, R2 or linearised) */
  long long r2_evals;
  long long launches;     /* kernel launches issued by the library */
  double t;               /* simulated time */
  long long arnoldi_cols; /* sum over Arnoldi iterations of the columns
                             orthogonalised against (j + 1 at column j) */
  long long pc_exact_blocks; /* learned preconditioner: element blocks that
                                failed their probe check and got the exact
                                inverse instead (summed over builds) */
  long long pc_apply_tc;     /* 1 when the last preconditioner build put the
                                BJ_ext apply on the tensor cores (one FP64
                                block shared by all elements, applied through
                                exact BF16 digit-plane products; environment
                                HBPC_PC_TC=0 at creation keeps the CUDA-core
                                apply), else 0 */
} hbpc_stats;

/* Phases of the per-launch device timing (hbpc_profile_*). */
enum {
  HBPC_PHASE_JV = 0,        /* Jacobian-vector product passes (Eq. 23/24) */
  HBPC_PHASE_OPERATOR = 1,  /* residual, R1, R2 passes outside the Krylov loop */
  HBPC_PHASE_DOT = 2,       /* Arnoldi multi-dot passes */
  HBPC_PHASE_UPDATE = 3,    /* Arnoldi update + norm passes */
  HBPC_PHASE_VECTOR = 4,    /* norms, solution update, stage combinations */
  HBPC_PHASE_PC = 5,        /* BJ_ext apply */
  HBPC_PHASE_PC_BUILD = 6,  /* BJ_ext assembly, S = I - c1 J + c2 J^2, inverse */
  HBPC_NPHASES = 7
};

typedef struct hbpc_ctx hbpc_ctx;

/* Create a context: computes the basis (Sec. 3.1.1) on the host, allocates all
 * device memory the method needs (zero-filled) and binds to the current CUDA
 * device and the given stream (cudaStream_t, NULL = default).  N >= 1 and
 * (N+1) <= 8; a (law, dim, N, node family) whose kernels are not compiled in is
 * HBPC_ERR_UNSUPPORTED before any device call.
 * Environment, read at creation: HBPC_VERBOSE=1 prints the Newton and GMRES
 * iterations on stderr; HBPC_GRAPH=0 launches the kernels of the GMRES
 * iterations one by one instead of replaying each batch of four iterations as
 * a CUDA graph captured on the context's stream (the default; a stream the
 * caller is capturing, a phase-profiled call or a capture the runtime refuses
 * also take direct launches). */
hbpc_status hbpc_create(hbpc_ctx** out, const hbpc_mesh* mesh, int N, int nodes,
                        const hbpc_physics* phys, const hbpc_solver* solver,
                        void* cuda_stream);

/* Free all device memory of the context.  Accepts NULL. */
void hbpc_destroy(hbpc_ctx* ctx);

/* Number of state values n_dof and of variables per node. */
long long hbpc_ndof(const hbpc_ctx* ctx);
int hbpc_nvar(const hbpc_ctx* ctx);

/* Physical node coordinates, host output x[dim][n_E][(N+1)^dim] (FP64). */
hbpc_status hbpc_node_coords(const hbpc_ctx* ctx, double* x);

/* 1-D basis of degree N (Sec. 3.1.1), host outputs: nodes xi[N+1], weights
 * w[N+1], Dhat[(N+1)*(N+1)] row-major with Dhat[i][j] = -(w_j/w_i) l_i'(xi_j),
 * lm[N+1] = l_i(-1), lp[N+1] = l_i(+1).  Any output may be NULL. */
hbpc_status hbpc_basis(int N, int nodes, double* xi, double* w, double* Dhat,
                       double* lm, double* lp);

/* Copy the state w^n in (out): `w` has n_dof FP64 values, on the device if
 * on_device != 0, else on the host. */
hbpc_status hbpc_set_state(hbpc_ctx* ctx, const double* w, int on_device);
hbpc_status hbpc_get_state(const hbpc_ctx* ctx, double* w, int on_device);
hbpc_status hbpc_set_time(hbpc_ctx* ctx, double t);

/* Advance the state by n_steps HBPC(q, k_max) steps (Algorithm 1, Sec. 2.1).
 * On non-convergence the state stays at the last completed step and
 * HBPC_ERR_NO_CONVERGENCE is returned; a non-finite Newton residual or update
 * (for instance from a state holding NaN) gives HBPC_ERR_NONFINITE, with the
 * state likewise left at the last completed step. */
hbpc_status hbpc_step(hbpc_ctx* ctx, int n_steps);

/* Advance the state from the context's time t (hbpc_set_time, 0 at creation)
 * to t_end (Algorithm 1 run to T_end): whole steps of the solver's dt while
 * they fit, then, if t_end - t is not a whole number of steps (a remainder of
 * more than 1e-10 dt), one last step of the remaining length, so that the
 * state lands on t_end exactly; the time is t_end afterwards.  t_end < t (by
 * more than 1e-10 dt) or not finite is HBPC_ERR_INVALID_ARG.  Errors as
 * hbpc_step; the time then counts the steps completed. */
hbpc_status hbpc_advance_to(hbpc_ctx* ctx, double t_end);

/* hbpc_advance_to(ctx, solver.t_end); HBPC_ERR_INVALID_ARG if the solver was
 * created without a final time (t_end = 0). */
hbpc_status hbpc_run(hbpc_ctx* ctx);

/* Corrector batching (the paper's outlook, Sec. 6; Algorithm 1 unchanged):
 * the right-hand sides of the s - 1 corrector stages of one sweep depend only
 * on the previous level, so with on = 1 every sweep solves them together as
 * one batched Newton-GMRES (stage l is instance l - 1 of an internal group
 * with the context's mesh, law, solver and precision; each stage keeps its own
 * Newton stopping test and, in the MIXED mode, its own GMRES; in FP64 mode the
 * stages share one GMRES with rows scaled by 1 / ||G_l||).  Every launch then
 * covers s - 1 stages.  The answer is the same to the Newton tolerance.
 * Allocates about (s - 1) times the context's solver memory on on = 1; 0
 * releases it.  HBPC_ERR_UNSUPPORTED for the Navier-Stokes law and the learned
 * preconditioner.  Runs on the context's stream. */
hbpc_status hbpc_set_corrector_batch(hbpc_ctx* ctx, int on);

/* Schur form of the Newton systems (Sec. 3.2.4, Eq. 19): with on = 1 every
 * Newton step solves J_Schur dW = -G1 + (alpha2 dt^2/2) (dR2/dsigma) G2 with
 * J_Schur = I - alpha1 dt dR1/dW + (alpha2 dt^2/2) dR2/dW
 * + (alpha2 dt^2/2) (dR1/dW)^2 by matrix-free GMRES (each product two
 * passes of the extended product of Eq. 23/24: on (z, 0) for dR1/dW z, then
 * on (z, dR1/dW z)), right preconditioned by the BJ_ext D blocks
 * (I - c1 J_i + c2 J_i^2)^-1 when the context has a block preconditioner, and
 * then sets dsigma = -G2 + (dR1/dW) dW.  The Newton stopping tests and the
 * root are those of the extended form.  FP64 mode and single problems only
 * (HBPC_ERR_UNSUPPORTED otherwise, also with corrector batching on).
 * Allocates three 2 n_dof vectors on the first on = 1; 0 returns to the
 * extended form. */
hbpc_status hbpc_set_schur(hbpc_ctx* ctx, int on);

/* Boundaries of direction `dir` (0 <= dir < dim): the lower (x_dir = lo) and
 * upper (x_dir = hi) ends get kinds kind_lo, kind_hi, both HBPC_BC_PERIODIC
 * (the periodic connection, the default) or both bounded:
 *   HBPC_BC_DIRICHLET  a constant exterior state: `state_*` points to n_var host
 *                      doubles (conservative variables; Euler: density and
 *                      pressure > 0), copied;
 *   HBPC_BC_WALL       the slip wall of the Euler equations: the exterior state
 *                      is the own trace with the momentum along dir reversed;
 *   HBPC_BC_NOSLIP     the adiabatic no-slip wall of the Navier-Stokes
 *                      equations: the exterior state is the own trace with its
 *                      whole momentum reversed; the BR2 lifting (Sec. 5.1.1)
 *                      sees exterior channels (v, T) = (-v, T) and the own
 *                      gradient with dT/dn reversed, so the wall velocity is
 *                      zero, the wall takes the own shear stress, does no work
 *                      and passes no heat.  A Dirichlet state gives the
 *                      Navier-Stokes lifting the state's (v, T) and the own
 *                      gradient.
 * A boundary face takes the numerical flux of Eq. 13 (or f~* of Sec. 3.1.2 for
 * R2) with that exterior state; the exterior direction of R2 is its time
 * derivative (zero for Dirichlet data, the mirrored own sigma at a wall), so
 * R2 stays the derivative of R1 and every Jacobian-vector product, the BJ_ext
 * and BJ^H_ext blocks and the mixed mode include the boundaries.  Not for the
 * scalar viscous term (nu > 0 with advection or Burgers: HBPC_ERR_UNSUPPORTED);
 * a slip wall needs the Euler equations, a no-slip wall Navier-Stokes; mixed
 * periodic/bounded ends, an unknown kind or a bad state are
 * HBPC_ERR_INVALID_ARG; nothing changes on an error.  Applies to the
 * following calls (the preconditioner is rebuilt). */
typedef enum { HBPC_BC_PERIODIC = 0, HBPC_BC_DIRICHLET = 1, HBPC_BC_WALL = 2, HBPC_BC_NOSLIP = 3 } hbpc_bc;
hbpc_status hbpc_set_boundary(hbpc_ctx* ctx, int dir, int kind_lo, const double* state_lo, int kind_hi,
                              const double* state_hi);

/* When the block preconditioner is built: every_newton_iteration = 1 (the
 * default) rebuilds it before every Newton iteration, as in the paper's study
 * (Sec. 4.1.2); 0 builds it once per Newton solve, at the solve's first
 * iterate X^0, and reuses it for the later iterations (the reuse the paper
 * suggests at the end of Sec. 4.1.2: fewer builds, possibly more GMRES
 * iterations; Newton still stops on the same residual).  Other values:
 * HBPC_ERR_INVALID_ARG.  The batch form sets every group. */
hbpc_status hbpc_set_pc_rebuild(hbpc_ctx* ctx, int every_newton_iteration);

/* Device-driven steps (Algorithm 1 with the Newton iteration of Eq. 17 and
 * restarted GMRES; no counterpart in the paper's host-driven solver).  With
 * on = 1 every hbpc_step / hbpc_advance_to step is ONE CUDA graph launch: the
 * stages are straight-line work, every Newton iteration and every GMRES cycle
 * a conditional WHILE node, a cycle's end and its restart IF nodes, and small
 * control kernels take the decisions the host takes otherwise (the stopping
 * tests of Sec. 3.2.1, the GMRES state, the iteration caps), so the host
 * waits once per step instead of once per few Arnoldi columns.  The kernels,
 * their order and hence the results are those of the host-driven step.  The
 * graph is captured on the first step and again whenever the solver settings,
 * the operator parameters (boundaries included) or launch shapes changed
 * (hbpc_advance_to's shorter last step captures once more).  A failed solve
 * ends the step with the same status as the host-driven step (HBPC_ERR_NONFINITE,
 * HBPC_ERR_NO_CONVERGENCE) and leaves the state at the previous step; the
 * counters (hbpc_get_stats) are read from the device after the step.  Covers
 * FP64 and mixed precision, no preconditioner, BJ_ext and BJ^H_ext, single
 * problems and batch groups; with the Schur form, corrector batching, the
 * learned preconditioner, training-data collection, phase profiling or a
 * stream the caller is capturing, steps run host-driven.  Allocates a small
 * control block and a capture stream on the first on = 1; on = 1 with the
 * Schur form, corrector batching or the learned preconditioner set is
 * HBPC_ERR_UNSUPPORTED. */
hbpc_status hbpc_set_step_graph(hbpc_ctx* ctx, int on);

/* Bounded waits.  Every call of the context waits for its stream before it
 * returns (and inside the Newton loop, for the residual norms).  With a limit
 * of `seconds` > 0 such a wait gives up after that long and the call returns
 * HBPC_ERR_TIMEOUT; 0 (the default) waits without a limit.  After
 * HBPC_ERR_TIMEOUT the work already enqueued keeps running on the device and
 * the context's state is unspecified: destroy the context (hbpc_destroy waits
 * for its stream to finish). */
hbpc_status hbpc_set_wait_limit(hbpc_ctx* ctx, double seconds);

/* r = R1(w), Eq. 12 with the flux of Eq. 13.  w, r: device, n_dof FP64. */
hbpc_status hbpc_eval_R1(hbpc_ctx* ctx, const double* w, double* r);

/* r = R2(w, s), Eq. 16.  w, s, r: device, n_dof FP64. */
hbpc_status hbpc_eval_R2(hbpc_ctx* ctx, const double* w, const double* s, double* r);

/* Extended residual of one implicit stage (Sec. 3.2.1):
 *   G = (W - b - alpha1 dt R1(W) + alpha2 dt^2/2 R2(W, S),  S - R1(W)).
 * X = (W, S) and G are device arrays of 2 n_dof FP64, b of n_dof. */
hbpc_status hbpc_eval_G(hbpc_ctx* ctx, const double* b, double alpha1, double alpha2,
                        const double* X, double* G);

/* Jacobian-vector product of the stage system at X applied to dX (Eq. 23, or
 * Eq. 24 for a linear flux; the context's precision selects the form).
 * X, dX, out: device, 2 n_dof FP64. */
hbpc_status hbpc_eval_Jv(hbpc_ctx* ctx, double alpha1, double alpha2, const double* X,
                         const double* dX, double* out);

/* Block preconditioner (BJ_ext or BJ^H_ext of Sec. 3.2.3, or the learned
 * blocks) built at the state W of X = (W, S) (BJ^H_ext: its Hessian blocks at
 * (W, S)) for the stage coefficients alpha1, alpha2, applied to `in`:
 * out = P^-1 in.  Needs a context with pc != HBPC_PC_NONE.  In the
 * MIXED precision mode the blocks S_e, their inverses and the apply are FP32
 * (what the Krylov loop uses); in FP64 mode everything is FP64 (a block
 * shared by all elements is applied through exact BF16 digit-plane products
 * on the tensor cores, rounded once to FP64; hbpc_stats.pc_apply_tc).
 * X, in, out: device, 2 n_dof FP64. */
hbpc_status hbpc_eval_pc(hbpc_ctx* ctx, double alpha1, double alpha2, const double* X,
                         const double* in, double* out);

/* Solve one implicit stage G(X) = 0 (Eq. 7-9) by Newton-GMRES from
 * X^0 = (W0, R1(W0)).  b, W0: device n_dof; W_out, S_out: device n_dof (S_out
 * may be NULL). */
hbpc_status hbpc_newton_solve(hbpc_ctx* ctx, const double* b, double alpha1, double alpha2,
                              const double* W0, double* W_out, double* S_out);

hbpc_status hbpc_get_stats(const hbpc_ctx* ctx, hbpc_stats* out);
hbpc_status hbpc_reset_stats(hbpc_ctx* ctx);

/* Switch the preconditioner of an existing context (allocates what it needs). */
hbpc_status hbpc_set_pc(hbpc_ctx* ctx, int pc);

/* Learned block preconditioner (the workload's addition; the paper has none).
 * At every build each learned block is checked with one random sign probe x:
 * if |M~ S x - x| > 0.5 |x| the element gets the exact inverse S^-1 (formed
 * and inverted like BJ_ext) instead; hbpc_stats.pc_exact_blocks counts them. */
/* Learned block preconditioner, details.
 * Network: f = standardised [W_e, c1, c2] (d_in = n_b + 2, zero padded to a
 * multiple of 16) -> tanh(256) -> tanh(256) -> O (n_b^2, padded to a multiple
 * of 8); M~_e = I + reshape(O) row-major.  BF16 tensor-core GEMMs with FP32
 * accumulation, FP32 master weights and Adam.  Parameters as one FP32 array:
 * W1 (256 x d_in_padded), b1 (256), W2 (256 x 256), b2, W3 (d_out_padded x 256),
 * b3 (d_out_padded), row-major weights (out x in), then the feature
 * standardisation mu (d_in_padded) and sd (d_in_padded): f = (raw - mu) / sd,
 * then 4 stage classes: keys (c1, c2) x 4 (c1 <= 0: unused) and their fixed
 * mean inverses minus I (4 x d_out_padded, row-major blocks); the block of
 * stage coefficients (c1, c2) is M~ = I + C_k + reshape(O), k the class with
 * equal keys, else the nearest.  Keys, means and standardisation are computed
 * from the replay buffer at the first hbpc_pc_train after hbpc_pc_model_init
 * (means from the stored exact inverses, zero without them). */
hbpc_status hbpc_pc_model_info(hbpc_ctx* ctx, int* d_in_padded, int* hidden, int* d_out_padded,
                               long long* n_params);
/* Random weights (normal, scaled by 1/sqrt(fan-in); W3 further by out_scale),
 * zero biases, Adam state cleared; standardisation and stage classes are
 * recomputed at the next hbpc_pc_train. */
hbpc_status hbpc_pc_model_init(hbpc_ctx* ctx, unsigned long long seed, double out_scale);
hbpc_status hbpc_pc_model_get(hbpc_ctx* ctx, float* params);        /* host output */
hbpc_status hbpc_pc_model_set(hbpc_ctx* ctx, const float* params);  /* host input */
/* Training losses of the learned preconditioner.
 * PROBE: L = sum_{s,p} |M~_s S_s x_p - x_p|^2 / (B P), S = I - c1 J + c2 J^2,
 *        with Rademacher probes x_p (what a preconditioner should achieve).
 * INVERSE: L = sum_s |M~_s - T_s|_F^2 / B against the exact block inverses
 *        T_s = S_s^-1 computed by the BJ_ext path during data collection (a
 *        well-conditioned regression, used to start training). */
typedef enum { HBPC_PC_LOSS_PROBE = 0, HBPC_PC_LOSS_INVERSE = 1 } hbpc_pc_loss;
/* Loss and gradient for given inputs (host): F (B x d_in_padded, already
 * standardised), J (B x n_b x n_b column-major: the element Jacobian for
 * PROBE, the target inverse for INVERSE), c12 (B x 2), X (B x P x n_b probes;
 * PROBE only, may be NULL for INVERSE).  B a multiple of 8, 1 <= P <= 16;
 * grads (host, n_params) may be NULL. */
hbpc_status hbpc_pc_loss_grad(hbpc_ctx* ctx, int loss_kind, int B, int P, const float* F, const float* J,
                              const float* c12, const float* X, double* loss, float* grads);
/* The network's block approximations for given inputs (host): F (B x
 * d_in_padded, already standardised), c12 (B x 2) -> M (B x n_b x n_b,
 * row-major) = I + C_k + reshape(O), the same BF16 GEMM chain with FP32
 * accumulation as the preconditioner build.  B a multiple of 8. */
hbpc_status hbpc_pc_model_forward(hbpc_ctx* ctx, int B, const float* F, const float* c12, float* M);
/* One Adam step (Kingma & Ba 2015; b1 = 0.9, b2 = 0.999, eps = 1e-8, the
 * training's settings and its step counter) of the network parameters with
 * the given gradient (host, the first n_params - (2 d_in_padded + classes)
 * entries: the weights and biases). */
hbpc_status hbpc_pc_adam_step(hbpc_ctx* ctx, const float* grads, double lr);
/* Sample `samples_per_newton` elements' (features, J_e, c1, c2) at every Newton
 * iteration that builds a block preconditioner into a replay buffer of
 * `capacity` samples (0 stops sampling); with the BJ_ext preconditioner the
 * exact block inverses S_e^-1 are stored too (targets of the INVERSE loss). */
hbpc_status hbpc_pc_collect(hbpc_ctx* ctx, int samples_per_newton, int capacity);
/* `iters` Adam steps of the given loss (hbpc_pc_loss) on random batches of the
 * replay buffer, `probes` Rademacher probes per sample for PROBE (SplitMix64 of
 * the seed); first and last batch losses to loss_first / loss_last (may be
 * NULL).  INVERSE needs every buffered sample to have its target
 * (HBPC_ERR_INVALID_ARG otherwise). */
hbpc_status hbpc_pc_train(hbpc_ctx* ctx, int loss_kind, int iters, int batch, int probes, double lr,
                          unsigned long long seed, double* loss_first, double* loss_last);

/* Per-launch device timing: while enabled, every kernel launch of the context
 * is bracketed by CUDA events on its stream (this adds a little host overhead;
 * use it in a separate measurement pass).  hbpc_profile_get writes, per phase
 * (HBPC_PHASE_*), the summed device milliseconds and the number of launches
 * into host arrays of n_phases entries; hbpc_profile_enable(ctx, 1) clears. */
hbpc_status hbpc_profile_enable(hbpc_ctx* ctx, int enable);
hbpc_status hbpc_profile_get(hbpc_ctx* ctx, double* ms, long long* launches, int n_phases);

/* Allocation-free Jacobian-vector product: the same result as hbpc_eval_Jv for
 * the discretisation described by (mesh, N, nodes, phys) and the time step dt,
 * without a context and without allocating any memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc
 * -- code that runs while a framework owns all device memory through its own
 * pool or arena, code with a fixed memory budget decided up front, or code that
 * must not trigger the implicit synchronisation and fragmentation an allocation
 * can cause.  Its scratch (R1(W) and R2(W, S) at X, the partial sums of the
 * ||dW||, ||dS|| reduction, a reduction ticket) is one file-scope device array
 * of about 4.2 MB that every GPU which loads the library holds until the
 * process exits.  Limits and behaviour:
 *  - n_dof must not exceed 262144 (else HBPC_ERR_INVALID_ARG, nothing launched);
 *  - the first call on a device looks up the array's device address with that
 *    device current, so make that first call before any stream capture;
 *  - all calls share the array, which keeps the last call's contents; each call
 *    clears the part that must start at zero, but calls that overlap on the GPU
 *    (concurrent streams or threads) race on it and must be serialised;
 *  - the device address is looked up once per device and kept; after
 *    cudaDeviceReset on that device it is stale, so do not call this entry
 *    point again in that process;
 *  - work is enqueued on cuda_stream (NULL = default) and the call returns when
 *    that stream has finished it, also when it fails after its first launch;
 *    errors are reported by hbpc_last_error(NULL).
 * X, dX, out: device, 2 n_dof FP64 (X = (W, S)).  `out` must not overlap X or
 * dX (the kernels read X and dX after they have begun writing out; an
 * overlapping out is HBPC_ERR_INVALID_ARG, nothing launched); X and dX may
 * overlap each other. */
hbpc_status hbpc_eval_Jv_noalloc(const hbpc_mesh* mesh, int N, int nodes, const hbpc_physics* phys,
                                 double dt, double alpha1, double alpha2, const double* X,
                                 const double* dX, double* out, void* cuda_stream);

/* FP64 FMA throughput of the current device in GFLOP/s (a few milliseconds of
 * independent FMA chains on every SM, best of three, CUDA events).  Used as the
 * arithmetic roofline of the FP64 kernels.  Allocates and frees a small buffer. */
hbpc_status hbpc_fp64_fma_peak(double* gflops);

/* Launch-shape autotuner (no counterpart in the paper): times, on the
 * context's own buffers, the candidate shapes of the Krylov reductions (blocks
 * = 1..4 x SMs or the row-tile count / 1..3; CGS2 columns at j = 16 and m/2)
 * and of the block-preconditioner
 * apply (1, 2, 4, 8 or 16 elements per block, at most 256 threads), median of
 * 7 launches each, and
 * keeps the fastest.  Call it before stepping or between steps; the result
 * changes only the summation order of the reductions.  out may be NULL. */
typedef struct {
  int krylov_blocks;        /* chosen blocks of the Krylov reductions */
  double krylov_us;         /* its time for the two probe columns (microseconds) */
  double krylov_us_default; /* the same at the creation-time shape */
  int pc_elems_per_block;   /* chosen elements per block of the apply */
  double pc_us;             /* its time per apply (0 without a block preconditioner) */
  double pc_us_default;
  int cooperative_cgs;      /* 1: CGS2 runs as one cooperative launch */
} hbpc_tuning;
hbpc_status hbpc_autotune(hbpc_ctx* ctx, hbpc_tuning* out);

/* ---- Batches of independent instances (no counterpart in the paper) -----
 * n_inst problems that share dim, law, flux, gamma, eps, lf_scale, a, eta_br2,
 * the node family and the solver settings (HBPC(q, k_max), dt, tolerances,
 * preconditioner NONE or BJEXT, precision), each with its own mesh (n, lo, hi),
 * degree N[i] and viscosity phys[i].nu.  Instances with the same N form
 * groups of at most max_per_group instances (<= 0: one group per N), formed
 * in order of size: one element numbering per group (each instance's elements
 * contiguous, padded to the operator kernel's elements per block), so every
 * kernel launch of the group covers all its instances; the Jacobian and the
 * block preconditioner are block diagonal over instances.  Newton stops per
 * instance (Sec. 3.2.1 tests applied to each instance's residual; converged
 * instances are frozen); one GMRES per Newton iteration covers the group's
 * active instances, row-scaled per instance.  Groups run concurrently, each on
 * its own stream driven by its own host thread. */
typedef struct hbpc_batch hbpc_batch;
hbpc_status hbpc_batch_create(hbpc_batch** out, int n_inst, const hbpc_mesh* meshes, const int* N, int nodes,
                              const hbpc_physics* phys, const hbpc_solver* solver, int max_per_group);
void hbpc_batch_destroy(hbpc_batch* b);                       /* accepts NULL */
int hbpc_batch_groups(const hbpc_batch* b);                   /* number of distinct N */
long long hbpc_batch_ndof(const hbpc_batch* b, int inst);     /* -1 for a bad index */
/* State of instance `inst` (canonical layout of that instance alone); host
 * memory unless on_device != 0. */
hbpc_status hbpc_batch_set_state(hbpc_batch* b, int inst, const double* w, int on_device);
hbpc_status hbpc_batch_get_state(hbpc_batch* b, int inst, double* w, int on_device);
/* Node coordinates of instance `inst`, host x[dim][n_E][(N+1)^dim]. */
hbpc_status hbpc_batch_node_coords(hbpc_batch* b, int inst, double* x);
/* R1 (Eq. 12, with the viscous term) of the current state of inst's group,
 * instance `inst`'s part copied to host r. */
hbpc_status hbpc_batch_eval_R1(hbpc_batch* b, int inst, double* r);
/* n_steps HBPC steps of every instance. */
hbpc_status hbpc_batch_step(hbpc_batch* b, int n_steps);
/* hbpc_set_step_graph for every group: each group's step is one graph launch. */
hbpc_status hbpc_batch_set_step_graph(hbpc_batch* b, int on);
/* hbpc_set_pc_rebuild for every group. */
hbpc_status hbpc_batch_set_pc_rebuild(hbpc_batch* b, int every_newton_iteration);
/* Counters summed over groups (steps, t: the maximum). */
hbpc_status hbpc_batch_get_stats(const hbpc_batch* b, hbpc_stats* out);
hbpc_status hbpc_batch_profile_enable(hbpc_batch* b, int enable);
/* hbpc_autotune for every group; out: n_out >= hbpc_batch_groups entries or NULL. */
hbpc_status hbpc_batch_autotune(hbpc_batch* b, hbpc_tuning* out, int n_out);
/* Message of the last failure of the batch (NULL: of the last failed create). */
const char* hbpc_batch_last_error(const hbpc_batch* b);

/* Message of the last failure on this context (static storage owned by the
 * context; "" if none).  Accepts NULL (returns the message of the last failed
 * hbpc_create). */
const char* hbpc_last_error(const hbpc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* HBPC_H */
