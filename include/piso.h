/*
 * piso.h - C ABI of the B300 (sm_103a) per-time-step PISO update.
 *
 * The library implements one time step of the incompressible collocated
 * finite-volume PISO scheme on structured multi-block grids with coordinate
 * transforms described in arXiv:2505.16992 (PICT), Sec. 2.1-2.3 and App. A:
 * assembly of the advection-diffusion matrix C = A + H, a BiCGStab predictor
 * solve (optionally ILU(0)-preconditioned, App. A.5), n pressure correctors
 * (divergence of h, preconditioned CG on the pressure matrix P: Jacobi or
 * y-line blocks, velocity correction), block-interface and boundary handling,
 * and the discrete adjoint of that step; plus the turbulence-statistics
 * operators of Sec. 2.5 (plane records, their merge and adjoint, budgets).
 *
 * Conventions (shared by every entry point):
 *   - Sides 0..5 = -x, +x, -y, +y, -z, +z (2D uses 0..3).
 *   - A block of resolution (nx, ny, nz) (nz = 1 in 2D) owns cells with local
 *     index x + nx*(y + ny*z); the domain index of a cell is the sum of the
 *     cell counts of the blocks added before it plus its local index.
 *   - Fields are structure-of-arrays in DEVICE memory: a velocity-like field
 *     is ndim arrays of N values back to back (component-major, [c][i]); a
 *     pressure-like field is N values.  The element type is double for
 *     PISO_FP64 and float for PISO_FP32.  The caller owns every field buffer;
 *     the library never retains a field pointer past the call that received it.
 *   - Values on a block side are given per boundary face, ordered by the two
 *     tangential cell indices with the lower axis fastest (x-sides: y then z;
 *     y-sides: x then z; z-sides: x then y), each face carrying ndim values
 *     (row-major [face][component], host memory, double).
 *   - Every call returns a piso_status; nothing aborts or traps.  On an error
 *     the outputs are unspecified, the inputs are untouched, and
 *     piso_last_error() describes the failure.
 *   - Device work is enqueued on the caller's CUDA stream (a cudaStream_t
 *     passed as void*, NULL = legacy default stream).
 */
#ifndef PISO_H
#define PISO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct piso_domain piso_domain;
typedef struct piso_batch piso_batch;

typedef enum {
  PISO_OK = 0,
  PISO_EINVAL = 1,      /* bad argument or domain description */
  PISO_ECUDA = 2,       /* a CUDA runtime call failed */
  PISO_ENOCONV = 3,     /* a Krylov solve hit its iteration limit (stats hold the counts) */
  PISO_EBREAKDOWN = 4,  /* a Krylov solve broke down (zero denominator) */
  PISO_ENAN = 5,        /* a residual became NaN */
  PISO_ETIMEOUT = 6,    /* a group barrier wait ran out (the step was abandoned) */
  PISO_ESTATE = 7,      /* call out of order (e.g. step before finalize) */
  PISO_ENOMEM = 8       /* device allocation failed */
} piso_status;

typedef enum {
  PISO_FP64 = 0,        /* double storage and arithmetic */
  PISO_FP32 = 1         /* float storage and stencil arithmetic; Krylov dot products and
                           norms accumulated with ~48-bit (float-pair) sums and reduced
                           across CTAs in double */
} piso_precision;

/* Solver options (App. A.1: two correctors; App. A.5: CG for the pressure,
 * BiCGStab for advection-diffusion).  Convergence: ||r||_2 <=
 * max(rtol * ||b||_2, atol) for each solve. */
typedef struct {
  int32_t n_correctors;  /* 1..4, default 2 */
  int32_t pred_grad_p;   /* 0 (default): predictor right-hand side of Eq. velRHSdiscrete;
                            1: add -grad p^n (Eq. advectionMat; unstable on anisotropic cells) */
  double adv_rtol;       /* BiCGStab relative tolerance */
  double p_rtol;         /* CG relative tolerance */
  double atol;           /* absolute tolerance for both */
  int32_t adv_maxit;     /* BiCGStab iteration limit */
  int32_t p_maxit;       /* CG iteration limit per corrector */
  int32_t block_threads; /* threads per CTA (multiple of 32, <= 768); 0 = 512 (see piso_autotune) */
  int32_t ctas;          /* CTAs for this domain; 0 = auto (one per SM, capped by size) */
  double timeout_s;      /* group-barrier wait limit in seconds (default 5) */
  int32_t fault_withhold_cta; /* fault injection for tests: this CTA of the domain skips its
                                 first barrier arrival, so every wait of the step runs out and
                                 the call returns PISO_ETIMEOUT; -1 (default) = off */
  double p_refine_rtol;  /* PISO_FP32 only: > 0 refines every pressure solve against a residual
                            b - P p evaluated in FP64 with the solution accumulated in FP64,
                            until ||b - P p|| <= p_refine_rtol ||b|| (each round an FP32 CG to
                            p_inner_rtol); 0 (default) = a single FP32 CG to p_rtol, finished
                            by such rounds (to p_rtol) only if it stalls */
  double p_inner_rtol;   /* inner tolerance per refinement round (default 1e-4) */
  int32_t grad_paths;    /* gradient paths kept by piso_step_adjoint (Sec. 2.4, Eq. jnone): a bit
                            set of PISO_GRAD_ADV and PISO_GRAD_P, default both (the exact adjoint).
                            A path left out treats that solve's output (u*, or every corrector's
                            pressure) as a constant of the backward pass, so its transposed solve
                            is skipped; 0 keeps only the bypass paths.  The forward step ignores it. */
  int32_t p_precond;     /* preconditioner of the pressure CG (the paper names none; App. A.5 uses a
                            plain CG): PISO_PRECOND_AUTO (default) picks the y-line preconditioner
                            when the grid is anisotropic in y (some cell with alpha_yy >= 4 alpha_kk,
                            k != y, as on wall-refined channels) and Jacobi otherwise;
                            PISO_PRECOND_JACOBI; PISO_PRECOND_LINE: the block diagonal of -P made of
                            its y-lines inside each block, solved exactly (Thomas factors formed once
                            per step; see p_line_split for how its CG iteration synchronises).
                            In batches (piso_batch_*) a member runs the line form only when its
                            options say PISO_PRECOND_LINE (a choice PISO_PRECOND_AUTO made from
                            the grid is not carried over: in a batch the line form needs
                            launch-wide staging for two of the longest such lines and runs split,
                            measured slower than Jacobi there); without room every member uses
                            Jacobi. */
  int32_t adv_precond;   /* preconditioner of the advection-diffusion BiCGStab (App. A.5: incomplete
                            LU, for grids with strongly varying cell sizes, enabled per case, and
                            optionally only after the plain solve failed):
                            PISO_ADV_PRECOND_NONE (default);
                            PISO_ADV_PRECOND_ILU: right-preconditioned by zero-fill ILU of C, the
                            factorisation formed once per step (the adjoint forms it again from the
                            recorded C and applies its transpose to the transposed solve);
                            PISO_ADV_PRECOND_ILU_ON_FAILURE: the plain BiCGStab first, and, if some
                            component did not converge (iteration limit, breakdown or NaN), a restart
                            from the same initial guess with the ILU preconditioner; the reported
                            iterations count both attempts.
                            Each CTA factors the diagonal block of C formed by the cells it owns
                            (couplings between CTAs are left out of the preconditioner only), so the
                            triangular solves need no grid-wide synchronisation; with ctas = 1 this
                            is ILU(0) of the whole matrix in cell order.  The level tables are built
                            on the host whenever the launch layout changes (finalize, set_options,
                            autotune).  Batches reject any value but NONE (PISO_EINVAL). */
  int32_t n_nonortho;    /* non-orthogonal meshes (App. A.2 "Non-Orthogonal Grids"): 0 (default)
                            rejects blocks whose cross metrics alpha_jk = J T_j . T_k (j != k) do
                            not vanish; 1..4 accepts them.  The cross derivatives of the viscous
                            term are split as Eq. difNonOrthoMatDiscrete and Eq. velRHSnonOrtho
                            state: the terms on a cell's direct neighbours join the matrix C, those
                            on its diagonal neighbours go to the right-hand side with the previous
                            iterate (the predictor's, each corrector's input velocity); the cross
                            derivatives of the pressure operator go to the right-hand side whole
                            with the previous pressure iterate (Eq. pressureRHSnonOrtho; P stays
                            symmetric for the CG); every predictor and pressure solve is repeated
                            n times (non-orthogonal corrector steps).  piso_step_adjoint runs those
                            loops in reverse (p^n then receives a gradient through the pressure
                            cross terms); the step record holds the iterates, hence the limit 4.
                            Batches and pred_grad_p = 1 reject such meshes (PISO_EINVAL).
                            Ignored on orthogonal meshes. */
  int32_t p_line_split;  /* how a y-line preconditioned CG iterates.  0 (default): with one group
                            barrier per iteration wherever every CTA of the launch can hold its own
                            lines and the lines next to them (halo lines) in shared memory: each
                            CTA then also solves its halo lines, so w = A u needs no second
                            barrier (the same recurrences; results differ from the split form
                            only by rounding).  1: always two barriers per iteration (a line phase,
                            then w = A u).  Domains whose lines do not fit, and batches, use the
                            split form; piso_pressure_line_fused reports which one a domain runs. */
} piso_options;

/* Values of piso_options.p_precond. */
#define PISO_PRECOND_AUTO 0
#define PISO_PRECOND_JACOBI 1
#define PISO_PRECOND_LINE 2

/* Values of piso_options.adv_precond. */
#define PISO_ADV_PRECOND_NONE 0
#define PISO_ADV_PRECOND_ILU 1
#define PISO_ADV_PRECOND_ILU_ON_FAILURE 2

/* Bits of piso_options.grad_paths. */
#define PISO_GRAD_ADV 1   /* paths through the advection (predictor) solve */
#define PISO_GRAD_P 2     /* paths through the pressure solves */

/* Per-step statistics (read back when a stats pointer is given). */
typedef struct {
  int32_t status;         /* piso_status of the step */
  int32_t error_bits;     /* 1 adv no-conv, 2 pressure no-conv, 4 breakdown, 8 NaN, 16 timeout */
  int32_t adv_iters[3];   /* BiCGStab iterations per velocity component */
  int32_t p_iters[4];     /* CG iterations per corrector (all rounds) */
  double adv_resid[3];    /* final BiCGStab residual norms */
  double p_resid[4];      /* final CG residual norms (the FP64 outer residual when refining) */
  int32_t p_rounds[4];    /* FP64 refinement rounds per corrector: 0 for a plain CG; a plain FP32
                             CG that stalled (its best residual norm did not halve in 200
                             iterations) and was finished by refinement counts as round 1 */
  double p_rhs_norm[4];   /* norm of each pressure solve's (projected) right-hand side */
  int32_t adv_precond_used; /* the BiCGStab ran ILU-preconditioned: 0 no, 1 from the start,
                               2 after the plain attempt failed (PISO_ADV_PRECOND_ILU_ON_FAILURE) */
  /* on non-orthogonal meshes adv_iters and p_iters sum the iterations of all
     non-orthogonal corrector steps */
} piso_stats;

/* Fill *o with the defaults listed above. */
void piso_default_options(piso_options* o);

/* Create an empty domain of dimension ndim (2 or 3) and precision prec.
 * Ownership of *out passes to the caller (release with piso_domain_destroy). */
piso_status piso_domain_create(int32_t ndim, int32_t prec, piso_domain** out);

/* Add a block (Sec. 2.2: a regular grid aligned to boundaries by a
 * precomputed transformation).  res = {nx, ny, nz} (nz = 1 in 2D); vertices is
 * HOST memory with (nz+1)(ny+1)(nx+1) points of ndim doubles, x fastest.
 * Metrics T = d xi / d x and J = det(d x / d xi) are formed at cell centres
 * from opposite face-centre differences (App. A.2 "Grid Transformations").
 * Grids whose cross metrics alpha_jk (j != k) do not vanish are rejected at
 * finalize unless piso_options.n_nonortho >= 1.  *block_id receives the
 * block's index. */
piso_status piso_block_add(piso_domain* d, const int32_t res[3], const double* vertices,
                           int32_t* block_id);

/* Join side sa of block a to side sb of block b, cell to cell (Sec. 2.2: a
 * conformal connection with matching resolution; App. A.3: it only changes the
 * neighbour lookup; App. B: the cuts of O- and C-grids).  Any two sides may be
 * joined.  The tangential axes of a side are its other axes in ascending order
 * (2D: one; 3D: two); the i-th tangential axis of sa runs along tangential axis
 * (axis_perm ? 1 - i : i) of sb (axis_perm is 0 in 2D), reversed when bit i of
 * flip_mask is set.  a == b with opposite sides and (0, 0) gives a periodic
 * direction; a side joined to itself (a == b, sa == sb) is a fold, e.g. the cut
 * of a C-grid, and needs a reversed axis of even length (no cell may meet
 * itself).  The neighbour across a joint that exchanges or reverses axes keeps
 * its own frame: its fluxes, metrics and differences are read through it, such
 * domains run the extended kernel instantiation and the pressure CG uses the
 * Jacobi preconditioner.  PISO_EINVAL for mismatched resolutions or out-of-
 * range axis_perm / flip_mask. */
piso_status piso_connect(piso_domain* d, int32_t a, int32_t sa, int32_t b, int32_t sb, int32_t axis_perm,
                         int32_t flip_mask);

/* Dirichlet velocity on a block side (App. A.3: values live on the face;
 * pressure is implicitly zero-Neumann there).  values: HOST, [face][ndim]. */
piso_status piso_set_dirichlet(piso_domain* d, int32_t blk, int32_t side, const double* values);

/* Advective (non-reflecting) outflow on a block side (App. A.3, Eq. advOut):
 * before every step each face value moves towards its cell value with the
 * factor c/(1+c), c = 2 dt |T_j . u_m|, and all outflow faces are then scaled
 * so the outflow balances the inflow; during the step the side acts as a
 * Dirichlet side.  u_m: HOST ndim doubles; values: HOST initial face values. */
piso_status piso_set_advective_outflow(piso_domain* d, int32_t blk, int32_t side,
                                       const double* u_m, const double* values);

/* Validate the description, build metrics and connection tables, upload them
 * and allocate the workspace.  opts may be NULL (defaults).  No further
 * blocks or boundaries may be added afterwards. */
piso_status piso_finalize(piso_domain* d, const piso_options* opts);

/* Replace the solver options of a finalized domain (launch shape included). */
piso_status piso_set_options(piso_domain* d, const piso_options* opts);

/* Copy the domain's current options to *opts (host), e.g. after piso_autotune. */
piso_status piso_get_options(const piso_domain* d, piso_options* opts);

/* The pressure preconditioner the domain's next step uses (PISO_PRECOND_JACOBI
 * or PISO_PRECOND_LINE; PISO_PRECOND_AUTO resolved from the grid), or -1 for a
 * NULL or unfinalized domain. */
int32_t piso_pressure_precond(const piso_domain* d);

/* 1 when the domain's next step runs its y-line preconditioned CG in the
 * fused form (one group barrier per iteration; see p_line_split), 0 when it
 * runs the split form or the Jacobi CG, -1 for a NULL or unfinalized domain.
 * The plan behind the fused form (own and halo lines per CTA, neighbour slots)
 * is built on the host whenever the launch layout changes. */
int32_t piso_pressure_line_fused(const piso_domain* d);

/* 1 when the domain's next step runs its Jacobi CG sweep on four consecutive
 * cells per thread with vector loads and stores (every block's nx a multiple
 * of 4, no joint that exchanges or reverses axes, and cells walked in passes
 * interleaved over the CTAs because a CTA's range exceeds its shared-memory
 * neighbour table), 0 when it runs one cell per thread or another
 * preconditioner, -1 for a NULL or unfinalized domain.  Both forms compute
 * the same iterates up to the summation order of the dot products. */
int32_t piso_pressure_cg_vec4(const piso_domain* d);

int64_t piso_num_cells(const piso_domain* d);
int32_t piso_num_boundary_faces(const piso_domain* d);

/* Bytes of a tape: the intermediates one forward step records for its adjoint
 * (u^n, C, u*, and per corrector h, the pressure and the corrected velocity,
 * plus the boundary values used).  Device memory, caller-owned. */
size_t piso_tape_bytes(const piso_domain* d);

/* One PISO step (App. A.1): u_out, p_out <- step(u_in, p_in, dt, nu, S).
 * u_in/u_out: device [ndim][N]; p_in/p_out: device [N]; u_out may alias u_in
 * and p_out may alias p_in.  S: device [ndim][N] per-unit-volume source, or
 * NULL.  The returned pressure has zero mean.  tape: device buffer of
 * piso_tape_bytes() that receives this step's intermediates, or NULL to keep
 * them in the domain's own workspace (valid until the next step).  Advective
 * outflow faces of the domain are updated in place.  If stats is non-NULL the
 * call waits for the step and fills it; otherwise it returns after enqueueing
 * (read the outcome later with piso_last_stats). */
piso_status piso_step(piso_domain* d, const void* u_in, const void* p_in, void* u_out,
                      void* p_out, double dt, double nu, const void* S, void* tape,
                      void* stream, piso_stats* stats);

/* Launch-shape autotuner (no counterpart in the paper; a B300 execution
 * choice): time one forward step of the given state (device u, p, S as for
 * piso_step; the inputs are not modified and the outflow boundary state is
 * restored) for each candidate shape - CTA width 512 or 768 threads, CTA count
 * one per SM or one cell per thread, and, when p_precond is PISO_PRECOND_AUTO
 * on a y-anisotropic grid, both pressure preconditioners - and make the
 * fastest the domain's shape (its options then name the chosen preconditioner
 * explicitly; read them with piso_get_options).  Results are cached per
 * process by (ndim, precision, cells, blocks, correctors, p_precond).
 * threads_out, ctas_out, ms_out (host, may be NULL) receive the choice and its
 * time (-1 when it came from the cache).  Synchronises the stream. */
piso_status piso_autotune(piso_domain* d, const void* u, const void* p, double dt, double nu, const void* S,
                          void* stream, int32_t* threads_out, int32_t* ctas_out, double* ms_out);

/* Forward step that allocates nothing (the paper has no counterpart; this is
 * a service of this library).  Some callers cannot allocate device memory at
 * the time they step - for example a process whose device memory is already
 * fully reserved by another framework's caching allocator, or a
 * latency-critical loop that must not risk an allocation or its failure
 * mid-run.  piso_step_static computes the same step as piso_step (same
 * arguments except the tape, same kernel, same results), but its scratch -
 * the workspace, the step record and the control words - lives in one fixed
 * 32 MiB buffer compiled into this library (every GPU that loads the library
 * holds it until the process exits), not in memory from cudaMalloc.  The
 * caller still provides the inputs and outputs.
 *   - Size limit: domains whose scratch exceeds 32 MiB are rejected with
 *     PISO_EINVAL and a message giving the bytes needed (about 43,000 cells
 *     for a 3D FP64 domain, 87,000 for 3D FP32, more in 2D).
 *   - Set-up: the first call on each device looks up the buffer's device
 *     address with that device current; make that first call before any
 *     stream capture.
 *   - Sharing: every call (every domain, every stream) uses the same buffer,
 *     which keeps the last call's contents; calls that overlap on the GPU
 *     race and corrupt each other's results.
 *   - The step record lives in the shared buffer: piso_step_adjoint cannot use
 *     it, and a piso_step_adjoint with tape NULL after this call returns
 *     PISO_ESTATE (run piso_step, with the domain's own workspace, before an
 *     adjoint).
 *   - Advective outflow faces of the domain are updated as by piso_step. */
piso_status piso_step_static(piso_domain* d, const void* u_in, const void* p_in, void* u_out, void* p_out,
                             double dt, double nu, const void* S, void* stream, piso_stats* stats);

/* Wait for the last enqueued step (or adjoint) of the domain and report it. */
piso_status piso_last_stats(piso_domain* d, piso_stats* stats);

/* Adjoint of one step (Sec. 2.3, App. A.4): given du_out = dL/du^{n+1} and
 * dp_out = dL/dp^{n+1} (device; dp_out may be NULL for zero), write
 * du_in = dL/du^n, dp_in = dL/dp^n, dS = dL/dS (each device, caller-owned,
 * may be NULL to skip) and *dnu = dL/dnu (host double, may be NULL).
 * tape is the buffer filled by the forward step, or NULL for the domain's own
 * record of its last forward step; that record exists only when the last
 * forward step of the domain was a piso_step with tape NULL (or a batch step),
 * otherwise (no step yet, or after piso_step_static, piso_autotune or a
 * piso_step into a caller tape) a NULL tape returns PISO_ESTATE.  Linear solves are differentiated by transposed
 * solves (C^T via BiCGStab, P symmetric via CG).  Boundary velocities are
 * differentiable too (App. A.4): dL/d(boundary values before the step's
 * advective-outflow update) is kept in the domain (read it with
 * piso_get_boundary_adjoint), and the outflow update (Eq. advOut) is
 * differentiated, so du_in includes the path through the outflow faces. */
piso_status piso_step_adjoint(piso_domain* d, const void* tape, const void* du_out,
                              const void* dp_out, void* du_in, void* dp_in, void* dS,
                              double* dnu, void* stream, piso_stats* stats);

/* Copy the domain's current boundary-face values (device, [ndim][nbf]) to the
 * host array values ([ndim][nbf] doubles), or set them from it. */
piso_status piso_get_boundary(piso_domain* d, double* values);
piso_status piso_set_boundary(piso_domain* d, const double* values);

/* dL/d(boundary-face values) computed by the domain's last piso_step_adjoint
 * (or batch adjoint), with respect to the values the step started from (before
 * its advective-outflow update): host [ndim][nbf] doubles, the face order of
 * piso_set_dirichlet.  Synchronises with the device. */
piso_status piso_get_boundary_adjoint(piso_domain* d, double* values);

/* Last error message of the domain (or of the most recent failing creation
 * call when d is NULL).  The string is owned by the library. */
const char* piso_last_error(const piso_domain* d);

/* Release the domain and its device memory. */
void piso_domain_destroy(piso_domain* d);

/* ---- batches: independent simulations of uneven size in one launch ----
 * Each domain keeps its own CTA group, barrier and Krylov scalars; groups
 * run to their own convergence inside one persistent launch.  All domains
 * must share ndim and precision and be finalized. */
piso_status piso_batch_create(piso_domain* const* domains, int32_t n, const piso_options* opts,
                              piso_batch** out);

/* One step of every domain: arrays of n device pointers / values. */
piso_status piso_batch_step(piso_batch* b, const void* const* u_in, const void* const* p_in,
                            void* const* u_out, void* const* p_out, const double* dt,
                            const double* nu, const void* const* S, void* stream,
                            piso_stats* stats);

piso_status piso_batch_step_adjoint(piso_batch* b, const void* const* du_out,
                                    const void* const* dp_out, void* const* du_in,
                                    void* const* dp_in, void* const* dS, double* dnu,
                                    void* stream, piso_stats* stats);

/* Launch-shape autotuner of a batch (no counterpart in the paper; a B300
 * execution choice): times one forward step of the given state (arrays of n
 * device pointers / values as for piso_batch_step; the inputs are not modified
 * and the members' boundary values are restored) with CTAs of 512 and 768
 * threads, with all co-resident CTAs and with three quarters of them (each
 * layout apportioned by estimated work), keeps the fastest, then balances its
 * split by measured work: each member's forward and adjoint steps are timed
 * alone on the CTA count the layout gives it, the CTAs are re-apportioned in
 * proportion to time x CTAs, and the new split is kept while the batch's
 * forward + adjoint launches get faster (two rounds).  The result holds for
 * the batch's later launches.  threads_out, ctas_out, ms_out (host, may be
 * NULL) receive the shape and the forward-launch time of the kept layout.
 * Allocates trial outputs; synchronises the stream; the members' step records
 * are left invalid (run a batch step before an adjoint). */
piso_status piso_batch_autotune(piso_batch* b, const void* const* u_in, const void* const* p_in, const double* dt,
                                const double* nu, const void* const* S, void* stream, int32_t* threads_out,
                                int32_t* ctas_out, double* ms_out);

void piso_batch_destroy(piso_batch* b);

/* ---- turbulence statistics (Sec. 2.5 "Operators for Turbulence Statistics";
 * Sec. 3.3 "Losses from Turbulence Statistics") ----
 * A record holds, for every plane y = const of a single-block domain (the
 * homogeneous directions are x and, in 3D, z), in doubles:
 *   [n, mean[nq], m2[nq][nq], m3[nq][nq][nq] (order 3 only)]
 * with n the number of samples, mean_i = (1/n) sum q_i and the central moments
 * m2_ij = (1/n) sum a_i a_j, m3_ijk = (1/n) sum a_i a_j a_k, a = q - mean; a
 * domain's records are [ny][record_size] arrays in DEVICE memory, caller-owned.
 * Averaging over time is merging frame records (an online pairwise update), so
 * no frame needs to be stored.  Every call enqueues on the stream and returns
 * a status; errors name the violated condition via piso_last_error(domain). */
typedef struct piso_plane_stats piso_plane_stats;

/* Statistics of nq per-cell fields (nq <= 12) up to order 2 or 3 (order 3
 * needs nq <= 4) on a finalized single-block domain.  Ownership of *out passes
 * to the caller (release with piso_stats_destroy). */
piso_status piso_stats_create(piso_domain* d, int32_t nq, int32_t order, piso_plane_stats** out);

/* Doubles per plane of a record, and the number of planes (ny); -1 for NULL. */
int32_t piso_stats_record_size(const piso_plane_stats* s);
int32_t piso_stats_planes(const piso_plane_stats* s);

/* Record of one frame: q DEVICE [nq][N] in the domain's storage precision ->
 * rec (device [ny][record_size]).  If acc is non-NULL it is merged with the
 * frame (acc <- merge(acc, rec)); an acc plane with n = 0 starts empty.  Each
 * plane is split over several CTAs whose partial records (in a scratch buffer
 * of the statistics object: calls on one object must not overlap on the GPU)
 * are merged in a fixed order, so results are deterministic. */
piso_status piso_stats_frame(piso_plane_stats* s, const void* q, double* rec, double* acc, void* stream);

/* a <- merge(a, b): the record of the union of both sample sets, per plane. */
piso_status piso_stats_merge(piso_plane_stats* s, double* a, const double* b, void* stream);

/* Adjoint of a record with respect to one frame's fields: dq += (d rec / d q)^T
 * grad, with q the frame (device [nq][N]), rec its record or an accumulated
 * record that contains it (then the derivative is that of the accumulated
 * statistics with respect to this frame's samples), grad = dL/d(rec) in the
 * record layout (the n entries are ignored), dq device [nq][N] accumulated. */
piso_status piso_stats_frame_adjoint(piso_plane_stats* s, const void* q, const double* rec, const double* grad,
                                     void* dq, void* stream);

/* Cell-centred gradients of the velocity and pressure (the central
 * differences of Eq. velCorrDiscrete mapped with T): grad_u [ndim][ndim][N]
 * with grad_u[i][k] = d u_i / d x_k, grad_p [ndim][N] (device, storage
 * precision, either may be NULL).  At Dirichlet faces the missing neighbour is
 * the ghost 2 u_b - u_P for the velocity and p_P for the pressure. */
piso_status piso_cell_gradients(piso_domain* d, const void* u, const void* p, void* grad_u, void* grad_p,
                                void* stream);

/* Turbulent energy budget per plane from three records of one domain: rec_u
 * of the velocity (nq = ndim, order 3), rec_g of its gradient (nq = ndim^2,
 * field i*ndim + k = d u_i / d x_k) and rec_p of (u, grad p) (nq = 2 ndim):
 * out (device [5][ny][ndim][ndim] doubles) = production
 * -(R_ik dU_j/dx_k + R_jk dU_i/dx_k), dissipation 2 nu <d_k u_i' d_k u_j'>,
 * turbulent transport -d<u_i' u_j' v'>/dy, viscous diffusion nu d^2 R_ij/dy^2,
 * velocity pressure-gradient -(<u_i' d_j p> + <u_j' d_i p>).  y-derivatives of
 * the profiles use three-point formulas on {-y side, plane centres, +y side}
 * with zero values at the sides (no-slip walls). */
piso_status piso_stats_budget(const piso_plane_stats* su, const double* rec_u, const piso_plane_stats* sg,
                              const double* rec_g, const piso_plane_stats* sp, const double* rec_p, double nu,
                              double* out, void* stream);

void piso_stats_destroy(piso_plane_stats* s);

/* Library version string. */
const char* piso_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PISO_H */
