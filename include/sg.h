/*
 * sg.h -- C ABI of the GB300 (sm_103a) initial-guess / SEM / Jacobi-PCG library.
 *
 * Method: Austin, Chalmers & Warburton, "Initial Guesses for Sequences of
 * Linear Systems in a GPU-Accelerated Incompressible Flow Solver"
 * (arXiv:2009.10863).  The problem (Sec. 2) is a sequence A x_k = b_k of SPD
 * systems, one per time step; each is solved by preconditioned CG (Sec. 5.3)
 * from an initial guess built from earlier solutions by right-hand-side
 * projection (Sec. 2, Algorithms 1-2) or by polynomial extrapolation (Sec. 3).
 *
 * Conventions for every entry point:
 *  - Vectors are DEVICE pointers to contiguous arrays of n = sg_op_size(op)
 *    elements of the handle's dtype (SG_F64: double, SG_F32: float), owned by
 *    the caller.  They must be 16-byte aligned.  Global node g of an
 *    ex*ey*ez-element mesh of degree p is g = ix + nx*(iy + ny*iz),
 *    nx = p*ex + 1 (x fastest).
 *  - Workspaces are DEVICE buffers owned by the caller, sized by the matching
 *    *_workspace_bytes() query, 256-byte aligned, and must outlive the handle
 *    (guess) or the call (PCG).  The library allocates only the small
 *    per-operator coefficient tables (sg_op_create, < 8 KB), the instantiated
 *    PCG iteration graphs it caches on an operator (at most 8 per operator,
 *    released by sg_op_destroy) and one pinned host word per host thread for
 *    convergence polls.
 *  - A handle is used by one host thread at a time; different handles may be
 *    used concurrently.
 *  - ``stream`` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call is stream-ordered and asynchronous unless stated.
 *  - Return value: SG_OK (0) on success, SG_NOT_CONVERGED (1) as a warning,
 *    a negative SG_ERR_* code on failure.  On failure handle state is left
 *    unchanged and sg_last_error() returns a message (thread-local).  Errors
 *    are reported, never trapped on the device.
 *  - Dirichlet conditions hold on all six faces of the unit box: the operator
 *    ignores boundary entries of its input and writes 0 there.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_op_s* sg_op_t;
typedef struct sg_guess_s* sg_guess_t;
typedef struct sg_batch_s* sg_batch_t;

enum sg_dtype { SG_F64 = 0, SG_F32 = 1 };

/* Guess methods (Sec. 4, Table 1 nomenclature). */
enum sg_method {
  SG_ZERO = 0,          /* x0 = 0                                            */
  SG_LAST = 1,          /* x0 = x_{k-1} (degree-0 extrapolation, Sec. 3.1)   */
  SG_EXTRAP = 2,        /* EXTRAP(m, s): least squares, Eq. LSQRCoeffs       */
  SG_PROJ_QR = 3,       /* QR(s): rolling-QR projection, Algorithm 2         */
  SG_PROJ_CLASSIC = 4,  /* CLASSIC(s): restarted projection, Algorithm 1     */
  SG_SPEXTRAP = 5,      /* SPEXTRAP(m, s): sparse, Eq. CPQRCoeffs            */
  SG_PROJ_ENERGY = 6    /* ENERGY(s): the rolling window of QR(s) in the
                           energy inner product -- X~ A-orthonormal, guess
                           x0 = X~ X~^T b minimising ||x - A^{-1} b||_A over
                           the span (Sec. 2's projection in Fischer's norm);
                           CGS2 coefficients X~^T (A x), ||x~||_A, same
                           Givens downdate, acceptance ||x~||_A > eps_rel
                           ||x_k||_A.  No counterpart among the paper's
                           Algorithms 1-2, which use the Euclidean form.   */
};

/* PCG stopping rules (Sec. 6.4). */
enum sg_criterion {
  SG_STOP_REL_B = 0,      /* ||r|| <= tol * ||b||                            */
  SG_STOP_INITRESID = 1,  /* ||r|| <  tol * max(||r0||, 1), Eq. StopCritINITRESID */
  SG_STOP_RHS = 2         /* ||r|| <  tol * max(||b||, 1),  Eq. StopCritRHS  */
};

enum sg_status {
  SG_OK = 0,
  SG_NOT_CONVERGED = 1,   /* PCG hit maxit; x holds the last iterate        */
  SG_ERR_INVALID = -1,    /* bad argument (size, alignment, dtype, range)    */
  SG_ERR_CUDA = -2,       /* a CUDA runtime call failed                      */
  SG_ERR_BREAKDOWN = -3,  /* PCG: p^T A p <= 0 or a non-finite value         */
  SG_ERR_TIMEOUT = -4,    /* a bounded device-side wait expired              */
  SG_ERR_STATE = -5       /* call not valid for this handle/method           */
};

#define SG_MAX_HISTORY 16 /* largest history size s                         */
#define SG_MAX_DEGREE 8   /* largest GLL degree p                           */
#define SG_BATCH_MAX 4    /* largest number of systems in one batch         */

int sg_version(void);
const char* sg_last_error(void);

/* ------------------------------------------------------------------------
 * Operator: matrix-free GLL spectral-element A = K + lambda*M on the unit
 * box split into ex*ey*ez equal axis-aligned hexahedra, degree p
 * (Sec. 5.1; Helmholtz form of Eq. VelocityEqn, Poisson form of Eq.
 * PressureEqn with lambda = 0).  K is the GLL-quadrature stiffness matrix,
 * M the diagonal GLL mass matrix, both assembled by gather-scatter.
 * ------------------------------------------------------------------------ */

/* Create an operator.  1 <= p <= SG_MAX_DEGREE, ex,ey,ez >= 1, lambda >= 0,
 * dtype SG_F64 or SG_F32 (arithmetic and storage type of sg_sem_apply and
 * sg_pcg_solve).  Allocates < 8 KB of device tables (the operator kernel's
 * coefficients) on the current device.  On a host without a CUDA device it
 * allocates nothing; the handle then answers sg_op_size and sg_op_gll, and
 * every launch through it returns SG_ERR_STATE. */
int sg_op_create(sg_op_t* op, int ex, int ey, int ez, int p, double lambda, int dtype);
/* Element layers in z that one CTA of the operator kernel marches through
 * (a tuning and testing knob of the tiled operator of Sec. 5.1): zl >= 1
 * fixes it (clamped to ez), 0 restores the automatic choice (about 8 CTAs per
 * SM).  Results agree to rounding for every zl.  Drops the PCG graphs cached
 * on the operator.  SG_ERR_INVALID for a NULL handle or zl < 0. */
int sg_op_set_layers(sg_op_t op, int zl);
int sg_op_destroy(sg_op_t op);
/* n = (p*ex+1)(p*ey+1)(p*ez+1); returns -1 for a NULL handle. */
int64_t sg_op_size(sg_op_t op);
/* Host copies of the 1D GLL nodes and weights on [-1,1] (p+1 each). */
int sg_op_gll(sg_op_t op, double* nodes, double* weights);

/* y = A x (Sec. 5.1).  x, y: device, n elements, must not alias. */
int sg_sem_apply(sg_op_t op, const void* x, void* y, void* stream);

/* diag(A) with 1 on Dirichlet nodes (the Jacobi preconditioner, Sec. 5.3). */
int sg_op_diagonal(sg_op_t op, void* diag, void* stream);

/* ------------------------------------------------------------------------
 * Jacobi-preconditioned CG (Sec. 5.3) with the stopping rules of Sec. 6.4.
 * ------------------------------------------------------------------------ */

/* Bytes of device workspace sg_pcg_solve needs for this operator. */
size_t sg_pcg_workspace_bytes(sg_op_t op);

/* Solve A x = b.  b: device input; x: device, initial guess on entry,
 * solution on exit (Dirichlet entries set to 0).  tol > 0, maxit >= 0,
 * criterion from sg_criterion.  workspace: device, sg_pcg_workspace_bytes.
 * iters, relres: HOST outputs (may be NULL) -- the iteration count and the
 * final true relative residual ||b - A x|| / ||b||; with relres NULL the
 * extra operator application that measures the true residual is skipped.
 * The call synchronises with ``stream`` once, at the end.  The iterations run
 * as one CUDA graph launch (a conditional WHILE node over the operator step and
 * the update, whose last block ends the loop on convergence, breakdown or
 * maxit), built on first use per (operator, workspace address) and cached on
 * the operator until sg_op_destroy.  While sg_profile_enable is on (each
 * kernel timed), or if graphs cannot be built, the host launches the
 * iterations in chunks and polls a done flag after each chunk.  Returns SG_OK,
 * SG_NOT_CONVERGED (maxit reached) or SG_ERR_BREAKDOWN. */
int sg_pcg_solve(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion,
                 void* workspace, int* iters, double* relres, void* stream);

/* The same solve, enqueued on ``stream`` without waiting: set-up kernels and
 * the iteration graph of sg_pcg_solve (no host poll, no synchronisation).  x
 * and b must stay valid until the stream reaches that point; the outcome is
 * read with sg_pcg_result on the same workspace before the next solve in it.
 * No counterpart in the paper (Sec. 5.3's PCG, launched asynchronously).
 * Returns SG_OK once enqueued, SG_ERR_INVALID, or SG_ERR_CUDA when the
 * iteration graph cannot be built. */
int sg_pcg_solve_async(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion,
                       void* workspace, void* stream);

/* Outcome of the last solve run in ``workspace``: iters (HOST, may be NULL);
 * synchronises with ``stream``.  Returns SG_OK, SG_NOT_CONVERGED or
 * SG_ERR_BREAKDOWN as sg_pcg_solve would have. */
int sg_pcg_result(sg_op_t op, void* workspace, int* iters, void* stream);

/* relres = ||b - A x|| / ||b|| (HOST output; Dirichlet entries ignored) using
 * a PCG workspace of this operator.  Synchronises with ``stream``. */
int sg_residual_norm(sg_op_t op, const void* b, const void* x, void* workspace, double* relres, void* stream);

/* ------------------------------------------------------------------------
 * Mixed precision: FP32 operator, PCG vectors and history wrapped in FP64
 * iterative refinement (the FP32 form of the operator of Sec. 5.1 and of the
 * PCG of Sec. 5.3, with the FP64 residual deciding convergence).
 * ------------------------------------------------------------------------ */

/* Element-wise conversion between FP64 and FP32 device vectors of n entries
 * (dst = (dst type) src).  src_dtype != dst_dtype. */
int sg_convert(const void* src, int src_dtype, void* dst, int dst_dtype, int64_t n, void* stream);

/* Workspace bytes for sg_ir_solve with this operator pair. */
size_t sg_ir_workspace_bytes(sg_op_t op64, sg_op_t op32);

/* Solve A x = b to ||b - A x|| <= tol ||b|| (FP64 residual).  op64 (SG_F64)
 * and op32 (SG_F32) must describe the same mesh, degree and lambda.  b, x:
 * FP64 device vectors (x: initial guess in, solution out; Dirichlet entries
 * set to 0).  Each outer step forms r = b - A x in FP64, solves A d = r with
 * FP32 Jacobi-PCG to ||r_inner|| <= t ||r|| (at most maxit_inner iterations,
 * from d = 0), t = min(0.1, max(inner_tol, tol ||b|| / (2 ||r||))) -- a step
 * is not solved tighter than the outer target needs -- and adds x += d in
 * FP64, until the FP64 residual
 * meets tol or max_outer steps were taken.  outer_iters, inner_iters (total
 * FP32 PCG iterations), relres: HOST outputs, may be NULL.  Synchronises
 * with ``stream`` once per outer step.  Returns SG_OK, SG_NOT_CONVERGED
 * (max_outer reached) or a negative error. */
int sg_ir_solve(sg_op_t op64, sg_op_t op32, const void* b, void* x, double tol, double inner_tol,
                int max_outer, int maxit_inner, void* workspace, int* outer_iters, int* inner_iters,
                double* relres, void* stream);

/* The same problem by one FP32 Jacobi-PCG whose residual is replaced by the
 * FP64 residual at reliable updates (residual replacement, van der Vorst & Ye
 * 2000; no counterpart in the paper, whose solver runs in FP64): whenever the
 * FP32 residual has dropped by t = min(0.1, max(delta, tol ||b|| / (2 ||r||)))
 * since the last update, x += x32 in FP64, r = b - A64 x, the FP32 residual
 * and preconditioned residual are reset from r and CG continues with its
 * search direction (beta from the replaced residual) instead of restarting.
 * Same operators, vectors, workspace (sg_ir_workspace_bytes) and errors as
 * sg_ir_solve.  max_updates bounds the FP64 updates, maxit_inner the FP32
 * iterations in total.  updates, inner_iters, relres: HOST outputs, may be
 * NULL.  Synchronises with ``stream`` once per update (once in all when the
 * guess already meets tol: the first inner solve is enqueued before the host
 * sees the initial residual and does no work then). */
int sg_ir_solve_ru(sg_op_t op64, sg_op_t op32, const void* b, void* x, double tol, double delta,
                   int max_updates, int maxit_inner, void* workspace, int* updates, int* inner_iters,
                   double* relres, void* stream);

/* ------------------------------------------------------------------------
 * Batched sequences.  The paper keeps one history space per velocity
 * component and one for the pressure (Sec. 6.1) and solves each system by
 * PCG (Sec. 5.3).  A batch advances up to SG_BATCH_MAX such systems -- each on
 * its own mesh, same degree p = 7, own lambda -- in one persistent cooperative
 * launch per CG iteration (operator work items of every system, a grid
 * barrier, vector updates of every system, a second barrier), replayed from a
 * CUDA graph, inside FP64 iterative refinement.  Histories/guesses stay per
 * system (sg_guess_* handles).
 * ------------------------------------------------------------------------ */

/* Workspace bytes for a batch of nseq systems (ops64[k]: SG_F64, ops32[k]:
 * SG_F32 operator of the same mesh and lambda, p = 7). */
size_t sg_batch_workspace_bytes(int nseq, const sg_op_t* ops64, const sg_op_t* ops32);
/* Create a batch on caller-owned workspace (zeroed here; synchronises). */
int sg_batch_create(sg_batch_t* b, int nseq, const sg_op_t* ops64, const sg_op_t* ops32, void* workspace);
int sg_batch_destroy(sg_batch_t b);
/* Autotuner: times candidate launch shapes (work-item depth in element layers
 * x CTAs per SM) on the batch and keeps the fastest.  Outputs (HOST, may be
 * NULL): the chosen depth, CTAs per SM and ms per persistent iteration.
 * Overwrites the batch's internal vectors; synchronises. */
int sg_batch_tune(sg_batch_t b, int* best_zl, int* best_blocks_per_sm, double* best_ms, void* stream);
/* Solve A_k x_k = b_k for every system k to ||b_k - A_k x_k|| <= tol ||b_k||
 * (FP64 residuals).  bvec[k], xvec[k]: FP64 device vectors (x: initial guess
 * in, solution out).  Per outer step: FP64 residual of every unconverged
 * system, one batched FP32 PCG solve (system k to the relative tolerance t_k
 * that sg_ir_solve uses, from its own residual), x += d.
 * outer_iters, inner_iters, relres: HOST arrays of nseq (may be NULL).
 * Synchronises.  Returns SG_OK, SG_NOT_CONVERGED, SG_ERR_TIMEOUT (a grid
 * barrier wait expired) or another negative error. */
int sg_batch_ir_solve(sg_batch_t b, const void* const* bvec, void* const* xvec, double tol, double inner_tol,
                      int max_outer, int maxit_inner, int* outer_iters, int* inner_iters, double* relres,
                      void* stream);

/* Self-test of the bounded device-side wait used by the batched kernel (no
 * counterpart in the paper): one cooperative launch of one CTA per SM passes
 * a grid barrier twice.  With extra_blocks > 0 the barrier waits for CTAs that
 * do not exist, so each wait gives up after spin_limit polls (~64 ns each),
 * records the expiry and returns; the call then returns SG_ERR_TIMEOUT and the
 * device stays usable.  scratch: >= 16 bytes of device memory.  Synchronises. */
int sg_selftest_barrier(int extra_blocks, long long spin_limit, void* scratch, void* stream);

/* ------------------------------------------------------------------------
 * Time-stepped Helmholtz sequence and its reverse-time adjoint (FP64).
 * Sequence (implicit time stepping, Sec. 5.2, with the Helmholtz systems of
 * Eq. VelocityEqn): A x_k = M (lam x_{k-1} + f_k), A = K + lam M (the
 * operator of sg_op_create with that lambda), M the GLL mass matrix of
 * Sec. 5.1.  Loss L = sum_k ||x_k - x*_k||^2.  Adjoint, backward in time:
 * A g_k = 2 (x_k - x*_k) + lam M g_{k+1}; dL/df_k = M g_k;
 * dL/dlam = sum_k g_k^T M (x_{k-1} - x_k).  All vectors: FP64 device, n
 * entries; Dirichlet entries of the outputs are 0.  The solves are
 * sg_pcg_solve calls; these entry points build right-hand sides and
 * accumulate (deterministically) into a device double *acc.
 * ------------------------------------------------------------------------ */

/* Workspace bytes for sg_adjoint_accum / sg_sqdiff_accum (zero it once before
 * first use; the kernels leave it ready for the next call). */
size_t sg_seq_workspace_bytes(sg_op_t op);
/* rhs = M (a x + f); x or f may be NULL (treated as 0), not both. */
int sg_mass_rhs(sg_op_t op, double a, const void* x, const void* f, void* rhs, void* stream);
/* rhs = c (x - xs) + a M gnext on interior nodes; gnext may be NULL. */
int sg_adjoint_rhs(sg_op_t op, double c, const void* x, const void* xs, double a, const void* gnext,
                   void* rhs, void* stream);
/* mg = M g (mg may be NULL); acc[0] += g^T M (xprev - x) (xprev NULL = 0). */
int sg_adjoint_accum(sg_op_t op, const void* g, const void* xprev, const void* x, void* mg, double* acc,
                     void* workspace, void* stream);
/* acc[0] += ||x - xs||^2 over interior nodes. */
int sg_sqdiff_accum(sg_op_t op, const void* x, const void* xs, double* acc, void* workspace, void* stream);

/* ------------------------------------------------------------------------
 * Allocation-free PCG.  The paper has no counterpart: this entry point is for
 * callers that cannot allocate device memory -- code whose device memory is
 * owned by a host framework that hands out no more, or a time-critical loop
 * that must not enter the driver's allocation path.  It runs the same solver
 * as sg_pcg_solve, but its scratch (the PCG vectors, reduction partials and
 * state) is a file-scope static __device__ array of SG_NOALLOC_SCRATCH_BYTES,
 * held by every GPU that loads the library until the process exits.  It calls
 * no cudaMalloc, cudaFree, cudaHostAlloc or other allocating routine; it polls
 * convergence through pageable host memory, and kernel timing is off for it.
 *  - Operators with more than SG_NOALLOC_MAX_NODES nodes are rejected with
 *    SG_ERR_INVALID (message via sg_last_error()).
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture on that device.
 *  - The operator must have been created on the device that is current at
 *    the call (the array used is the current device's); otherwise the call
 *    returns SG_ERR_INVALID.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; the call resets what must start at zero itself.  Calls whose
 *    work overlaps on the GPU (other streams, other host threads) race on the
 *    array: serialise them.
 * Arguments, outputs and return codes are those of sg_pcg_solve without the
 * workspace.  Synchronises with ``stream``.
 * ------------------------------------------------------------------------ */
#define SG_NOALLOC_MAX_NODES 131072
#define SG_NOALLOC_SCRATCH_BYTES (6815744) /* 6.5 MiB */
int sg_pcg_solve_noalloc(sg_op_t op, const void* b, void* x, double tol, int maxit, int criterion,
                         int* iters, double* relres, void* stream);

/* ------------------------------------------------------------------------
 * Initial guesses (Sec. 2-3).  A guess handle keeps the history spaces in
 * the caller's workspace: for EXTRAP/SPEXTRAP/LAST a ring of s solutions
 * (Sec. 3, Eq. ExtrapExpn); for PROJ_QR/PROJ_CLASSIC the right-hand-side
 * basis B~ and solutions X~ (A X~ = B~, B~ orthonormal) plus the triangular
 * factor R (Sec. 2, Algorithms 1-2).  All control state (d, R, ring head)
 * stays on the device, so form/update never synchronise.
 * ------------------------------------------------------------------------ */

/* Workspace bytes for a guess handle of this size/method/dtype. */
size_t sg_guess_workspace_bytes(int64_t n, int s, int method, int dtype);

/* Create a guess handle.  1 <= s <= SG_MAX_HISTORY (history size M);
 * degree_m: extrapolation degree (0 <= m <= s-1; -1 selects floor(sqrt(s)));
 * eps_rel: projection rejection threshold -- a new direction is kept only if
 * ||b~|| after CGS2 exceeds eps_rel * ||A x|| (Sec. 2, "small relative to
 * b"); op: required for PROJ_* (the update forms b~ = A x, Algorithm 2),
 * ignored otherwise; workspace: device, sg_guess_workspace_bytes bytes, zeroed
 * by this call (stream-ordered on the legacy default stream). */
int sg_guess_create(sg_guess_t* g, int64_t n, int s, int method, int degree_m, double eps_rel,
                    sg_op_t op, void* workspace, int dtype);
int sg_guess_destroy(sg_guess_t g);

/* Form the initial guess for right-hand side b (Algorithm 2 first line, or
 * Eq. ExtrapExpn).  With no history yet, x0 is left as passed in (the
 * caller's arbitrary x0, Sec. 2 notation); ZERO writes 0.  b, x0: device.
 * x0 may be the pointer returned by sg_guess_next_slot. */
int sg_guess_form(sg_guess_t g, const void* b, void* x0, void* stream);

/* EXTRAP/SPEXTRAP/LAST: device pointer of the ring slot the next solution
 * will occupy.  A solver that leaves x_k there makes the history update free
 * (App. A: "stores the solutions in place").  NULL for other methods. */
void* sg_guess_next_slot(sg_guess_t g);

/* Add solution x (of A x = b) to the history.  EXTRAP: copies x into the
 * next slot unless x already is that slot.  PROJ_QR: Algorithm 2 after the
 * solve -- b~ = A x, Givens downdate when d = M, CGS2, rejection test.
 * PROJ_CLASSIC: Algorithm 1 after the solve.  b is not read. */
int sg_guess_update(sg_guess_t g, const void* x, const void* b, void* stream);

/* Checkpoint of a guess handle (no counterpart in the paper; a time stepper
 * that restarts needs its history back).  sg_guess_image_bytes: size of the
 * HOST image (a header plus the handle's workspace contents: history columns,
 * projection state and R), 0 for a NULL handle.  sg_guess_export writes the
 * image to ``image`` (HOST, caller-owned, sg_guess_image_bytes(g) bytes).
 * sg_guess_import restores an image of image_bytes bytes into a handle
 * created with the same n, s, method, degree and dtype -- for projection
 * handles also the same eps_rel and an operator of the same mesh, degree,
 * lambda and dtype, under which the stored history is orthonormal -- after
 * which form/update continue exactly as they would have in the exported
 * handle.  The header is checked before anything is copied (size, kind,
 * ring position consistent with an update count); on SG_ERR_INVALID the
 * handle is unchanged.  Both synchronise with ``stream``. */
size_t sg_guess_image_bytes(sg_guess_t g);
int sg_guess_export(sg_guess_t g, void* image, void* stream);
int sg_guess_import(sg_guess_t g, const void* image, size_t image_bytes, void* stream);

/* Debug/inspection (synchronises ``stream``): current history dimension d
 * (PROJ) or stored-solution count (EXTRAP), and, if R is not NULL, the
 * s*s row-major FP64 factor R (PROJ) or the current s coefficients beta
 * (EXTRAP, oldest first, zero-padded). */
int sg_guess_info(sg_guess_t g, int* d, double* R, void* stream);

/* ------------------------------------------------------------------------
 * Kernel timing (library-side CUDA events around the launches of one kernel
 * class, recorded on the launching stream).  kernel ids: 0 sem_apply,
 * 1 pcg_apply (operator + fused p-update), 2 pcg_update, 3 extrap,
 * 4 proj_dots, 5 proj_lincomb, 6 proj_update (Givens + CGS2 sweeps).
 * ------------------------------------------------------------------------ */
int sg_profile_enable(int on);
/* Synchronises; total milliseconds and launch count since the last reset. */
int sg_profile_read(int kernel_id, double* total_ms, long long* launches);
int sg_profile_reset(void);
/* Number of kernels this library has launched in the process so far. */
long long sg_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
