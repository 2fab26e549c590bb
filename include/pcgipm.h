/*
 * pcgipm.h -- C ABI of the GB300 preconditioned inexact interior-point QP solver.
 *
 * Method: Karim & Solomonik, "Efficient Preconditioners for Interior Point
 * Methods via a new Schur Complement-Based Strategy".  The QP (Sec. 1,
 * eq. [qp]) is
 *
 *     minimise 1/2 x'Hx + c'x   subject to   A x = b,   C x >= d,
 *
 * H (n x n) symmetric positive definite, A (m1 x n) of full row rank, C (m2 x n).
 * The hot path is the preconditioned CG solve of the inequality-constraint
 * reduced system K_F dnu = r_nu (Sec. 4.1, eq. [ineq-const-reduced]) with
 *
 *     K_F = D + [C 0] K0^{-1} [C'; 0],   K0 = [H A'; A 0],   D = V^{-1} S,
 *
 * which is the paper's D - [C 0] F^{-1} [C'; 0] with F = [-H A'; A 0] = -J K0 J,
 * J = diag(-I_n, I_m1).  K0 is factored once per QP (the setup phase of Sec. 4.1)
 * and reused at every IPM iteration; K_F is never formed (Sec. 5.2: a product
 * with C', a solve with the K0 factor, a product with C).
 *
 * Conventions for every call below
 * --------------------------------
 * - Dense matrices are row-major FP64 with leading dimension equal to their
 *   column count; vectors are FP64.
 * - ptr_kind = QP_PTR_HOST: pointers are host memory (pageable or pinned);
 *   the call copies in/out and returns after the results are in place.
 *   ptr_kind = QP_PTR_DEVICE: pointers are device memory of the current CUDA
 *   device; the call is ordered on the solver's stream and returns after the
 *   results are written (it synchronises that stream).
 * - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *   Outputs are written into caller-owned buffers.
 * - All device work runs on opts.stream (a cudaStream_t cast to void*), or on
 *   a stream the library creates when it is NULL.
 * - Every call returns QP_OK (0) or a negative status from the enum below;
 *   qp_strerror gives its text.  A call that fails leaves the handle usable
 *   unless it returned QP_ECUDA (a CUDA runtime error; the handle should be
 *   destroyed).
 */
#ifndef PCGIPM_H
#define PCGIPM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum qp_status {
    QP_OK = 0,
    QP_EINVAL = -1,       /* bad dimension, NULL pointer, NaN/Inf input, asymmetric H */
    QP_ENOMEM = -2,       /* device allocation failed */
    QP_ESINGULAR = -3,    /* A H^{-1} A' has a non-positive pivot: A rank-deficient (Sec. 1 assumes full rank) */
    QP_ENOTCONVEX = -4,   /* H has a non-positive pivot: not positive definite (Sec. 1 assumption) */
    QP_EMAXIT = -5,       /* IPM iteration limit reached without meeting the tolerances */
    QP_ENUMERIC = -6,     /* NaN/Inf appeared during the iteration */
    QP_ETIMEOUT = -7,     /* a bounded device-side wait expired */
    QP_EAGAIN = -8,       /* result not ready yet */
    QP_ECUDA = -9,        /* CUDA runtime error */
    QP_ESTATE = -10       /* call out of order (e.g. solve before qp_factor_K0) */
};

enum qp_precision {
    QP_PREC_FP64 = 0,     /* factor, C copies and PCG all in FP64 */
    QP_PREC_FP32 = 1      /* mixed: C copies, K0 factor and PCG in FP32 until FP64 refinement
                             contracts by less than 4x per sweep, then in FP64 (a second, FP64
                             factor of K0); P_H in FP32 until its factorization needs a shift, then
                             in FP64; FP64 residuals, refinement, step logic.  With mixed_fallback,
                             a QP whose FP32 K0 factor meets a pivot below FP32 resolution is
                             factored and solved in FP64 from the start */
};

enum qp_precond {
    QP_PC_AUTO = 0,       /* P_L if m1 >= n/2 else P_H (Corollaries 1 and 2: n-m1+1 vs m1+1 iterations);
                             a QP started on P_L moves to QP_PC_PH_EXACT for its remaining IPM
                             iterations once a P_L solve ends without converging: the non-unit
                             eigenvalues of P_L^{-1} K_F are 1 + lambda(X), X >= 0 unbounded as
                             entries of D go to 0 (Sec. 4.3, Theorem 1), while those of
                             P_H^{-1} K_F are 1 - lambda(Y) in (0, 1] (Theorem 2) */
    QP_PC_PL = 1,         /* P_L = D, Sec. 4.2 eq. [preconditioner-1] */
    QP_PC_PH_EXACT = 2,   /* P_H = D + C H^{-1} C', Sec. 4.2 eq. [preconditioner-2] */
    QP_PC_PH_DIAG = 3,    /* P_H with diag(H)^{-1}, the variant of the experiments (Sec. 5.2, PH-KF) */
    QP_PC_NONE = 4        /* unpreconditioned CG on K_F (the U-KF variant of Sec. 6) */
};

enum qp_pcg_mode {
    QP_MODE_PARITY = 0,   /* each Newton direction refined against its FP64 residual */
    QP_MODE_PAPER = 1     /* one PCG solve per direction at the paper's eps = 1e-3, no refinement (Sec. 6) */
};

enum qp_ptr_kind { QP_PTR_HOST = 0, QP_PTR_DEVICE = 1 };

/* qp_opts.pcg_form: -1 lets qp_create choose (see qp_opts.pcg_form). */
enum qp_pcg_form { QP_FORM_AUTO = -1 };

typedef struct qp_s *qp_t;   /* opaque; owns every device buffer it allocates */

typedef struct {
    int precision;        /* enum qp_precision */
    int precond;          /* enum qp_precond */
    int pcg_mode;         /* enum qp_pcg_mode */
    int max_ipm;          /* IPM iteration limit (default 100) */
    int max_pcg;          /* PCG iteration limit per solve (default 4 * m2 + 50) */
    int refine_max;       /* refinement sweeps per Newton direction after the first solve (default 5) */
    double pcg_tol;       /* PCG relative residual tolerance; <= 0 selects the mode's default */
    double refine_tol;    /* stop refining when |rho|_2 <= refine_tol |rhs|_2 (default 1e-11) */
    double tol_feas;      /* scaled primal/dual infeasibility tolerance (default 1e-10) */
    double tol_mu;        /* stop when mu <= tol_mu (1 + |f|) (default 1e-11) */
    int pcg_check_every;  /* >= 0: PCG runs as one persistent kernel per solve (default 8, unused);
                             < 0: per-phase kernels in CUDA graphs of |value| iterations */
    int mixed_fallback;   /* QP_PREC_FP32 only: 1 (default) lets a QP move its operator and P_H to
                             FP64 when FP32 stops sufficing; 0 keeps FP32 (shifting P_H as needed) */
    int pcg_blocks;       /* blocks of the persistent PCG kernel: 0 (default) = about one per 512 KB
                             streamed per iteration (8 to 16 for a small QP, launched as one
                             thread-block cluster; up to one per SM); k > 0 = at most k (with 1 the
                             grid barriers become block barriers).  Results do not depend on it:
                             every reduction has a fixed order independent of the grid. */
    int blocking_wait;    /* 1: host waits on the solver's stream yield the CPU instead of spinning
                             (many QPs in flight on more host threads than cores); default 0 */
    int pcg_form;         /* how the persistent PCG kernel applies K_F (Sec. 5.2: a product with C',
                             a solve with the K0 factor, a product with C).  0 (default): the solve
                             as one product with M0 = [K0^{-1}]_11 = R^{-1} R^{-T} - Et' Et, the (1,1)
                             block of the inverse of the factorization, formed once per QP in FP64
                             (three matrix phases, 2 m2 n + n^2 elements per iteration).  2: the
                             forward and the back solve with the stored inverse factor as two
                             phases ([R^{-T}; Et] u, then [R^{-1} | Et'] [z1; -z2]; four matrix
                             phases, 2 m2 n + n^2 + 2 m1 n elements).  1: the same product through
                             B = L^{-1}[C'; 0] = [R^{-T} C'; Et C'], formed once per QP:
                             K_F p = D p + B1'(B1 p) - B2'(B2 p) (two matrix phases; 2 (n + m1) m2
                             elements).  3: the low-rank form (Sec. 4.3, Lemma 2: M0 has rank
                             r = n - m1): M0 = Z Z' by r steps of a pivoted Cholesky once per QP,
                             V = C Z, K_F p = D p + V (V' p) (two matrix phases, 2 m2 r elements;
                             QP_ESINGULAR if M0's numerical rank is below r; a handle that chose
                             it by QP_FORM_AUTO takes form 0 instead).  All four are the
                             same operator; the per-phase kernels (pcg_check_every < 0) always use
                             the two triangular solves.  QP_FORM_AUTO (default): 3 when C is dense,
                             1 <= r = n - m1 <= 1024 and 2 m2 r <= (2 m2 n + n^2) / 2 (few degrees
                             of freedom), else 0; the choice is reported in
                             qp_stats.pcg_form_used. */
    int factor_tc;        /* QP_PREC_FP32 with pcg_form 0 or 2: 1 forms the FP32 operator's K0 factor
                             (and M0) in FP32 storage with FP64 diagonal-block pivots and the dense
                             contractions -- the blocked Cholesky's trailing and inverse updates,
                             G = A R^{-1}, A H^{-1} A', L_S^{-1} G, Et, M0 -- on the tcgen05 tensor
                             cores (FP32-accurate 3xTF32 splits); a pivot below 1e-6 of its diagonal
                             entry falls back to the default.  0 (default): the factor is formed in
                             FP64 on the CUDA cores and rounded once (an FP32-accurate factor carries
                             about cond(H) u32 of relative error into H^{-1}; GB300 has no FP64
                             tensor path at useful rates). */
    int autotune;         /* 1 (default): a QP whose persistent PCG kernel spans more than one
                             thread-block cluster times a dozen iterations on a few grid sizes
                             (the rule's, 3/4 and 1/2 of it, one block per SM) before its first
                             solve in each precision and preconditioner, and keeps the fastest;
                             results do not depend on the grid (fixed-order reductions), only
                             the time does.  0: the rule of pcg_blocks alone. */
    int factor_bk;        /* 1: also factor K0 = [H A'; A 0] as P K0 P' = L D L' with Bunch-Kaufman
                             partial pivoting (the paper's setup factorization, Sec. 6: SYTRF) on the
                             GPU, check its inertia against (n, m1) (Sec. 4.1; QP_ENOTCONVEX
                             otherwise, QP_ESINGULAR for a zero column) and form M0 = [K0^{-1}]_11
                             = Z' D^{-1} Z, Z = L^{-1} P [I_n; 0], from it (pcg_form 0 and 3); the
                             other K0 solves keep the structured factor.  0 (default): M0 from the
                             structured factor R^{-1} R^{-T} - Et' Et. */
    void *stream;         /* cudaStream_t, or NULL for a library-created stream */
} qp_opts;

typedef struct {
    int status;           /* last status of qp_ipm_solve */
    int precond_used;     /* resolved enum qp_precond at the end of the last solve */
    int ipm_iters;
    long long pcg_iters_total;
    int newton_solves;    /* reduced solves (predictor + corrector + refinement corrections) */
    int refine_sweeps;    /* total refinement corrections */
    double res_p, res_d, mu, obj;   /* final scaled residuals, mu, objective */
    double t_factor_ms;   /* device time of qp_factor_K0 */
    double t_solve_ms;    /* wall time of the last qp_ipm_solve */
    double t_pcg_ms;      /* device time spent in PCG iterations during the last solve */
    double t_precond_ms;  /* device time of the per-iteration P_H factorizations */
    int op64_solves;      /* QP_PREC_FP32: reduced solves run with the FP64 operator after a switch */
    int op64_switch_iter; /* QP_PREC_FP32: IPM iteration of the switch to the FP64 operator, or -1 */
    int pc64_switch_iter; /* QP_PREC_FP32: IPM iteration of the switch to an FP64 P_H factor, or -1 */
    int pc_switch_iter;   /* QP_PC_AUTO: IPM iteration of the switch from P_L to P_H, or -1 */
    int factor_tc;        /* 1 if the FP32 K0 factor was formed on the tensor cores (qp_opts.factor_tc) */
    int pcg_form_used;    /* the handle's pcg_form (QP_FORM_AUTO resolved at qp_create) */
    int pcg_grid;         /* blocks of the last persistent PCG launch (after autotuning) */
    int k0_inertia_pos;   /* qp_opts.factor_bk: positive, negative eigenvalues of D (K0's inertia), */
    int k0_inertia_neg;   /*   and the number of 2x2 pivots; -1 without factor_bk */
    int k0_pivots_2x2;
} qp_stats;

/* Fill *opts with the defaults listed in the struct comments. */
void qp_opts_default(qp_opts *opts);

/*
 * Create a QP handle from the problem data of Sec. 1, eq. [qp]:
 * H (n x n, symmetric), c (n), A (m1 x n, m1 may be 0 with A = b = NULL),
 * b (m1), C (m2 x n, dense), d (m2).  Requires 1 <= n, 0 <= m1 <= n, 1 <= m2.
 * Copies everything to the device; validates symmetry of H (relative 1e-12)
 * and finiteness (QP_EINVAL).  opts may be NULL (defaults).
 */
int qp_create(qp_t *out, int n, int m1, int m2,
              const double *H, const double *c, const double *A, const double *b,
              const double *C, const double *d, const qp_opts *opts, int ptr_kind);

/*
 * qp_create with C given in compressed sparse row form: C_rowptr (m2 + 1 ints,
 * C_rowptr[0] = 0, non-decreasing), C_colidx (C_rowptr[m2] ints in [0, n)),
 * C_val (C_rowptr[m2] doubles); entries repeated within a row are summed.  The
 * pattern is checked on the device (QP_EINVAL for a bad pointer array or column
 * index).  The sparse pattern is the one the serving workload draws (8 entries
 * per row; the paper assumes sparse data, Sec. 5); C is expanded into the same
 * dense device layout as qp_create's, so every later call behaves identically.
 */
int qp_create_csr(qp_t *out, int n, int m1, int m2,
                  const double *H, const double *c, const double *A, const double *b,
                  const int *C_rowptr, const int *C_colidx, const double *C_val,
                  const double *d, const qp_opts *opts, int ptr_kind);

/*
 * Setup phase (Sec. 4.1: F is factored once per QP, before the IPM iterations).
 * Factors K0 = [H A'; A 0] = L diag(I_n, -I_m1) L' with L = [R' 0; G L_S],
 * H = R'R, G = A R^{-1}, A H^{-1} A' = L_S L_S' (the inertia of Sec. 4.1:
 * n pivots of H and m1 of F_H, all checked positive in FP64).  The triangular
 * factors are stored inverted (R^{-T}, L_S^{-1} G, L_S^{-1}) in the working
 * precision so that each triangular solve is a parallel triangular
 * matrix-vector product.  For P_H it also forms T = C H^{-1} C' (or
 * C diag(H)^{-1} C').  Idempotent.  Returns QP_ENOTCONVEX / QP_ESINGULAR on a
 * non-positive pivot.
 */
int qp_factor_K0(qp_t qp);

/*
 * One product q = K_F p with the implicit K_F (Sec. 5.2, three steps) for a
 * caller-given positive diagonal D (m2).  D, p, q: m2 vectors.  Runs in the
 * handle's working precision.  Needs qp_factor_K0.
 */
int qp_kf_apply(qp_t qp, const double *D, const double *p, double *q, int ptr_kind);

/*
 * Solve K0 [a; b] = [u; w] with the stored factor (forward solve, D^{-1},
 * back solve of the LDL' factor; Sec. 4.1 setup/solve split).  u, a: n;
 * w, b: m1 (w may be NULL for zero; b may be NULL if not wanted).
 */
int qp_k0_solve(qp_t qp, const double *u, const double *w, double *a, double *b, int ptr_kind);

/*
 * The hot path by itself: preconditioned CG on K_F dnu = rhs (Sec. 4.1,
 * eq. [ineq-const-reduced]) from a zero start, stopping when
 * |r|_2 <= tol |rhs|_2 or after maxit iterations (Sec. 6 settings).
 * D (m2, positive) parameterises K_F and P_L / P_H as in Theorems 1 and 2.
 * precond: enum qp_precond (AUTO resolves as in qp_opts).  iters / relres may
 * be NULL.  Returns QP_EMAXIT if maxit was reached before tol (dnu still holds
 * the last iterate).
 */
int qp_pcg_reduced_solve(qp_t qp, const double *D, const double *rhs, double *dnu,
                         int precond, double tol, int maxit, int *iters, double *relres,
                         int ptr_kind);

/*
 * Full primal-dual IPM (Sec. 2) whose Newton directions come from the reduced
 * system: per iteration FP64 residuals (eq. [rhs-KKT4]), D = V^{-1} S,
 * [P_H: refactor D + T], Mehrotra predictor and corrector each solved by
 * r_nu -> PCG -> recovery (eq. [schur-delta-x]) -> ds (eq. [delz]) and, in
 * PARITY mode, refined against the FP64 residual of the 3x3 system
 * (eq. [augmented]); one step length with fraction-to-boundary 0.995.
 * Outputs x (n), lam (m1), nu (m2), s (m2) may be NULL individually; obj,
 * ipm_iters, pcg_iters_total may be NULL.  Runs qp_factor_K0 first if needed.
 */
int qp_ipm_solve(qp_t qp, double *x, double *lam, double *nu, double *s,
                 double *obj, int *ipm_iters, long long *pcg_iters_total, int ptr_kind);

/* Per-QP outcome of qp_batch_solve. */
typedef struct {
    int status;             /* qp_ipm_solve status of this QP */
    int ipm_iters;
    long long pcg_iters;
    double obj, res_p, res_d, mu;
    double solve_ms;        /* wall time of this QP's factor + solve */
    double wait_ms;         /* server: submission to admission (0 in qp_batch_solve) */
    double latency_ms;      /* server: submission to result ready (solve_ms in qp_batch_solve) */
} qp_result;

/*
 * Solve `count` independent QPs (handles from qp_create, possibly of different
 * sizes) concurrently on the current GPU: up to `max_concurrent` host workers
 * (0 = 16) each take the next unsolved handle and run qp_factor_K0 and
 * qp_ipm_solve on that handle's own stream; the persistent PCG kernel of a small
 * QP uses a grid sized to its per-iteration bytes, so several QPs' kernels share
 * the GPU.  results[i] receives QP i's outcome; solutions stay in the handles
 * (qp_get_solution).  Each handle must have been created with opts.stream NULL
 * (its own stream).  Returns QP_OK when every QP converged, else the first
 * non-OK status (every QP is attempted).  Batched workloads: the 512 dense QPs of
 * uneven size (n in [64, 512]) the method is measured on.
 */
int qp_batch_solve(qp_t *qps, int count, int max_concurrent, qp_result *results);

/* Copy the last qp_ipm_solve iterate of `qp` (x: n, lam: m1, nu: m2, s: m2; any may be NULL). */
int qp_get_solution(qp_t qp, double *x, double *lam, double *nu, double *s, int ptr_kind);

/* Copy the handle's counters and timings into *st. */
int qp_get_stats(qp_t qp, qp_stats *st);

/* Bytes of device memory the handle holds (after qp_factor_K0: its peak). */
size_t qp_device_bytes(qp_t qp);

/*
 * Upper bound on the device memory a handle of these sizes and options can hold
 * at any time from qp_create to qp_destroy, setup scratch included: the FP64
 * problem copies, the operator factor (both precisions when QP_PREC_FP32 may
 * move to FP64), and the P_H matrices when the preconditioner is or may become
 * P_H (QP_PC_AUTO).  Used for admission by the server below.  opts may be NULL.
 */
size_t qp_device_bytes_bound(int n, int m1, int m2, const qp_opts *opts);

/*
 * Per-PCG-iteration algorithmic traffic of the handle's hot path in bytes,
 * for a given preconditioner: 2 m2 n (C' and C) + the triangles of the
 * stored K0 factor + [P_H] m2^2 + the vector traffic, times the element size.
 */
double qp_pcg_bytes_per_iter(qp_t qp, int precond);

/*
 * Time the hot path: run `iters` PCG iterations (no early stop) on K_F with
 * diagonal D (device or host per ptr_kind) after `warmup` untimed ones and
 * return the mean device time of one iteration in *ms_per_iter (CUDA events
 * on the solver stream).  Needs qp_factor_K0.
 */
int qp_time_pcg_iteration(qp_t qp, const double *D, int precond, int warmup, int iters,
                          double *ms_per_iter, int ptr_kind);

/*
 * Largest n accepted by qp_kf_apply_static (its intermediate vectors live in a
 * fixed device array of 4 * QP_STATIC_MAX_N + QP_STATIC_MAX_N doubles, 320 KiB).
 */
#define QP_STATIC_MAX_N 8192

/*
 * q = K_F p without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory themselves
 * -- code that runs under a memory allocator it does not own (a framework's
 * caching allocator, a host application that hands over fixed buffers), inside a
 * region where cudaMalloc would synchronise the device or is not allowed, or on
 * a device-memory budget fixed in advance -- and so cannot create a qp_t handle.
 *
 * It computes the same product as qp_kf_apply in FP64 from a factored K0 the
 * caller supplies, all as row-major device arrays with leading dimension equal
 * to their column count:
 *   C  (m2 x n)  the inequality matrix,
 *   WH (n x n)   R^{-T}, the inverse of the lower Cholesky factor of H
 *                (H = R'R; lower triangle, zeros above it),
 *   Gt (m1 x n)  L_S^{-1} A R^{-1} with L_S L_S' = A H^{-1} A' (NULL if m1 = 0),
 *   D, p (m2) inputs, q (m2) output.
 * Chain: u = C'p, z1 = WH u, z2 = -Gt z1, t = z1 + Gt' z2, y = WH' t,
 * q = D o p + C y.  Requires 1 <= n <= QP_STATIC_MAX_N, 0 <= m1 <= n, m2 >= 1
 * (QP_EINVAL otherwise).  It calls no cudaMalloc/cudaFree and no allocating
 * library routine: the intermediate vectors live in one file-scope device array
 * that every device which uses the library's module holds until the process
 * exits (under lazy module loading, the default since CUDA 12.2, the array is
 * reserved when the module is first used on a device, not when the library is
 * loaded).  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current), which may load the module;
 * make that first call before any stream capture.  The work is enqueued on
 * `stream` (a cudaStream_t cast to void*, NULL = the default stream) and the
 * call returns without waiting.  QP_ECUDA: an error was already pending when
 * the call began (it is left in place), or a launch failed; an error during
 * execution shows at the caller's next synchronisation with the stream.  All
 * calls on a device share the array: calls that overlap on the GPU (different
 * streams, or different host threads) race on it and must be serialised by the
 * caller.  Every intermediate is written before it is read, so nothing left by
 * an earlier call affects a later one.
 */
int qp_kf_apply_static(int n, int m1, int m2, const double *C, const double *WH, const double *Gt,
                       const double *D, const double *p, double *q, void *stream);

/*
 * Serving (continuous batching).  A server owns a device-memory budget and up
 * to max_slots QPs in flight on the current GPU.  qp_server_submit copies a
 * QP's host data into the server and returns at once with a ticket; requests
 * are admitted in submission order as soon as a slot is free and the request's
 * qp_device_bytes_bound fits in what the budget has left (a request that does
 * not fit waits, and those behind it wait too, so a large QP is never starved).
 * An admitted QP is created, factored and solved on its own stream while others
 * run, its K0 factor and IPM state resident on the device for the whole solve;
 * the persistent PCG kernels of QPs in flight share the GPU (each grid sized by
 * its QP's per-iteration bytes).  When a QP finishes, its device memory is
 * released and the next requests are admitted.  The paper has no serving layer;
 * each QP is solved exactly as qp_ipm_solve solves it alone, so results do not
 * depend on what else is in flight.
 */
typedef struct qp_server_s *qp_server_t;

/* One QP of a submission: host pointers, layouts as in qp_create / qp_create_csr
 * (exactly one of C and C_rowptr non-NULL). */
typedef struct {
    int n, m1, m2;
    const double *H, *c, *A, *b;
    const double *C;
    const int *C_rowptr, *C_colidx;
    const double *C_val;
    const double *d;
} qp_problem;

/* Aggregate counters of a server. */
typedef struct {
    long long submitted, completed, failed;
    int queued, active;
    size_t reserved_bytes;       /* sum of the bounds of the QPs in flight */
    size_t peak_reserved_bytes;
    size_t peak_device_bytes;    /* largest qp_device_bytes seen for one QP */
} qp_server_stats;

/*
 * Start a server: hbm_budget_bytes of device memory for QPs in flight (0 = 90%
 * of the device's free memory), max_slots QPs in flight (0 = 16); every QP is
 * solved with *opts (NULL = defaults; opts->stream must be NULL).
 */
int qp_server_create(qp_server_t *out, size_t hbm_budget_bytes, int max_slots, const qp_opts *opts);

/*
 * Queue one QP (its data is copied before the call returns) and return its
 * ticket.  QP_EINVAL for bad sizes or pointers; QP_ENOMEM when the QP's bound
 * exceeds the whole budget (it could never be admitted); QP_ESTATE after
 * qp_server_destroy began.
 */
int qp_server_submit(qp_server_t srv, const qp_problem *qp, unsigned long long *ticket);

/*
 * Non-blocking: QP_EAGAIN while the ticket's QP is queued or running.  Once it
 * is done, fills *r (r->status is the solve's status) and copies the solution
 * into any non-NULL host buffer (x: n, lam: m1, nu: m2, s: m2), releases the
 * ticket and returns QP_OK.  QP_EINVAL for an unknown or released ticket.
 */
int qp_server_poll(qp_server_t srv, unsigned long long ticket, qp_result *r,
                   double *x, double *lam, double *nu, double *s);

/* Block until every submitted QP is done or timeout_ms passes (< 0: no limit);
 * QP_ETIMEOUT in the second case. */
int qp_server_drain(qp_server_t srv, double timeout_ms);

int qp_server_get_stats(qp_server_t srv, qp_server_stats *st);

/* Finish the QPs in flight and the queued ones, stop the workers, free the server. */
void qp_server_destroy(qp_server_t srv);

/*
 * Number of this library's kernel launches that have reached the current
 * device since it was loaded (each kernel counts itself once; graph-launched
 * kernels included).  Synchronises the device.  Returns 0 on a CUDA error.
 */
unsigned long long qp_kernel_launches(void);

void qp_destroy(qp_t qp);
const char *qp_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* PCGIPM_H */
