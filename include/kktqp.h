/*
 * kktqp.h - C ABI of the GB300 Krylov interior point library.
 *
 * Solves convex quadratic programs
 *
 *     min 1/2 x'Hx + p'x   s.t.  lA <= A x <= uA,  C x = b,  lx <= x <= ux     (Eq. (1))
 *
 * with the primal-dual interior point method of Liu, Fredriksson & Markidis
 * (arXiv 2308.00637): each Newton step solves the doubly augmented KKT system
 * (Eq. (9)) with Jacobi-preconditioned conjugate gradients, applied matrix-free
 * from H, A, A' and the diagonal D built from slacks and multipliers (section
 * 3.2); step lengths by the ratio test (Eq. (10)); mu divided by 10 whenever
 * the residual norm drops below mu (Algorithm 1).
 *
 * Conventions shared by every entry point
 *  - Pointers may be host or device memory (CUDA unified addressing decides);
 *    the library copies inputs at qp_create and the caller keeps ownership of
 *    every buffer it passes.  All device memory is owned by the handle and is
 *    released by qp_destroy.
 *  - Absent bounds are +-INFINITY.
 *  - All work is ordered on the stream given at qp_create (NULL = legacy
 *    default stream).  A handle is used by one host thread at a time.
 *  - Every call returns a kq_status; none throws across the ABI.  After a
 *    non-OK status qp_last_error(h) returns a message.
 *  - Multiplier layout ("padded"): the KKT unknown of Eq. (9) is stored as
 *        [ x (n) | lam_e (me) | lam_lA (m) | lam_uA (m) ]      NKP = n + me + 2m
 *    where entries of lam_lA / lam_uA for rows whose bound is infinite are
 *    identically zero (those rows are decoupled identity rows in K).
 *  - Units: solutions (x, multipliers, slacks) returned by ipm_solve are in
 *    the caller's original units.  kkt_apply / kkt_pcg_solve work on the
 *    internally scaled system (objective scaled by sigma = 1/max(1, max H_ii,
 *    |p|_inf), each A/C row and its bounds by 1/||row||_2).
 */
#ifndef KKTQP_H
#define KKTQP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kq_problem *kq_handle;
typedef int kq_status;

enum {
  KQ_OK = 0,
  KQ_ERR_ARG = 1,          /* invalid argument / unsupported combination      */
  KQ_ERR_CUDA = 2,         /* a CUDA runtime call failed                       */
  KQ_ERR_OOM = 3,          /* device allocation failed                         */
  KQ_ERR_NOT_CONVEX = 4,   /* PCG met p'Kp <= 0: K not SPD (H not convex)      */
  KQ_WARN_PCG_MAXIT = 5,   /* PCG stopped at its iteration cap; step was taken */
  KQ_ERR_IPM_MAXIT = 6,    /* IPM iteration cap reached; best iterate returned */
  KQ_ERR_TIMEOUT = 7,      /* a device-side grid barrier exceeded its budget   */
  KQ_ERR_NUMERIC = 8,      /* NaN/Inf met in data or iterates                  */
  KQ_ERR_STATE = 9         /* call order violated (e.g. backward before solve) */
};

/* H operator kinds (section 2.2 / section 3.2: H used only through products) */
enum { KQ_H_DENSE = 0,     /* explicit symmetric n x n, row-major              */
       KQ_H_CSR_LSQ = 1,   /* H = 2 P' diag(w) P, P CSR (rows x n)             */
       KQ_H_LOWRANK = 2,   /* H = Z diag(w) Z' + diag(d0), Z dense n x k       */
                           /* row-major (w, d0 optional: Z Z' by default); the */
                           /* quasi-Newton form H0 + U W U' of section 2.1     */
       KQ_H_RBF = 3 };     /* Gaussian-kernel SVM dual (Eq. (6)): H_ij =       */
                           /* y_i y_j exp(-gamma |x_i - x_j|^2), formed once at */
                           /* create on the device from the samples X (n x d,  */
                           /* F64 row-major) and stored as a dense H           */
/* constraint-matrix kinds (the general rows l <= A x <= u of Eq. (1)) */
enum { KQ_A_NONE = 0,      /* no general rows                                   */
       KQ_A_DENSE = 1,     /* m x n row-major                                   */
       KQ_A_CSR = 2,       /* m x n CSR (val, col, rowptr), any H kind          */
       KQ_A_ROWS_OF_P = 3 };/* rows of the CSR_LSQ operator's P (dose limits)  */
/* storage types */
enum { KQ_F64 = 0, KQ_F32 = 1, KQ_BF16 = 2 };
/* arithmetic of the K products inside PCG */
enum { KQ_PREC_F64 = 0,    /* FP64 vectors, dots, diagonal and step; FP64-class */
                           /* products: double-float on the FP32 pipe where the */
                           /* matrix data is exact in FP32 (~2^-48 per term),   */
                           /* native FP64 otherwise                             */
       KQ_PREC_MIXED = 1 };/* FP32 matvec + FP32 accumulation; FP64 dots,
                              diagonal, step and FP64 residual refinement       */

typedef struct {
  int kind;                /* KQ_H_*                                            */
  int dtype;               /* storage of val/Z/H: KQ_F64, KQ_F32 or KQ_BF16     */
                           /* (RBF: of the formed H; X is always F64)          */
  int64_t rows;            /* CSR_LSQ: rows of P;  LOWRANK, DENSE, RBF: n      */
  int64_t cols;            /* CSR_LSQ: n; LOWRANK: k; DENSE: n; RBF: d features*/
  int64_t nnz;             /* CSR_LSQ: nonzeros of P                            */
  const void *val;         /* DENSE: H; LOWRANK: Z; CSR_LSQ: P values; RBF: X   */
  const int32_t *col;      /* CSR_LSQ column indices (sorted not required)     */
  const int64_t *rowptr;   /* CSR_LSQ row pointers (rows+1)                    */
  const double *w;         /* CSR_LSQ row weights (rows), H = 2 P'diag(w)P;    */
                           /* LOWRANK column weights (k, NULL = all 1);        */
                           /* RBF labels y (n, NULL = all 1)                   */
  const double *d0;        /* LOWRANK diagonal H0 (n, NULL = 0)                 */
  double gamma;            /* RBF kernel width (> 0, finite)                    */
} kq_hop;

typedef struct {
  int kind;                /* KQ_A_*                                            */
  int dtype;               /* DENSE, CSR: KQ_F64 or KQ_F32                      */
  int64_t m;               /* number of rows                                    */
  const void *val;         /* DENSE: m x n row-major; CSR: nnz values           */
  const int32_t *rows;     /* ROWS_OF_P: row ids into P (m), strictly increasing*/
  int64_t nnz;             /* CSR: nonzeros                                     */
  const int32_t *col;      /* CSR: column of each nonzero (0 <= col < n)        */
  const int64_t *rowptr;   /* CSR: row pointers (m + 1, rowptr[0] = 0,          */
                           /*      rowptr[m] = nnz, non-decreasing)             */
} kq_amat;

typedef struct {
  double gamma;            /* ratio-test factor, Eq. (10); paper: 0.99          */
  double mu0;              /* initial mu (1.0)                                  */
  double mu_tol;           /* return when ||r|| < mu and mu < mu_tol (1e-6)     */
  int ipm_maxit;           /* Algorithm 1's N (200)                             */
  double pcg_tol;          /* relative unpreconditioned residual (1e-7)         */
  int pcg_maxit;           /* PCG iterations per Newton solve (5000)            */
  int precision;           /* KQ_PREC_*.  MIXED: once a Newton solve has timed  */
                           /* an FP64 product (its residual check) at under     */
                           /* twice an FP32 iteration (latency-bound problems), */
                           /* the rest of the solve runs in FP64                */
  int refine_steps;        /* MIXED: FP32 correction solves before FP64 (6); the */
                           /* batched solver hands a QP to FP64 earlier once one*/
                           /* of its FP32 solves fails to halve its residual    */
  double inner_tol;        /* MIXED: relative tolerance of each FP32 solve      */
  double timeout_s;        /* device barrier budget per wait (seconds)         */
  int grid_ctas;           /* 0 = auto; else persistent-kernel grid size        */
  int verbose;             /* 1 = one line per IPM iteration on stderr          */
  int record;              /* 1 = keep one kq_ipm_iter per IPM iteration        */
                           /*     (qp_iteration_log); default 0                 */
  int graph;               /* ipm_solve_batch: 1 = capture the lock-step IPM    */
                           /*     iteration once in a CUDA graph and replay it, */
                           /*     every decision taken on the device; 0 = host- */
                           /*     driven launches (default 1)                   */
  int warm_start;          /* ipm_solve: 1 = each Newton solve after the first  */
                           /*     starts from the previous Newton direction     */
                           /*     when that at least halves the FP64 residual,  */
                           /*     else from zero (section 6 lists warm starts   */
                           /*     as future work); default 0 (paper: from zero) */
} kq_ipm_opts;

/* One IPM iteration's record (opts.record = 1): the quantities the paper
 * follows per iteration -- CG iterations per Newton solve (section 5.1), the
 * primal, dual and complementarity infeasibilities (section 5.2) and the
 * conditioning of the Jacobi-preconditioned doubly augmented system (section
 * 5.3).  lanczos_min / lanczos_max are the extreme eigenvalues of the
 * Lanczos tridiagonal matrix built from the first PCG pass's alpha and beta
 * coefficients: Ritz values, so they lie inside the spectrum of
 * diag(K)^-1/2 K diag(K)^-1/2 and kappa_jacobi = max/min is a lower bound of
 * its condition number that tightens as the pass runs longer.  diag_ratio =
 * max diag(K) / min diag(K) is a lower bound of the condition number of the
 * unpreconditioned K.  Infeasibilities in scaled units, after the step. */
typedef struct {
  int it;
  int pcg_iters;           /* all passes of the Newton solve                    */
  int pcg_iters_f64;
  int lanczos_steps;       /* coefficients used (first pass, at most 5000)      */
  double mu;               /* barrier parameter of the Newton solve             */
  double res_norm;         /* ||r||_2 after the step (before any mu update)     */
  double primal_inf, dual_inf, compl_inf;
  double alpha_x, alpha_lam;
  double pcg_rel_res;      /* true relative residual of the Newton solve        */
  double pcg_ms;           /* device time of its persistent launches            */
  double lanczos_min, lanczos_max, kappa_jacobi, diag_ratio;
} kq_ipm_iter;

typedef struct {
  int status;              /* final kq_status                                   */
  int ipm_iters;
  double mu_final;
  double res_norm;         /* ||r||_2 of Eq. (7)'s right-hand side, scaled units*/
  double primal_inf, dual_inf, compl_inf;   /* section 5.2 norms, scaled units  */
  long long pcg_iters;     /* total PCG iterations over the solve               */
  int pcg_maxit_hits;      /* Newton solves that stopped at pcg_maxit           */
  double time_s;           /* wall time of ipm_solve                            */
  double pcg_time_s;       /* device time inside PCG solves (CUDA events)       */
  double pcg_kernel_ms;    /* device time of the persistent PCG kernels only    */
  long long pcg_launches;  /* persistent PCG kernel launches                    */
  long long pcg_products;  /* K*v products inside PCG kernels (iterations+applies)*/
  long long kernel_launches; /* all kernels this call launched                   */
  long long pcg_iters_f64; /* MIXED: PCG iterations run in FP64 (rescue passes) */
  long long pcg_products_f64;  /* products inside FP64 launches (passes + residuals) */
  double pcg_kernel_ms_f64;    /* device time of the FP64 persistent launches       */
  long long pcg_launches_f64;  /* FP64 persistent launches (passes + residuals)     */
  int switched_to_f64;     /* MIXED: IPM iteration after which the solve ran in   */
                           /* FP64 (0 = never; see kq_ipm_opts.precision)         */
} kq_ipm_stats;

typedef struct {
  double tol;              /* relative unpreconditioned residual                */
  int maxit;
  int precision;           /* KQ_PREC_*                                         */
  int refine_steps;
  double inner_tol;
} kq_pcg_opts;

typedef struct {
  int status;
  int iters;               /* PCG iterations over all passes                    */
  int passes;              /* correction solves (1 unless refinement ran)       */
  double rel_res;          /* true ||rhs - K z|| / ||rhs|| in FP64              */
  double kernel_ms;        /* device time of the persistent kernels             */
  int iters_f64;           /* iterations of FP64 passes (all of them in F64)    */
  int products_f64;        /* products inside FP64 launches (passes + residuals)*/
  double kernel_ms_f64;    /* device time of the FP64 persistent launches       */
  int launches_f64;        /* FP64 persistent launches (passes + residuals)     */
  int products;            /* K*v products inside the persistent kernels        */
} kq_pcg_stats;

/* Fill *o with the paper's settings (gamma 0.99, mu/10, mu_tol 1e-6, PCG tol
 * 1e-7, 5000 PCG iterations; section 3.2 and section 5.1) and FP64. */
void kq_default_ipm_opts(kq_ipm_opts *o);
void kq_default_pcg_opts(kq_pcg_opts *o);

/* qp_create: problem statement of Eq. (1) with bounds separated (section 3.1).
 *  n      variables;  H  operator (required);  p  linear term (n)
 *  A      general rows (may be NULL = none) with lA, uA (m each, +-inf = absent)
 *  me     equality rows; C dense me x n row-major FP64 and b (me); NULL if me=0
 *  lx,ux  variable bounds (n each, may be NULL = free)
 *  stream cudaStream_t (as void*), NULL for the default stream
 * Supported: every H kind (DENSE F64/F32/BF16, CSR_LSQ with F32 values,
 * LOWRANK F32/F64) with A NONE or CSR (F64/F32 values) and any number of
 * equality rows; DENSE A (F64/F32) with DENSE H; ROWS_OF_P with CSR_LSQ H.
 * CSR structures (P and A) are checked on the device: a row pointer out of
 * order or a column outside [0, n) gives KQ_ERR_ARG.  A NaN or infinity in p
 * or on the diagonal of H gives KQ_ERR_NUMERIC.  Other errors: KQ_ERR_ARG for
 * bad sizes or an unsupported combination, KQ_ERR_OOM, KQ_ERR_CUDA.  *out is
 * NULL on error. */
kq_status qp_create(kq_handle *out, int64_t n, const kq_hop *H, const double *p,
                    const kq_amat *A, const double *lA, const double *uA,
                    int64_t me, const double *C, const double *b,
                    const double *lx, const double *ux, void *stream);

/* qp_update: replace the data that a differentiable QP layer varies -- the
 * linear term p (n), the row bounds lA, uA (m) and the equality right-hand
 * side b (me) -- keeping H, A, C, the variable bounds and every device
 * structure built at qp_create.  Any pointer may be NULL (kept); host or
 * device memory; unscaled values.  The scaling rule of qp_create is applied
 * again (sigma from the new |p|_inf).  The next ipm_solve starts from the
 * initial point.  Synchronises the handle's stream.  KQ_ERR_NUMERIC for NaN or
 * Inf in p. */
kq_status qp_update(kq_handle h, const double *p, const double *lA, const double *uA,
                    const double *b);

/* ipm_solve: Algorithm 1 from the initial point (or from the state set by
 * qp_set_state).  Outputs (any may be NULL), original units:
 *  x (n); lam_lA, lam_uA (m, zero where the bound is absent); lam_lx, lam_ux
 *  (n); lam_e (me).  Returns KQ_OK on convergence, KQ_ERR_IPM_MAXIT (outputs
 *  hold the last iterate), or an error. */
kq_status ipm_solve(kq_handle h, const kq_ipm_opts *opts, double *x,
                    double *lam_lA, double *lam_uA, double *lam_lx,
                    double *lam_ux, double *lam_e, kq_ipm_stats *stats);

/* qp_iteration_log: the records of the last ipm_solve run with
 * opts.record = 1 (see kq_ipm_iter).  Copies min(cap, count) records to out
 * (host memory); *count = records available.  KQ_ERR_STATE if no recorded
 * solve ran. */
kq_status qp_iteration_log(kq_handle h, kq_ipm_iter *out, int cap, int *count);

/* kkt_pcg_solve: Jacobi-PCG on the K of Eq. (9) at the current iterate and
 * barrier parameter, scaled units, padded layout (NKP = n + me + 2m).
 * rhs, sol: NKP doubles.  z0 = 0. */
kq_status kkt_pcg_solve(kq_handle h, const double *rhs, double *sol,
                        const kq_pcg_opts *opts, kq_pcg_stats *stats);

/* kkt_apply: out = K v (Eq. (9)) at the current iterate, FP64 or MIXED
 * arithmetic, scaled units, padded layout. */
kq_status kkt_apply(kq_handle h, const double *v, double *out, int precision);

/* kkt_diag: Jacobi diagonal diag(K) at the current iterate (NKP). */
kq_status kkt_diag(kq_handle h, double *diag);

/* qp_backward: after a converged ipm_solve, gradients of L = gbar'x* with
 * respect to p, lA, uA and b by one extra PCG solve with the converged K
 * (K [v; w] = [gbar; 0]).  Original units; outputs may be NULL.  Rows or
 * entries whose bound is infinite get 0.  KQ_ERR_STATE if no solve ran. */
kq_status qp_backward(kq_handle h, const double *gbar, double *grad_p,
                      double *grad_lA, double *grad_uA, double *grad_b,
                      const kq_pcg_opts *opts, kq_pcg_stats *stats);

/* Iterate access (checkpoint / warm start / testing), scaled units.
 * x (n); s_lA, s_uA, lam_lA, lam_uA (m); s_lx, s_ux, lam_lx, lam_ux (n);
 * lam_e (me); *mu.  Entries for absent bounds are ignored on set and returned
 * as s = 1, lam = 0 on get. */
kq_status qp_get_state(kq_handle h, double *x, double *s_lA, double *s_uA,
                       double *s_lx, double *s_ux, double *lam_lA,
                       double *lam_uA, double *lam_lx, double *lam_ux,
                       double *lam_e, double *mu);
kq_status qp_set_state(kq_handle h, const double *x, const double *s_lA,
                       const double *s_uA, const double *s_lx,
                       const double *s_ux, const double *lam_lA,
                       const double *lam_uA, const double *lam_lx,
                       const double *lam_ux, const double *lam_e, double mu);

/* qp_residuals: residual blocks of Eq. (7) at the current iterate and mu
 * (scaled units): r_H (n), r_lA, r_uA, r_c1, r_c2 (m), r_lx, r_ux, r_c3,
 * r_c4 (n), r_e (me), plus the doubly augmented right-hand side of Eq. (9)
 * rhs (NKP) and *norm = ||r||_2.  Any pointer may be NULL. */
kq_status qp_residuals(kq_handle h, double *r_H, double *r_lA, double *r_uA,
                       double *r_c1, double *r_c2, double *r_lx, double *r_ux,
                       double *r_c3, double *r_c4, double *r_e, double *rhs,
                       double *norm);

/* Scale factors chosen at create: *sigma, rhoA (m), rhoC (me). */
kq_status qp_scaling(kq_handle h, double *sigma, double *rhoA, double *rhoC);

/* Sizes: n, m, me, NKP. */
kq_status qp_sizes(kq_handle h, int64_t *n, int64_t *m, int64_t *me, int64_t *nkp);

const char *qp_last_error(kq_handle h);
void qp_destroy(kq_handle h);

/* ------------------------------------------------------------------------
 * Batched solve of many dense QPs of uneven size (Algorithm 1 in lock step
 * over the batch; each IPM iteration runs ONE persistent PCG launch for every
 * QP still iterating, with teams of CTAs sized by each QP's bytes per K*v
 * product).  The paper solves one QP at a time; batching is this library's
 * packaging of the same method.
 * ------------------------------------------------------------------------ */
typedef struct kq_batch_s *kq_batch;

/* One QP of a batch: the arguments of qp_create (H must be DENSE; every QP of a
 * batch stores H and A in the same types: BF16 H with F32 A, or F64 / F64). */
typedef struct {
  int64_t n;
  kq_hop H;
  const double *p;
  kq_amat A;             /* kind KQ_A_NONE for no general rows                */
  const double *lA, *uA;
  int64_t me;
  const double *C, *b;
  const double *lx, *ux;
} kq_qp_desc;

typedef struct {
  int converged;         /* QPs that met the mu rule                          */
  int ipm_iters_max;     /* lock-step IPM iterations run                      */
  long long ipm_iters_total;
  long long pcg_iters;   /* summed over QPs                                   */
  int pcg_maxit_hits;
  int max_active;
  double pcg_kernel_ms;  /* device time of the batched PCG launches (graph:   */
                         /* of the whole replayed iterations)                 */
  long long pcg_launches;
  double time_s;
  int graph_captures;    /* opts.graph: captures (one, plus one each time QPs */
                         /* finished) and replays of the lock-step iteration  */
  int graph_replays;
} kq_batch_stats;

/* Create nqp QPs (copies of the inputs, as qp_create) ordered on `stream`. */
kq_status qp_create_batch(kq_batch *out, int nqp, const kq_qp_desc *descs, void *stream);
/* Solve all QPs from their initial points.  x: nqp pointers (host or device,
 * n_i doubles each, original units; NULL entries skipped).  status: nqp codes
 * (KQ_OK or KQ_ERR_IPM_MAXIT).  Returns KQ_OK when every QP converged. */
kq_status ipm_solve_batch(kq_batch b, const kq_ipm_opts *opts, double *const *x, int *status,
                          kq_batch_stats *stats);
kq_status qp_batch_info(kq_batch b, int *nqp, int64_t *n);
/* QP i's IPM iterations and PCG iterations in the last ipm_solve_batch. */
kq_status qp_batch_qp_stats(kq_batch b, int i, int *ipm_iters, long long *pcg_iters);
/* Autotuner support for the batched products (no paper counterpart).
 * qp_batch_time_product: device time (ms, mean over reps launches after one
 * warm-up) of one K*v product of QP i alone, on a team of `team` CTAs, in
 * KQ_PREC_F64 or KQ_PREC_MIXED arithmetic, with the column-blocked A' pass
 * from n >= colpass_min_n on (0: the current setting).
 * qp_batch_set_tuning: the table the scheduler then uses, per size bucket
 * k = floor(log2 n) (k >= nbuckets uses the last): team_cap[k] CTAs at most per
 * QP and t_prod_us[k] (one product on one CTA) as the QP's cost per iteration;
 * colpass_min_n as above.  nbuckets = 0 restores the default (cost = bytes per
 * product, no cap, colpass from n = 512). */
kq_status qp_batch_time_product(kq_batch b, int i, int team, int precision, int colpass_min_n,
                                int reps, double *ms);
kq_status qp_batch_set_tuning(kq_batch b, int nbuckets, const int *team_cap,
                              const double *t_prod_us, int colpass_min_n);

/* The current iterate of QP i of the batch (after ipm_solve_batch: its final
 * iterate) in original units, as ipm_solve returns it: x (n_i), lam_lA, lam_uA
 * (m_i, zero where the bound is absent), lam_lx, lam_ux (n_i), lam_e (me_i).
 * Any pointer may be NULL; host or device memory.  Synchronises the batch's
 * stream. */
kq_status qp_batch_solution(kq_batch b, int i, double *x, double *lam_lA, double *lam_uA,
                            double *lam_lx, double *lam_ux, double *lam_e);
const char *qp_batch_last_error(kq_batch b);
const char *kq_batch_error(void);
void qp_batch_destroy(kq_batch b);

/* kkt_pcg_solve_static: the same persistent Jacobi-PCG solve of the doubly
 * augmented system, for callers that cannot allocate device memory (a fixed,
 * pre-reserved memory budget; an allocator that must not be bypassed).  The
 * paper has no counterpart; this is a packaging of the library's dense PCG
 * kernel.  It allocates nothing: its work space is one static device array of
 * about 0.76 MB that every GPU loading the library holds until the process
 * exits, shared by all calls.
 *  n, m      0 < n <= 4096, 0 <= m <= 4096; larger sizes return KQ_ERR_ARG
 *  H         n x n symmetric (row-major, FP64, device), already scaled
 *  A         m x n general rows (row-major, FP64, device), all two-sided
 *  Dl, Du    m each (device): the D blocks, finite and > 0 (else KQ_ERR_ARG)
 *  dg        n (device): the bound term of Q = H + diag(dg)
 *  rhs, sol  n + 2m (device), layout [x | lam_l | lam_u]; z0 = 0
 *  tol       relative unpreconditioned residual; maxit iterations
 *  stream    cudaStream_t or NULL; *iters, *rel_res (recursive) may be NULL
 * All pointers must be device memory.  The first call on a device looks up
 * the array's device address; make that first call before any stream capture.
 * Every call waits for its stream (it reads status words back) before it
 * returns.  The array keeps the last call's contents (its counters are
 * cleared on entry), so calls that overlap on the GPU race: serialise them.
 * Calls after cudaDeviceReset are not supported.  KQ_WARN_PCG_MAXIT if the
 * tolerance was not met; errors are reported by kq_global_error(). */
kq_status kkt_pcg_solve_static(int64_t n, int64_t m, const double *H, const double *A,
                               const double *Dl, const double *Du, const double *dg,
                               const double *rhs, double *sol, double tol, int maxit,
                               void *stream, int *iters, double *rel_res);

/* kq_barrier_selftest: self-test of the bounded device waits that every
 * persistent kernel relies on (section 3.2's PCG runs as one cooperative
 * launch with grid barriers; no paper counterpart).  Launches `ctas` CTAs
 * that each enter the library's grid barrier once with an arrival target one
 * above the CTAs launched, so the barrier cannot complete; each CTA gives up
 * after budget_s seconds (0 < budget_s <= 5) and records KQ_ERR_TIMEOUT.
 * Returns KQ_ERR_TIMEOUT (expected), *gave_up = CTAs that gave up,
 * *elapsed_ms = device time of the launch.  The CUDA context stays usable.
 * Synchronises the device; allocates four words (freed before return). */
kq_status kq_barrier_selftest(int ctas, double budget_s, int *gave_up, double *elapsed_ms);

/* Library-wide: message of the last failure of a call that had no handle
 * (qp_create). */
const char *kq_global_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KKTQP_H */
