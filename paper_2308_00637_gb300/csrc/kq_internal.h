// Internal structures of the Krylov IPM library (host + device views).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>
#include "../../include/kktqp.h"

// Device view of a scaled problem (all pointers are device memory).
struct DevProb {
  int64_t n = 0, m = 0, me = 0, nkp = 0;
  int hkind = 0, hdtype = 0;
  double hscale = 1.0;               // sigma (DENSE, LOWRANK): H_scaled = hscale * H
  double wfac = 1.0;                 // CSR_LSQ: sigma / (sigma at create), applied to the
                                     // FP32 row tables (the FP64 w2 is rescaled in place)
  float wfac32 = 1.f;                // wfac in FP32 (FP32 products)
  // DENSE H (scaled by sigma), n x n row-major with leading dimension hld
  // (rows padded with zeros to a multiple of 8 entries; 0 means n)
  const void *Hd = nullptr;
  int64_t hld = 0, ald = 0;
  // CSR_LSQ: H = P' diag(w2) P, w2 = 2 sigma w
  int64_t nP = 0, nnz = 0;
  const int64_t *rowptr = nullptr;
  const int32_t *col = nullptr;
  const float *val = nullptr;
  const double *w2 = nullptr;
  const int32_t *prow2a = nullptr;   // nP: A-row id or -1
  const int32_t *arows = nullptr;    // m: P row of A row
  // LOWRANK: H = sigma (Z diag(zw) Z' + diag(d0)), Z n x k row-major
  int64_t k = 0;
  const void *Z = nullptr;
  const double *zw = nullptr;        // k column weights (null: all 1)
  const double *d0 = nullptr;        // n diagonal H0, unscaled (null: 0)
  // general rows, stored unscaled (the row scale rhoA is applied on the fly):
  // DENSE m x n row-major (leading dimension ald), or CSR (arowptr, acol, aval)
  int akind = 0, adtype = 0;
  const void *Ad = nullptr;
  const int64_t *arowptr = nullptr;  // CSR: m + 1
  const int32_t *acol = nullptr;     // CSR: annz
  const void *aval = nullptr;        // CSR: annz values (adtype)
  int64_t annz = 0;
  const double *rhoA = nullptr;      // m: 1 / ||A_i||_2
  const double *lA = nullptr, *uA = nullptr;   // scaled, m
  const uint8_t *hasl = nullptr, *hasu = nullptr;
  // equality rows (scaled), me x n row-major, and rhs
  const double *Cd = nullptr, *b = nullptr;
  const double *p = nullptr;         // scaled linear term
  const double *lx = nullptr, *ux = nullptr;
  const uint8_t *haslx = nullptr, *hasux = nullptr;
  const double *hdiag = nullptr;     // diag(H) scaled (zeros for CSR_LSQ: added in pass)
  // device-side control (the batched solver's captured graph): when set, the
  // IPM kernels return at once unless *gate != 0, mu is read from *mu_dev and
  // the step lengths from axal[0..1]
  const int *gate = nullptr;
  const double *mu_dev = nullptr;
  const double *axal = nullptr;
};

// Per-QP state of the batched solver's device-side control (captured graph).
struct QpCtl {
  int active;        // Algorithm 1 still iterating (gate of the IPM kernels)
  int ran;           // ran a PCG pass in the current pass (gate of its follow-up)
  int pcg_done;      // the current Newton solve has finished
  int fp32_ok;       // FP32 correction passes still pay for this QP
  int used;          // PCG iterations of the current Newton solve
  int w_prev;        // PCG iterations of the previous Newton solve (team costs)
  int f32_pays;      // MIXED: this QP's products are large enough for FP32 passes
  int kexp;          // mu = mu0 10^-kexp
  int ipm_iters;
  int status;        // KQ_OK once converged; an error code if a step failed
  int maxit_hits;    // Newton solves stopped at the iteration cap
  int prec;          // precision of the current pass
  long long pcg_iters;
  double mu, bnorm, resn, resn_before, tol_rel;
  double ax, al;     // step lengths of the current iteration (Eq. (10))
};

// Device state of the iterate (scaled units).
struct DevState {
  double *x, *slx, *sux, *llx, *lux;  // n
  double *sl, *su, *ll, *lu;          // m
  double *le;                         // me
};

// Per-iterate KKT data produced by the residual pass.
struct DevKKT {
  double *Dl, *Du, *cl, *cu;   // m: D blocks and masked inverses
  double *dg;                  // n
  double *diag;                // nkp Jacobi diagonal
  double *rhs;                 // nkp doubly augmented rhs
  double *rH, *rlx, *rux, *rc3, *rc4;   // n
  double *rlA, *ruA, *rc1, *rc2;        // m
  double *re;                           // me
  double mu;
};

// CSR staging tables.  A chunk is a run of consecutive rows of P whose
// nonzeros (rounded out to 16-byte boundaries) fit one shared-memory stage.
// Its descriptors are [header, one per row, sentinel]:
//   header   {off = number of rows, a = -1, or the row index of a single
//             over-long row that is read from global memory}
//   row      {off = start of the row inside the staged chunk, a = A-row id or -1,
//             w2 = 2 sigma w_r as an FP32 pair hi + lo (hi alone in FP32
//             products; hi + lo, 48 significant bits, in FP64 products)}
//   sentinel {off = end of the last row}
struct RowDesc { int32_t off; int32_t a; float w2hi; float w2lo; };
struct ChunkInfo { int64_t src; int32_t nelem; int32_t desc0; int32_t ndesc; int32_t pad; };

// Register-streamed CSR layout (FP32 products, rows of at most 128 nonzeros,
// column windows of at most 65536).  Each row's nonzeros are padded to a
// multiple of four and stored as groups of four (one 16-byte load of values
// and one 8-byte load of 16-bit window-relative columns per lane); slot
// 4*l + q of a row belongs to lane l, load component q.  The host
// permutes a row's nonzeros so that the 32 lanes of one component hit
// distinct shared-memory banks where the row allows.
struct RowSlot { int32_t off4; int32_t len4; int32_t a; float w2; };
constexpr int KQ_MAX_STAGES = 8;

// Shared-memory layout of the staged CSR kernel (byte offsets), identical on
// host (to size the launch) and device.
struct CsrLayout {
  size_t pw, acc, arho, acs, aDl, aDu, apl, apu, afl, tab, stage0, stage_bytes, val_off,
      col_off, desc_off, bar, total;
};
__host__ __device__ inline size_t kq_up128(size_t x) { return (x + 127) & ~(size_t)127; }
__host__ __device__ inline CsrLayout csr_layout(int win_cap, int a_cap, int ch_cap, int desc_cap,
                                                int tab_cap, int stages) {
  CsrLayout L;
  size_t o = 0;
  L.pw = o; o = kq_up128(o + 8 * (size_t)win_cap);
  L.acc = o; o = kq_up128(o + 8 * (size_t)win_cap);
  L.arho = o; o += 8 * (size_t)a_cap;
  L.acs = o; o += 8 * (size_t)a_cap;
  L.aDl = o; o += 8 * (size_t)a_cap;
  L.aDu = o; o += 8 * (size_t)a_cap;
  L.apl = o; o += 8 * (size_t)a_cap;
  L.apu = o; o += 8 * (size_t)a_cap;
  L.afl = o; o = kq_up128(o + (size_t)a_cap);
  L.tab = o; o = kq_up128(o + sizeof(ChunkInfo) * (size_t)tab_cap);
  L.val_off = 0;
  L.col_off = kq_up128(4 * (size_t)ch_cap);
  L.desc_off = L.col_off + kq_up128(4 * (size_t)ch_cap);
  L.stage_bytes = L.desc_off + kq_up128(16 * (size_t)desc_cap);
  L.stage0 = o; o += (size_t)stages * L.stage_bytes;
  L.bar = o; o += 8 * (size_t)stages;
  L.total = kq_up128(o);
  return L;
}

constexpr int KQ_LANCZOS_CAP = 5000;   // PCG iterations whose coefficients are kept

// Work space of the persistent PCG kernels.
struct PcgWork {
  int G = 0;                   // CTAs of the cooperative launch
  int threads = 0;
  int win_cap = 0;             // smem window capacity (elements)
  size_t smem = 0;             // dynamic smem bytes
  double *r = nullptr, *y = nullptr, *pb0 = nullptr, *pb1 = nullptr;
  double *qlam = nullptr;      // me + 2m
  double *accx64 = nullptr;    // n
  float *accx32 = nullptr;     // n
  double *g64 = nullptr;       // k + me (LOWRANK)
  double *coefA = nullptr;     // m (DENSE column pass)
  double *dinv = nullptr;      // nkp: 1 / diag(K) of the current solve
  double *lanczos = nullptr;   // 2 * KQ_LANCZOS_CAP: PCG alpha, beta (records)
  float *p32_0 = nullptr, *p32_1 = nullptr, *y32 = nullptr;  // nkp FP32 copies (register-streamed CSR)
  double *slots = nullptr;     // 4 * G
  unsigned int *bar = nullptr; // [count, gen]
  int *err = nullptr;          // device error flag
  int *iters = nullptr;        // device iteration count
  double *resn = nullptr;      // device final recursive residual^2, bb
  ChunkInfo *chunks = nullptr;
  int32_t *cta_chunk = nullptr;
  RowDesc *rdesc = nullptr;
  int32_t *a_lo = nullptr, *a_hi = nullptr;
  int a_cap = 0, ch_cap = 0, desc_cap = 0, tab_cap = 0;
  int stages = 4, copy_piece = 16384, producer = 0;
  // register-streamed CSR operator (FP32 products)
  bool rows_ok = false;
  RowSlot *rslot = nullptr;    // nP
  float *rval = nullptr;       // 4 * sum(len4)
  uint16_t *rcol = nullptr;    // 4 * sum(len4), 16-bit offsets from the CTA's window start
  int rws = 0;                 // stride of the per-warp accumulators (floats)
  int stag_window = 200;       // FP32 pass stagnation window (iterations)
  int pf_dist = 0;             // L2 prefetch distance in warp steps (0: off)
  size_t smem_rows = 0;
  float *rw2lo = nullptr;      // nP: low part of the FP32-split row weight (FP64 products)
  bool rows64_ok = false;      // FP64 products also register-streamed
  size_t smem_rows64 = 0;
  int threads_rows64 = 256;
  int64_t *row_begin = nullptr;   // G+1 partition of rows (P rows / dense rows)
  int32_t *win_lo = nullptr, *win_hi = nullptr;  // G column windows (CSR)
  int *h_pinned = nullptr;     // pinned host mirror for status words
};

struct kq_problem {
  int dev = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  int64_t n = 0, m = 0, me = 0, nkp = 0;
  double sigma = 1.0;
  double sigma_create = 1.0;    // sigma when the row tables were built
  double hmax = 0.0;            // max_i H_ii of the unscaled H (for sigma)
  DevProb P;
  DevState S;
  DevKKT K;
  PcgWork W;
  std::vector<void *> allocs;   // every device allocation, freed at destroy
  // scratch for IPM kernels
  double *hx = nullptr, *t = nullptr, *tC = nullptr, *acc1 = nullptr, *acc2 = nullptr,
         *acc3 = nullptr, *yP = nullptr, *g = nullptr;
  double *z = nullptr, *zref = nullptr, *tmp = nullptr;
  double *dsl = nullptr, *dsu = nullptr, *dslx = nullptr, *dsux = nullptr, *dllx = nullptr,
         *dlux = nullptr;
  double *red = nullptr;        // reduction partials
  double *red_out = nullptr;    // reduction results (device)
  double *h_red = nullptr;      // pinned host mirror of results
  double inf2[3] = {0, 0, 0};   // squared primal, dual, complementarity norms (section 5.2)
  double *rhoC = nullptr;       // equality row scales (me)
  int *dflags = nullptr;        // reduction kind flags (8)
  bool state_set = false;       // qp_set_state supplied the starting iterate
  double mu = 1.0;
  int mu_exp = 0;
  bool kkt_valid = false;       // K data matches the current state and mu
  bool solved = false;          // a converged ipm_solve ran
  int num_sms = 0;
  double timeout_s = 2.0;
  long long launches = 0;       // kernels launched by this handle
  float last_kernel_ms = 0.f;   // device time of this handle's last persistent PCG launch
  long long pcg_launches = 0;   // persistent PCG launches (solve + apply)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // per-IPM-iteration records (opts.record)
  bool record = false;
  bool warm_next = false;      // the next pcg_solve starts from the z it is given          // the current ipm_solve keeps records
  bool lz_on = false;           // the next PCG launch writes its alpha, beta
  int lz_steps = 0;             // Lanczos estimates of the last recorded pass
  double lz_min = 0.0, lz_max = 0.0;
  std::vector<kq_ipm_iter> iter_log;
  // batched solver's captured graph: reductions stay on the device, and the
  // vector helpers of a correction pass run only when *vec_gate != 0
  bool graph_mode = false;
  const int *vec_gate = nullptr;
  // batched solver: this QP's totals over the last ipm_solve_batch
  long long batch_pcg_iters = 0;
  int batch_ipm_iters = 0;
};

// ---------------------------------------------------------------- host helpers
kq_status kq_fail(kq_problem *h, kq_status st, const std::string &msg);
#define KQ_CUDA(h, call)                                                       \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return kq_fail((h), KQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// pcg.cu
kq_status pcg_setup(kq_problem *h, int grid_ctas);
// Solve K z = rhs (device pointers, padded layout) with Jacobi PCG.
kq_status pcg_solve(kq_problem *h, const double *rhs, double *z, const kq_pcg_opts &o,
                    kq_pcg_stats *st);
// out = K v in FP64 (prec = KQ_PREC_F64) or mixed arithmetic.
kq_status pcg_apply(kq_problem *h, const double *v, double *out, int prec, float *ms);
double pcg_last_kernel_ms(const kq_problem *h);
// Lanczos extreme eigenvalues from the alpha, beta of the last recorded pass
void lanczos_extremes(kq_problem *h, int iters);
// Work buffers of one persistent PCG launch, provided by the caller.
struct PcgRawWork {
  double *r, *y, *pb0, *pb1, *qlam, *slots, *resn;
  void *accx;
  unsigned int *bar;
  int *err, *iters;
};
kq_status pcg_dense_raw(const DevProb &P, const double *Dl, const double *Du, const double *cl,
                        const double *cu, const double *dg, const double *diag, const double *rhs,
                        double *z, const PcgRawWork &w, int G, double tol, int maxit,
                        double timeout_s, cudaStream_t stream, int *iters, double *rr,
                        double *bb, std::string *msg);

// batched dense PCG (pcg.cu)
// Tuning of the batched dense products (the autotuner's table, per size
// bucket floor(log2 n)): measured time of one K*v product on one CTA (the
// scheduler's cost), the team size beyond which it stops paying, and the n
// from which the A' part runs as the column-blocked second pass.
struct BatchTune {
  std::vector<int> team_cap;
  std::vector<double> t_prod_us;
  int colpass_min_n = 512;
  int force_team = 0;          // timing runs: the team size of the single problem
};

struct BatchPcg {
  int nqp = 0, G = 0, max_n = 0;
  BatchTune tune;
  // captured-graph path: three argument arrays (FP32 solve, FP64 solve, FP64
  // apply), per-QP control, status words of the three launch kinds
  unsigned char *gargs = nullptr;
  QpCtl *ctl = nullptr;
  double **redout = nullptr;       // per QP: its handle's reduction results
  int *g_iters = nullptr, *g_err = nullptr;
  double *g_resn = nullptr;
  int *d_count = nullptr, *h_count = nullptr;
  int gblocks = 0;
  size_t gsmem[3] = {0, 0, 0};
  // device-side team plan before every correction pass (dev_sched): the
  // per-product cost and the team-size cap of every QP
  int dev_sched = 0;
  double *q_cost = nullptr;
  int *q_cap = nullptr;
  std::vector<void *> allocs;
  unsigned char *args = nullptr, *teams = nullptr;
  int *cta_team = nullptr, *team_qps = nullptr;
  int *d_iters = nullptr, *d_err = nullptr;
  double *d_resn = nullptr;
  unsigned char *h_status = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long long launches = 0;
};
kq_status batch_pcg_setup(BatchPcg &B, int nqp, int sms, int max_n, std::string &err);
void batch_pcg_free(BatchPcg &B);
kq_status batch_pcg_launch(BatchPcg &B, const std::vector<kq_problem *> &hs,
                           const std::vector<int> &idx, const std::vector<const double *> &rhs,
                           const std::vector<double *> &out, const std::vector<double> &tol,
                           const std::vector<int> &maxit, int apply, int prec, cudaStream_t s,
                           std::vector<int> &iters, std::vector<int> &errs,
                           std::vector<double> &rr, std::vector<double> &bb, float *ms,
                           std::string &err, const std::vector<double> *weight = nullptr);

// captured-graph path of the batched solver (pcg.cu): per-QP argument arrays
// and teams over the problems with weight > 0, the three kinds of batched
// launch, and the device-side control kernels (QpCtl)
kq_status batch_graph_prepare(BatchPcg &B, const std::vector<kq_problem *> &hs,
                              const std::vector<double> &weight, std::string &err);
kq_status batch_graph_launch(BatchPcg &B, const kq_problem *h0, int which, cudaStream_t s,
                             std::string &err);
void batch_graph_pcg_init(BatchPcg &B, int mixed, cudaStream_t s);
void batch_graph_pass_setup(BatchPcg &B, int pass, const kq_pcg_opts &o, cudaStream_t s);
void batch_graph_schedule(BatchPcg &B, cudaStream_t s);
// MIXED in a batch: FP32 correction passes only for a QP whose product reads
// at least the L2's capacity.  Smaller products are latency-bound in a batch,
// and the lock-step passes put a QP's FP32 correction passes behind the other
// QPs' FP64 pass, so the FP32 passes cost more than they save there.
constexpr double KQ_BATCH_F32_MIN_BYTES = 128.0e6;
bool batch_f32_pays(const kq_problem *h);
void batch_graph_pass_finish(BatchPcg &B, int pass, int last, int maxit, cudaStream_t s);
void batch_graph_step(BatchPcg &B, double gamma, cudaStream_t s);
void batch_graph_mu_rule(BatchPcg &B, double mu0, double mu_tol, cudaStream_t s);
void batch_graph_count(BatchPcg &B, cudaStream_t s);

// ipm kernels (ipm.cu)
kq_status kkt_assemble(kq_problem *h);   // residuals, rhs, D, diag at state & mu
kq_status init_state(kq_problem *h);
kq_status reduce_async(kq_problem *h, int ncols, int min_mask, int off);
kq_status assemble_enqueue(kq_problem *h);                      // -> h_red[0..2]
void assemble_finish(kq_problem *h, double *norm2, double *rH2);
kq_status recover_enqueue(kq_problem *h);                       // -> h_red[4..5]
void recover_finish(kq_problem *h, double gamma, double *ax, double *al);
kq_status update_enqueue(kq_problem *h, double ax, double al);
kq_status outputs_enqueue(kq_problem *h, double *x, double *lam_lA, double *lam_uA,
                          double *lam_lx, double *lam_ux, double *lam_e);
kq_status vec_add_enqueue(kq_problem *h, double *z, const double *dz);
kq_status vec_resid_enqueue(kq_problem *h, const double *rhs, const double *kz, double *res);  // -> h_red[8]
