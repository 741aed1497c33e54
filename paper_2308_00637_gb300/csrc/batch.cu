// Batched solve of many dense convex QPs of uneven size (Algorithm 1 run in
// lock step over the batch).  Each QP keeps its own device data (created with
// qp_create on the batch's stream); per IPM iteration the whole batch shares
// ONE persistent PCG launch in which teams of CTAs, sized by each QP's bytes
// per product, run the QPs' Jacobi-PCG solves concurrently (pcg.cu).  The
// per-QP residual, recovery and update kernels are enqueued for every active
// QP with one host synchronisation per phase.
#include "common.cuh"
#include "kq_internal.h"
#include <chrono>
#include <cstdio>
#include <cmath>
#include <string>
#include <vector>

struct kq_batch_s {
  cudaStream_t stream = nullptr;
  std::vector<kq_problem *> qps;
  BatchPcg B;
  std::string err;
  int max_n = 0;
};

namespace {
thread_local std::string g_batch_err;

kq_status bfail(kq_batch b, kq_status st, const std::string &msg) {
  if (b) b->err = msg;
  else g_batch_err = msg;
  return st;
}

// Batched Jacobi-PCG with the same refinement as the single-problem solver:
// z = 0; res = rhs; passes of {solve K dz = res (FP32 products while the
// refinement budget lasts, then FP64); z += dz; res = rhs - K z in FP64}.
kq_status batch_pcg(kq_batch b, const std::vector<int> &act, const kq_pcg_opts &o,
                    std::vector<long long> &iters_out, std::vector<int> &maxit_hit,
                    double *kernel_ms, const std::vector<double> &last_iters) {
  auto &hs = b->qps;
  const int k = (int)act.size();
  cudaStream_t s = b->stream;
  std::vector<double> bnorm(k, 0.0), resn(k, 0.0);
  std::vector<int> used(k, 0), done(k, 0);
  iters_out.assign(k, 0);
  maxit_hit.assign(k, 0);
  for (int j = 0; j < k; ++j) {
    kq_problem *h = hs[act[j]];
    if (cudaMemsetAsync(h->z, 0, h->nkp * sizeof(double), s) != cudaSuccess ||
        cudaMemcpyAsync(h->tmp, h->K.rhs, h->nkp * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return bfail(b, KQ_ERR_CUDA, "batch PCG init");
  }
  const int mixed = o.precision == KQ_PREC_MIXED;
  const int max_passes = (mixed ? o.refine_steps : 0) + 3;
  // per QP: FP32 correction passes only for QPs whose products are large
  // enough (batch_f32_pays), and while they pay (a pass that does not halve
  // the true residual hands that QP to FP64 passes)
  std::vector<int> fp32_ok(k, 0);
  for (int j = 0; j < k; ++j) fp32_ok[j] = mixed && batch_f32_pays(hs[act[j]]);
  std::vector<double> resn_before(k, 0.0);
  for (int pass = 0; pass < max_passes; ++pass) {
    std::vector<int> idx;
    std::vector<int> map;
    std::vector<int> pprec;
    for (int j = 0; j < k; ++j) {
      if (done[j]) continue;
      const int budget = o.maxit - used[j];
      if (budget <= 0) { done[j] = 1; continue; }
      idx.push_back(act[j]);
      map.push_back(j);
      pprec.push_back((fp32_ok[j] && pass < o.refine_steps) ? KQ_PREC_MIXED : KQ_PREC_F64);
      resn_before[j] = resn[j];
    }
    if (idx.empty()) break;
    // one launch per precision group
    for (int prec : {KQ_PREC_MIXED, KQ_PREC_F64}) {
      std::vector<int> gidx, gmap;
      std::vector<const double *> rhs;
      std::vector<double *> out;
      std::vector<double> tol, wts;
      std::vector<int> maxit;
      for (size_t q = 0; q < idx.size(); ++q) {
        if (pprec[q] != prec) continue;
        const int j = map[q];
        kq_problem *h = hs[act[j]];
        double rel = pass == 0 ? o.tol : o.tol * bnorm[j] / std::max(resn[j], 1e-300);
        if (prec == KQ_PREC_MIXED) rel = std::max(rel, o.inner_tol);
        rel = std::min(rel, 0.5);
        gidx.push_back(act[j]);
        gmap.push_back(j);
        rhs.push_back(h->tmp);
        out.push_back(h->zref);
        tol.push_back(rel);
        maxit.push_back(o.maxit - used[j]);
        wts.push_back(last_iters[act[j]]);
      }
      if (gidx.empty()) continue;
      std::vector<int> its, errs;
      std::vector<double> rr, bb;
      float ms = 0.f;
      std::string e;
      kq_status rc = batch_pcg_launch(b->B, hs, gidx, rhs, out, tol, maxit, 0, prec, s, its, errs,
                                      rr, bb, &ms, e, &wts);
      if (rc != KQ_OK) return bfail(b, rc, e);
      *kernel_ms += ms;
      for (size_t q = 0; q < gidx.size(); ++q) {
        const int j = gmap[q];
        if (errs[q] != 0)
          return bfail(b, errs[q] == 7 ? KQ_ERR_TIMEOUT : (errs[q] == 4 ? KQ_ERR_NOT_CONVEX : KQ_ERR_NUMERIC),
                       "batched PCG failed on QP " + std::to_string(act[j]));
        if (pass == 0) bnorm[j] = std::sqrt(bb[q]);
        used[j] += its[q];
        iters_out[j] += its[q];
        kq_problem *h = hs[act[j]];
        vec_add_enqueue(h, h->z, h->zref);
      }
    }
    std::vector<int> its, errs;
    std::vector<double> rr, bb;
    float ms = 0.f;
    std::string e;
    kq_status rc;
    // FP64 K z for every QP of this pass in one launch, then res = rhs - K z
    std::vector<const double *> zin;
    std::vector<double *> kz;
    for (size_t q = 0; q < idx.size(); ++q) {
      kq_problem *h = hs[idx[q]];
      zin.push_back(h->z);
      kz.push_back(h->zref);
    }
    std::vector<double> tol0(idx.size(), 0.0);
    std::vector<int> mx0(idx.size(), 0);
    rc = batch_pcg_launch(b->B, hs, idx, zin, kz, tol0, mx0, 1, KQ_PREC_F64, s, its, errs, rr, bb,
                          &ms, e);
    if (rc != KQ_OK) return bfail(b, rc, e);
    *kernel_ms += ms;
    for (size_t q = 0; q < idx.size(); ++q) {
      kq_problem *h = hs[idx[q]];
      vec_resid_enqueue(h, h->K.rhs, h->zref, h->tmp);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch PCG sync");
    for (size_t q = 0; q < idx.size(); ++q) {
      const int j = map[q];
      resn[j] = std::sqrt(hs[idx[q]]->h_red[8]);
      if (!(resn[j] == resn[j])) return bfail(b, KQ_ERR_NUMERIC, "batched PCG residual NaN");
      if (pprec[q] == KQ_PREC_MIXED && pass > 0 && resn[j] > 0.5 * resn_before[j]) fp32_ok[j] = 0;
      if (pprec[q] == KQ_PREC_MIXED && pass == 0 && resn[j] > 0.5 * bnorm[j]) fp32_ok[j] = 0;
      if (resn[j] <= o.tol * bnorm[j] || bnorm[j] == 0.0) done[j] = 1;
      else if (used[j] >= o.maxit) { done[j] = 1; maxit_hit[j] = 1; }
    }
  }
  for (int j = 0; j < k; ++j)
    if (resn[j] > o.tol * bnorm[j]) maxit_hit[j] = 1;
  return KQ_OK;
}

// One lock-step IPM iteration of the batch, enqueued for stream capture:
// correction passes of the Newton solves (precision, tolerance and stop taken
// by the control kernels), step recovery, step lengths, update, residuals at
// the current mu, the mu rule, residuals at the new mu, and the count of QPs
// still iterating (copied to pinned host memory).  Only QPs active at capture
// are enqueued; the others stay inactive.
kq_status enqueue_iteration(kq_batch b, const kq_ipm_opts &o, const kq_pcg_opts &po,
                            const std::vector<int> &act) {
  auto &hs = b->qps;
  BatchPcg &B = b->B;
  cudaStream_t s = b->stream;
  std::string e;
  const int mixed = po.precision == KQ_PREC_MIXED;
  const int max_passes = (mixed ? po.refine_steps : 0) + 3;
  batch_graph_pcg_init(B, mixed, s);
  for (int q : act) {
    kq_problem *h = hs[q];
    if (cudaMemsetAsync(h->z, 0, h->nkp * sizeof(double), s) != cudaSuccess ||
        cudaMemcpyAsync(h->tmp, h->K.rhs, h->nkp * sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return bfail(b, KQ_ERR_CUDA, "batch graph: PCG init");
  }
  for (int pass = 0; pass < max_passes; ++pass) {
    batch_graph_pass_setup(B, pass, po, s);
    batch_graph_schedule(B, s);   // teams over the QPs that run in this pass
    kq_status rc;
    if ((rc = batch_graph_launch(B, hs[0], 0, s, e)) != KQ_OK) return bfail(b, rc, e);
    for (int q : act) vec_add_enqueue(hs[q], hs[q]->z, hs[q]->zref);
    if ((rc = batch_graph_launch(B, hs[0], 2, s, e)) != KQ_OK) return bfail(b, rc, e);
    for (int q : act) vec_resid_enqueue(hs[q], hs[q]->K.rhs, hs[q]->zref, hs[q]->tmp);
    batch_graph_pass_finish(B, pass, pass == max_passes - 1, po.maxit, s);
  }
  for (int q : act)
    if (recover_enqueue(hs[q]) != KQ_OK) return bfail(b, KQ_ERR_CUDA, hs[q]->err);
  batch_graph_step(B, o.gamma, s);
  for (int q : act)
    if (update_enqueue(hs[q], 0.0, 0.0) != KQ_OK || assemble_enqueue(hs[q]) != KQ_OK)
      return bfail(b, KQ_ERR_CUDA, hs[q]->err);
  batch_graph_mu_rule(B, o.mu0, o.mu_tol, s);
  for (int q : act)
    if (assemble_enqueue(hs[q]) != KQ_OK) return bfail(b, KQ_ERR_CUDA, hs[q]->err);
  batch_graph_count(B, s);
  if (cudaGetLastError() != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch graph: enqueue");
  return KQ_OK;
}

void graph_mode(kq_batch b, bool on) {
  for (size_t q = 0; q < b->qps.size(); ++q) {
    kq_problem *h = b->qps[q];
    QpCtl *c = b->B.ctl + q;
    h->P.gate = on ? &c->active : nullptr;
    h->P.mu_dev = on ? &c->mu : nullptr;
    h->P.axal = on ? &c->ax : nullptr;   // ax, al adjacent in QpCtl
    h->vec_gate = on ? &c->ran : nullptr;
    h->graph_mode = on;
  }
}

// Algorithm 1 over the batch with the lock-step iteration replayed from a
// CUDA graph; the graph is captured again (teams rebalanced over the QPs
// still iterating, weighted by their last Newton solve's iterations) only
// when QPs have finished.
kq_status ipm_solve_batch_graph_on(kq_batch b, const kq_ipm_opts &o, double *const *x,
                                   int *status, kq_batch_stats *stats);

// Stream capture needs a stream other than the legacy default stream: when
// the batch was created on the default stream, the graph path runs on a
// private non-blocking stream (ordered after the default stream's work) and
// hands the handles back their stream afterwards.
kq_status ipm_solve_batch_graph(kq_batch b, const kq_ipm_opts &o, double *const *x, int *status,
                                kq_batch_stats *stats) {
  if (b->stream) return ipm_solve_batch_graph_on(b, o, x, status, stats);
  cudaStream_t ps = nullptr;
  if (cudaStreamSynchronize(nullptr) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) != cudaSuccess)
    return bfail(b, KQ_ERR_CUDA, "batch graph: private stream");
  b->stream = ps;
  for (kq_problem *h : b->qps) h->stream = ps;
  const kq_status rc = ipm_solve_batch_graph_on(b, o, x, status, stats);
  cudaStreamSynchronize(ps);
  b->stream = nullptr;
  for (kq_problem *h : b->qps) h->stream = nullptr;
  cudaStreamDestroy(ps);
  return rc;
}

kq_status ipm_solve_batch_graph_on(kq_batch b, const kq_ipm_opts &o, double *const *x,
                                   int *status, kq_batch_stats *stats) {
  auto t0 = std::chrono::steady_clock::now();
  auto &hs = b->qps;
  BatchPcg &B = b->B;
  const int nq = (int)hs.size();
  cudaStream_t s = b->stream;
  kq_pcg_opts po;
  po.tol = o.pcg_tol; po.maxit = o.pcg_maxit; po.precision = o.precision;
  po.refine_steps = o.refine_steps; po.inner_tol = o.inner_tol;
  kq_batch_stats st{};
  for (kq_problem *h : hs) {
    h->timeout_s = o.timeout_s > 0 ? o.timeout_s : 2.0;
    h->solved = false;
    h->state_set = false;
    h->mu = o.mu0;
    if (init_state(h) != KQ_OK || assemble_enqueue(h) != KQ_OK) return bfail(b, KQ_ERR_CUDA, h->err);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch init");
  double n2;
  for (kq_problem *h : hs) assemble_finish(h, &n2, nullptr);
  std::vector<double> weight(nq, 1.0);
  std::string e;
  kq_status rc = batch_graph_prepare(B, hs, weight, e);   // allocates the control words
  if (rc != KQ_OK) return bfail(b, rc, e);
  std::vector<QpCtl> ctl(nq);
  for (int q = 0; q < nq; ++q) {
    QpCtl &c = ctl[q];
    c = QpCtl{};
    c.active = 1;
    c.mu = o.mu0;
    c.status = KQ_ERR_IPM_MAXIT;
    c.f32_pays = batch_f32_pays(hs[q]);
  }
  if (cudaMemcpy(B.ctl, ctl.data(), nq * sizeof(QpCtl), cudaMemcpyHostToDevice) != cudaSuccess)
    return bfail(b, KQ_ERR_CUDA, "batch graph: control words");
  graph_mode(b, true);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int captured = nq, it = 0, count = nq;
  double ms_total = 0.0;
  kq_status out = KQ_OK;
  for (it = 1; it <= o.ipm_maxit; ++it) {
    if (!exec) {
      std::vector<int> act;
      for (int q = 0; q < nq; ++q)
        if (weight[q] > 0.0) act.push_back(q);
      if ((rc = batch_graph_prepare(B, hs, weight, e)) != KQ_OK) { out = bfail(b, rc, e); break; }
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        out = bfail(b, KQ_ERR_CUDA, "batch graph: begin capture");
        break;
      }
      rc = enqueue_iteration(b, o, po, act);
      const cudaError_t ce = cudaStreamEndCapture(s, &graph);
      if (rc != KQ_OK) { out = rc; break; }
      if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        out = bfail(b, KQ_ERR_CUDA, std::string("batch graph: capture: ") + cudaGetErrorString(ce));
        break;
      }
      st.graph_captures++;
      captured = (int)act.size();
    }
    cudaEventRecord(B.ev0, s);
    if (cudaGraphLaunch(exec, s) != cudaSuccess) { out = bfail(b, KQ_ERR_CUDA, "batch graph: launch"); break; }
    cudaEventRecord(B.ev1, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) { out = bfail(b, KQ_ERR_CUDA, "batch graph: replay"); break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, B.ev0, B.ev1);
    ms_total += ms;
    st.graph_replays++;
    count = *B.h_count;
    if (o.verbose) {
      fprintf(stderr, "batch graph ipm %3d active %4d replay %.1f ms\n", it, count, ms);
      fflush(stderr);
    }
    if (count == 0) break;
    if (count < captured) {
      // QPs finished: rebalance the teams over the others at the next capture
      if (cudaMemcpy(ctl.data(), B.ctl, nq * sizeof(QpCtl), cudaMemcpyDeviceToHost) != cudaSuccess) {
        out = bfail(b, KQ_ERR_CUDA, "batch graph: control read-back");
        break;
      }
      for (int q = 0; q < nq; ++q) weight[q] = ctl[q].active ? std::max(1, ctl[q].used) : 0.0;
      cudaGraphExecDestroy(exec);
      cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  graph_mode(b, false);
  if (out != KQ_OK) return out;
  if (cudaMemcpy(ctl.data(), B.ctl, nq * sizeof(QpCtl), cudaMemcpyDeviceToHost) != cudaSuccess)
    return bfail(b, KQ_ERR_CUDA, "batch graph: control read-back");
  for (int q = 0; q < nq; ++q) {
    const QpCtl &c = ctl[q];
    if (x && x[q]) outputs_enqueue(hs[q], x[q], nullptr, nullptr, nullptr, nullptr, nullptr);
    if (status) status[q] = c.status;
    hs[q]->mu = c.mu;
    hs[q]->solved = c.status == KQ_OK;
    hs[q]->batch_pcg_iters = c.pcg_iters;
    hs[q]->batch_ipm_iters = c.ipm_iters;
    hs[q]->kkt_valid = false;
    st.ipm_iters_max = std::max(st.ipm_iters_max, c.ipm_iters);
    st.ipm_iters_total += c.ipm_iters;
    st.pcg_iters += c.pcg_iters;
    st.pcg_maxit_hits += c.maxit_hits;
    if (c.status == KQ_OK) st.converged++;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch outputs");
  st.max_active = nq;
  st.pcg_kernel_ms = ms_total;
  st.pcg_launches = B.launches;
  st.time_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  for (int q = 0; q < nq; ++q)
    if (ctl[q].status != KQ_OK && ctl[q].status != KQ_ERR_IPM_MAXIT)
      return bfail(b, ctl[q].status, "QP " + std::to_string(q) + " failed");
  return st.converged == nq ? KQ_OK : KQ_ERR_IPM_MAXIT;
}

}  // namespace

extern "C" {

const char *kq_batch_error(void) { return g_batch_err.c_str(); }
const char *qp_batch_last_error(kq_batch b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void qp_batch_destroy(kq_batch b) {
  if (!b) return;
  for (kq_problem *h : b->qps) qp_destroy(h);
  batch_pcg_free(b->B);
  delete b;
}

kq_status qp_create_batch(kq_batch *out, int nqp, const kq_qp_desc *d, void *stream) {
  if (!out || nqp <= 0 || !d) return bfail(nullptr, KQ_ERR_ARG, "qp_create_batch: bad arguments");
  *out = nullptr;
  kq_batch b = new kq_batch_s();
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < nqp; ++i) {
    if (d[i].H.kind != KQ_H_DENSE) {
      qp_batch_destroy(b);
      return bfail(nullptr, KQ_ERR_ARG, "qp_create_batch: every QP needs a dense H");
    }
    kq_handle h = nullptr;
    const kq_status st = qp_create(&h, d[i].n, &d[i].H, d[i].p, d[i].A.kind == KQ_A_NONE ? nullptr : &d[i].A,
                                   d[i].lA, d[i].uA, d[i].me, d[i].C, d[i].b, d[i].lx, d[i].ux, stream);
    if (st != KQ_OK) {
      const std::string msg = "qp_create_batch: QP " + std::to_string(i) + ": " + kq_global_error();
      qp_batch_destroy(b);
      return bfail(nullptr, st, msg);
    }
    b->qps.push_back(h);
    b->max_n = std::max<int>(b->max_n, (int)d[i].n);
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  std::string e;
  const kq_status st = batch_pcg_setup(b->B, nqp, sms, b->max_n, e);
  if (st != KQ_OK) {
    qp_batch_destroy(b);
    return bfail(nullptr, st, "qp_create_batch: " + e);
  }
  *out = b;
  return KQ_OK;
}

kq_status qp_batch_solution(kq_batch b, int i, double *x, double *lam_lA, double *lam_uA,
                            double *lam_lx, double *lam_ux, double *lam_e) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  if (i < 0 || i >= (int)b->qps.size()) return bfail(b, KQ_ERR_ARG, "QP index out of range");
  kq_problem *h = b->qps[i];
  if (outputs_enqueue(h, x, lam_lA, lam_uA, lam_lx, lam_ux, lam_e) != KQ_OK)
    return bfail(b, KQ_ERR_CUDA, h->err);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch solution copy");
  return KQ_OK;
}

kq_status qp_batch_time_product(kq_batch b, int i, int team, int precision, int colpass_min_n,
                                int reps, double *ms) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  if (i < 0 || i >= (int)b->qps.size() || team < 1 || reps < 1 || !ms)
    return bfail(b, KQ_ERR_ARG, "qp_batch_time_product: bad arguments");
  kq_problem *h = b->qps[i];
  if (!h->kkt_valid && kkt_assemble(h) != KQ_OK) return bfail(b, KQ_ERR_CUDA, h->err);
  BatchTune saved = b->B.tune;
  b->B.tune.force_team = team;
  if (colpass_min_n > 0) b->B.tune.colpass_min_n = colpass_min_n;
  std::vector<kq_problem *> hs(b->qps.begin(), b->qps.end());
  std::vector<int> idx{i};
  std::vector<const double *> in{h->z};     // NKP entries, finite (zero or a direction)
  std::vector<double *> out{h->zref};
  std::vector<double> tol{0.0};
  std::vector<int> mx{0}, its, errs;
  std::vector<double> rr, bb;
  double total = 0.0;
  kq_status rc = KQ_OK;
  std::string e;
  for (int r = 0; r <= reps && rc == KQ_OK; ++r) {
    float t = 0.f;
    rc = batch_pcg_launch(b->B, hs, idx, in, out, tol, mx, 1,
                          precision == KQ_PREC_MIXED ? KQ_PREC_MIXED : KQ_PREC_F64, b->stream,
                          its, errs, rr, bb, &t, e);
    if (r > 0) total += t;   // the first launch warms up
  }
  b->B.tune = saved;
  if (rc != KQ_OK) return bfail(b, rc, e);
  *ms = total / reps;
  return KQ_OK;
}

kq_status qp_batch_set_tuning(kq_batch b, int nbuckets, const int *team_cap,
                              const double *t_prod_us, int colpass_min_n) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  if (nbuckets < 0 || nbuckets > 40 || (nbuckets > 0 && (!team_cap || !t_prod_us)))
    return bfail(b, KQ_ERR_ARG, "qp_batch_set_tuning: bad table");
  BatchTune t;
  for (int k = 0; k < nbuckets; ++k) {
    if (team_cap[k] < 1 || !(t_prod_us[k] > 0.0)) return bfail(b, KQ_ERR_ARG, "qp_batch_set_tuning: bad entry");
    t.team_cap.push_back(team_cap[k]);
    t.t_prod_us.push_back(t_prod_us[k]);
  }
  t.colpass_min_n = colpass_min_n > 0 ? colpass_min_n : 512;
  b->B.tune = t;
  return KQ_OK;
}

kq_status qp_batch_qp_stats(kq_batch b, int i, int *ipm_iters, long long *pcg_iters) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  if (i < 0 || i >= (int)b->qps.size()) return bfail(b, KQ_ERR_ARG, "QP index out of range");
  if (ipm_iters) *ipm_iters = b->qps[i]->batch_ipm_iters;
  if (pcg_iters) *pcg_iters = b->qps[i]->batch_pcg_iters;
  return KQ_OK;
}

kq_status qp_batch_info(kq_batch b, int *nqp, int64_t *n) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  if (nqp) *nqp = (int)b->qps.size();
  if (n)
    for (size_t i = 0; i < b->qps.size(); ++i) n[i] = b->qps[i]->n;
  return KQ_OK;
}

kq_status ipm_solve_batch(kq_batch b, const kq_ipm_opts *opts, double *const *x, int *status,
                          kq_batch_stats *stats) {
  if (!b) return bfail(nullptr, KQ_ERR_ARG, "null batch");
  auto t0 = std::chrono::steady_clock::now();
  kq_ipm_opts o;
  kq_default_ipm_opts(&o);
  if (opts) o = *opts;
  if (o.graph) return ipm_solve_batch_graph(b, o, x, status, stats);
  kq_pcg_opts po;
  po.tol = o.pcg_tol; po.maxit = o.pcg_maxit; po.precision = o.precision;
  po.refine_steps = o.refine_steps; po.inner_tol = o.inner_tol;
  auto &hs = b->qps;
  const int nq = (int)hs.size();
  cudaStream_t s = b->stream;
  kq_batch_stats st{};
  std::vector<double> mu(nq, o.mu0);
  std::vector<int> kexp(nq, 0), done(nq, 0), stat(nq, KQ_ERR_IPM_MAXIT), iters(nq, 0);
  for (kq_problem *h : hs) {
    h->timeout_s = o.timeout_s > 0 ? o.timeout_s : 2.0;
    h->solved = false;
    h->state_set = false;
    h->mu = o.mu0;
    h->batch_pcg_iters = 0;
    if (init_state(h) != KQ_OK || assemble_enqueue(h) != KQ_OK) return bfail(b, KQ_ERR_CUDA, h->err);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch init");
  double n2;
  for (kq_problem *h : hs) assemble_finish(h, &n2, nullptr);
  double kernel_ms = 0.0;
  std::vector<double> last_iters(nq, 1.0);   // PCG iterations of each QP's previous solve
  int it;
  for (it = 1; it <= o.ipm_maxit; ++it) {
    std::vector<int> act;
    for (int i = 0; i < nq; ++i) if (!done[i]) act.push_back(i);
    if (act.empty()) break;
    st.max_active = std::max(st.max_active, (int)act.size());
    std::vector<long long> pits;
    std::vector<int> hit;
    const double kms0 = kernel_ms;
    const kq_status rc = batch_pcg(b, act, po, pits, hit, &kernel_ms, last_iters);
    if (rc != KQ_OK) return rc;
    long long its_sum = 0;
    for (size_t j = 0; j < act.size(); ++j) {
      hs[act[j]]->batch_pcg_iters += pits[j];
      st.pcg_iters += pits[j];
      st.pcg_maxit_hits += hit[j];
      last_iters[act[j]] = (double)std::max<long long>(1, pits[j]);
      its_sum += pits[j];
    }
    if (o.verbose) {
      fprintf(stderr, "batch ipm %3d active %4zu pcg iters %8lld pcg %.1f ms\n", it, act.size(),
              its_sum, kernel_ms - kms0);
      fflush(stderr);
    }
    for (int i : act)
      if (recover_enqueue(hs[i]) != KQ_OK) return bfail(b, KQ_ERR_CUDA, hs[i]->err);
    if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch recover");
    for (int i : act) {
      double ax, al;
      recover_finish(hs[i], o.gamma, &ax, &al);
      if (!(ax == ax) || !(al == al)) return bfail(b, KQ_ERR_NUMERIC, "NaN step length");
      if (update_enqueue(hs[i], ax, al) != KQ_OK || assemble_enqueue(hs[i]) != KQ_OK)
        return bfail(b, KQ_ERR_CUDA, hs[i]->err);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch update");
    std::vector<int> reasm;
    for (int i : act) {
      assemble_finish(hs[i], &n2, nullptr);
      const double rn = std::sqrt(n2);
      if (!(rn == rn)) return bfail(b, KQ_ERR_NUMERIC, "residual NaN in QP " + std::to_string(i));
      iters[i] = it;
      if (rn < mu[i]) {
        if (mu[i] < o.mu_tol) {
          done[i] = 1;
          stat[i] = KQ_OK;
          hs[i]->solved = true;
          continue;
        }
        ++kexp[i];
        mu[i] = o.mu0 * std::pow(10.0, -(double)kexp[i]);
        hs[i]->mu = mu[i];
        reasm.push_back(i);
      }
    }
    for (int i : reasm)
      if (assemble_enqueue(hs[i]) != KQ_OK) return bfail(b, KQ_ERR_CUDA, hs[i]->err);
    if (!reasm.empty()) {
      if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch reassemble");
      for (int i : reasm) assemble_finish(hs[i], &n2, nullptr);
    }
  }
  for (int i = 0; i < nq; ++i) {
    if (x && x[i]) outputs_enqueue(hs[i], x[i], nullptr, nullptr, nullptr, nullptr, nullptr);
    if (status) status[i] = stat[i];
    hs[i]->batch_ipm_iters = iters[i];
    st.ipm_iters_max = std::max(st.ipm_iters_max, iters[i]);
    st.ipm_iters_total += iters[i];
    if (stat[i] == KQ_OK) st.converged++;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return bfail(b, KQ_ERR_CUDA, "batch outputs");
  st.pcg_kernel_ms = kernel_ms;
  st.pcg_launches = b->B.launches;
  st.time_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return st.converged == nq ? KQ_OK : KQ_ERR_IPM_MAXIT;
}

}  // extern "C"
