"""Benchmark: time-to-1e-6 of the Krylov IPM on the dose-shaped QP
(P 200k x 20k CSR, 2e7 nnz, 10k two-sided dose-limit rows, x >= 0).

One step = one full ipm_solve (Algorithm 1: residuals, right-hand side,
Jacobi diagonal, persistent PCG solves, step recovery, ratio test, update,
mu rule) from the initial point to mu < 1e-6, inputs resident in HBM.
``e2e`` repeats the step through the C ABI with host buffers: qp_create from
host arrays (upload inside the timed region), ipm_solve writing the solution
to host arrays, qp_destroy.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|f64]
        python bench.py --impl reference      (oracle arm, host cores)
        python bench.py --mode pcg --pcg-iters 200   (one PCG launch, for ncu)
Under torchrun (N > 1) every rank solves its own replica of the problem (the
method does not shard; replicas only) and value is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALGO_BYTES_NOTE = ("per K*v product: nnz*(4 B value + 4 B column) + (rows+1)*4 B row pointer "
                   "+ rows*4 B weight")
WORKLOAD = "dose_qp_200k_x_20k_nnz2e7"
METRIC = "time-to-1e-6 IPM solve (dose-shaped QP, PCG on the doubly augmented KKT system)"
# the benchmark workload (both arms)
CONFIG = {"workload": WORKLOAD, "rows": 200_000, "n": 20_000, "nnz": 20_000_000,
          "dose_limit_rows": 10_000, "l2": "inputs larger than L2 (P is 160 MB > 129 MB)"}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pcg_csr_dose200k_traffic.json")


def algo_bytes(qp) -> float:
    rows, nnz = qp.P.shape[0], qp.P.nnz
    return nnz * 8.0 + (rows + 1) * 4.0 + rows * 4.0


def stored_bytes(qp) -> float:
    """Bytes the register-streamed FP32 product reads per K*v: per row, its
    nonzeros padded to a multiple of 4 (4 B value + 2 B column each) and a
    16-byte row descriptor."""
    import numpy as np
    ln = np.diff(qp.P.indptr)
    return float(np.sum(4 * ((ln + 3) // 4)) * 6.0 + len(ln) * 16.0)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("pcg.cu", "common.cuh", "kq_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2308_00637_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def read_peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks during the timed region (started before, stopped after)."""

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            rows = []
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = max(mx, float(r[1]))
                for nm, v in zip(names, r[4:8]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx or None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle (reference arm, cpu_baseline)
# The oracle runs Algorithm 1 with a direct Newton solve per IPM iteration
# (banded-Schur Cholesky for this workload).  A complete solve takes minutes on
# a host, so a step of the CPU legs is ONE IPM iteration of the oracle's own
# trajectory from the initial point (a finished trajectory restarts); the
# per-solve value is the mean measured seconds per iteration times the
# oracle's iteration count for this workload (its stored full solve).
ORACLE_STEP_CODE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import qpgen, oracle
qp = qpgen.config1()
state = {{"gen": oracle.ipm_iterate(qp)}}
def one():
    t0 = time.perf_counter()
    st = next(state["gen"])
    if "result" in st:
        state["gen"] = oracle.ipm_iterate(qp)
    return time.perf_counter() - t0, st["it"]
warm = [one()[0] for _ in range({nwarm})]
times, its = [], []
for _ in range({nsteps}):
    t, it = one()
    times.append(t)
    its.append(it)
print(json.dumps({{"times": times, "iters": its, "warm_times": warm}}))
"""


def oracle_solve_estimate(r, nit):
    """Seconds of one full oracle solve from timed steps: the step that ran
    the set-up (scaling, initial point) with the first iteration, plus
    (nit - 1) x the mean of the steps without it."""
    if r.get("warm_times"):
        first, rest = r["warm_times"][0], r["times"]
    else:
        first, rest = r["times"][0], r["times"][1:]
    per = sum(rest) / len(rest) if rest else first
    return first + (nit - 1) * per, first, per
ORACLE_RESULTS = os.path.join(ROOT, "tests", "golden", "oracle_results.json")


def host_cpu():
    """CPU model and logical core count of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
        if model is None:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except Exception:
        pass
    return model or "unknown", os.cpu_count() or 1


def oracle_iters_per_solve():
    """IPM iterations of the oracle's own full solve of this workload."""
    return int(json.load(open(ORACLE_RESULTS))["c1"]["iters"])


def oracle_steps(nwarm: int, nsteps: int, threads: int):
    """Time nsteps oracle IPM iterations after nwarm untimed ones, in a child
    process whose BLAS uses `threads` threads."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-c", ORACLE_STEP_CODE.format(root=ROOT, nwarm=nwarm,
                                                                       nsteps=nsteps)],
                         capture_output=True, text=True, env=env, timeout=3600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


# The CPU restatement of the paper's own design (FP64 C++/OpenMP, matrix-free
# Eq. (9), Jacobi-PCG): a fixed number of PCG iterations on the first Newton
# system of the benchmark workload (the oracle supplies the system).
RESTATEMENT_CODE = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import qpgen, cpu_restatement as cr
from oracle import ipm as I
qp = qpgen.config1()
S = I.scale(qp)
st = I.initial_point(S)
r = I.residuals(S, st, 1.0)
dg, D, r1, r2 = I.reduced_system(S, st, r, 1.0)
rhs = I.doubly_augmented_rhs(S, D, r1, r2)
diag = I.jacobi_diagonal(S, dg, D)
sysc = cr.System(S.P, S.w2, S.A, S.L, S.U, dg, D)
sysc.pcg(diag, rhs, tol=0.0, maxit=3)
t0 = time.perf_counter()
_, it, rel = sysc.pcg(diag, rhs, tol=0.0, maxit={iters})
dt = time.perf_counter() - t0
print(json.dumps({{"iters": it, "seconds": dt, "bytes_per_apply": sysc.bytes_per_apply(),
                  "threads": cr.threads()}}))
"""


def restatement_pcg(iters: int, threads: int):
    """PCG iterations per second of the CPU restatement on the host cores."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads), OPENBLAS_NUM_THREADS=str(threads))
    out = subprocess.run([sys.executable, "-c", RESTATEMENT_CODE.format(root=ROOT, iters=iters)],
                         capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    r = json.loads(out.stdout.strip().splitlines()[-1])
    ips = r["iters"] / r["seconds"]
    return {"pcg_iters_per_s": ips, "gbs": r["bytes_per_apply"] * ips / 1e9,
            "threads": r["threads"], "iters": r["iters"], "seconds": r["seconds"],
            "sample": (f"{r['iters']} FP64 Jacobi-PCG iterations (fixed count) of the CPU "
                       f"restatement (C++/OpenMP, matrix-free Eq. (9)) on the first Newton "
                       f"system of the full 200k x 20k dose QP; gbs = bytes one apply reads "
                       f"({r['bytes_per_apply'] / 1e6:.0f} MB: P and A twice) x iterations/s")}


def cpu_baseline_line(nsteps=3):
    model, cores = host_cpu()
    nit = oracle_iters_per_solve()
    r = oracle_steps(0, nsteps, cores)
    total, first, per = oracle_solve_estimate(r, nit)
    try:
        rest = restatement_pcg(100, cores)
        one = restatement_pcg(20, 1)
        rest["one_thread"] = {k: one[k] for k in ("pcg_iters_per_s", "gbs", "iters", "seconds")}
    except Exception as e:   # reported, not fatal
        rest = {"error": str(e)[-300:]}
    return {"value": total, "unit": "s", "cores": cores, "kind": "oracle",
            "cpu": model,
            "sample": (f"IPM iterations {r['iters'][0]}-{r['iters'][-1]} of the FP64 oracle's own "
                       f"trajectory on the full 200k x 20k dose QP (direct banded-Schur Newton "
                       f"solves, BLAS on {cores} threads): the first with the set-up "
                       f"{first:.2f} s, the others {per:.2f} s each; value = first + "
                       f"{nit - 1} x {per:.2f} s for the {nit} IPM iterations of the oracle's "
                       f"full solve of this workload"),
            "s_per_ipm_iteration": per, "s_first_iteration_with_setup": first,
            "ipm_iterations_per_solve": nit,
            "pcg_restatement": rest}


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    model, cores = host_cpu()
    nit = oracle_iters_per_solve()
    r = oracle_steps(args.warmup, args.steps, cores)
    v, first, per = oracle_solve_estimate(r, nit)
    step_mean = sum(r["times"]) / len(r["times"])
    sample = (f"{args.steps} consecutive IPM iterations ({r['iters'][0]}-{r['iters'][-1]}) of the "
              f"FP64 oracle's own trajectory on the full 200k x 20k dose QP after {args.warmup} "
              f"untimed ones; each a direct banded-Schur Newton solve with BLAS on {cores} "
              f"threads ({model}); value = the step with the set-up and the first iteration "
              f"({first:.2f} s) + {nit - 1} x {per:.2f} s for the {nit} IPM iterations of the "
              f"oracle's full solve of this workload")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_mean * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator, seed 1)",
            "config": dict(CONFIG, precision="f64", parallelism="host cores"),
            "step": "one IPM iteration of the oracle (value scaled to one solve)",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "cpu": model, "sample": sample,
                             "value": v, "unit": "s"},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- GPU arm
def dose_kkt(qp, x, lam_lA, lam_uA, lam_lx, lam_ux):
    """The acceptance measure of the tests for the dose QP (H = 2 P' W P,
    limit rows = rows of P, bounds on x; no equality rows), restated here so
    that the GPU arm does not call the oracle: primal_rel = largest row-
    normalised limit or bound violation / (1 + |x|_inf); dual_rel = |r_H|_inf
    over the largest gradient term, r_H = H x + p - A'(lam_lA - lam_uA) -
    (lam_lx - lam_ux); kkt_rel = max of the two; and the objective."""
    import numpy as np
    P = qp.P.astype(np.float64)
    A = P[qp.a_rows]
    Px = P @ x
    Hx = 2.0 * (P.T @ (qp.w * Px))
    Ax = A @ x
    rn = np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    rn = np.where(rn > 0, rn, 1.0)
    lA, uA = np.asarray(qp.lA, float), np.asarray(qp.uA, float)
    with np.errstate(invalid="ignore"):
        v = np.maximum(np.where(np.isfinite(lA), lA - Ax, 0.0), np.where(np.isfinite(uA), Ax - uA, 0.0))
        lx, ux = np.asarray(qp.lx, float), np.asarray(qp.ux, float)
        vb = np.maximum(np.where(np.isfinite(lx), lx - x, 0.0), np.where(np.isfinite(ux), x - ux, 0.0))
    primal = max(float(np.max(np.maximum(v, 0.0) / rn)), float(np.max(np.maximum(vb, 0.0)))) / \
        (1.0 + float(np.max(np.abs(x))))
    ATl = np.asarray(A.T @ (lam_lA - lam_uA)).ravel()
    lxx = lam_lx - lam_ux
    rH = Hx + qp.p - ATl - lxx
    scale = 1.0 + max(float(np.max(np.abs(Hx))), float(np.max(np.abs(qp.p))),
                      float(np.max(np.abs(ATl))), float(np.max(np.abs(lxx))))
    dual = float(np.max(np.abs(rH))) / scale
    return {"primal_rel": primal, "dual_rel": dual, "kkt_rel": max(primal, dual),
            "objective": float(0.5 * x @ Hx + qp.p @ x)}


def max_over_ranks(x: float, dist, device: str) -> float:
    """The slowest rank's value (replicas: the job ends with the slowest one).
    `dist` is torch.distributed or None (one process)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def batch_bytes_per_product(q) -> float:
    """Algorithmic bytes of one K*v product of a batched dense QP: H (bf16
    bits or FP64) and A (FP32 or FP64), each read once."""
    hb = 2.0 if (q.meta or {}).get("H_bf16_bits") is not None else 8.0
    ab = 4.0 if (q.meta or {}).get("a_f32", False) else 8.0
    return hb * q.n * q.n + ab * q.m * q.n


def batch_line(kq, qps, prec, graph, peak, peak_src, head, ipm_maxit=200):
    """Solve a batch once and describe it: time, convergence, and the
    effective bandwidth of its products (algorithmic bytes x each QP's PCG
    iterations / device time of the solve's launches -- the whole replayed
    iteration in the graph form, so a lower bound there).  With ipm_maxit
    below Algorithm 1's N the line states the cost of that many lock-step
    IPM iterations."""
    import numpy as np
    b = kq.qp_create_batch(qps)
    xs = [np.zeros(q.n) for q in qps]
    rc, status, st = kq.ipm_solve_batch(b, kq.default_ipm_opts(precision=prec, graph=graph,
                                                               ipm_maxit=ipm_maxit), xs)
    per = [kq.qp_batch_qp_stats(b, i) for i in range(len(qps))]
    kq.qp_batch_destroy(b)
    byts = sum(batch_bytes_per_product(q) * it for q, (_, it) in zip(qps, per))
    gbs = byts / (st.pcg_kernel_ms * 1e-3) / 1e9 if st.pcg_kernel_ms > 0 else None
    return dict(head, **{"time_to_1e-6_s" if ipm_maxit >= 200 else "time_s": st.time_s,
                         "ipm_maxit": ipm_maxit, "converged": st.converged,
                         "status": int(rc), "ipm_iters_max": st.ipm_iters_max,
                         "pcg_iters": int(st.pcg_iters), "pcg_maxit_hits": st.pcg_maxit_hits,
                         "device_ms": st.pcg_kernel_ms, "graph_captures": st.graph_captures,
                         "graph_replays": st.graph_replays,
                         "sum_n2": int(sum(q.n * q.n for q in qps)),
                         "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                      "frac": gbs / peak if gbs else None, "peak_source": peak_src,
                                      "bytes": byts,
                                      "note": "bf16 H + f32 A per product x each QP's PCG iterations"
                                              " / device time of the solve"}})


def other_configs(kq, qpgen):
    """Time-to-1e-6 of the other configurations in both forms (one warm-up
    solve, one timed), for the record next to the benchmark line: c0 (dense
    n = 200), c2 (linear SVM dual), c4 (dose QP at 1/4 size), the RBF-kernel
    SVM dual of a1a's shape, and the first 32 QPs of the 512-QP batch with
    n <= 1024 (graph form)."""
    import numpy as np
    out = {}
    for name, mk in (("c0_dense_n200", qpgen.config0), ("c2_svm_50k", qpgen.config2),
                     ("c4_dose_50k_x_5k", qpgen.config4),
                     # Gaussian-kernel SVM dual of a1a's shape (Table 1: 1605
                     # variables, one equality; H formed on the device)
                     ("rbf_svm_1605x123", lambda: qpgen.rbf_svm_qp(1605, 123, seed=51))):
        qp = mk()
        d = {}
        for prec, form in ((kq.KQ_PREC_F64, "f64"), (kq.KQ_PREC_MIXED, "mixed")):
            h = kq.create_from(qp, device_tensors=True)
            x = np.zeros(qp.n)
            kq.ipm_solve(h, kq.default_ipm_opts(precision=prec), x=x)
            _, st = kq.ipm_solve(h, kq.default_ipm_opts(precision=prec), x=x)
            d[form] = {"time_s": st.time_s, "ipm_iters": st.ipm_iters, "pcg_iters": int(st.pcg_iters),
                       "switched_to_f64": st.switched_to_f64}
            kq.qp_destroy(h)
        out[name] = d
    sizes = qpgen.batch_sizes(512, 64, 4096)
    ids = [k for k, n in enumerate(sizes) if n <= 1024][:32]
    qps = [qpgen.batch_qp(k, sizes[k], light=True) for k in ids]
    peak, peak_src = read_peaks()
    d = {}
    for prec, form in ((kq.KQ_PREC_F64, "f64"), (kq.KQ_PREC_MIXED, "mixed")):
        ln = batch_line(kq, qps, prec, 1, peak, peak_src, {})
        d[form] = {k: ln[k] for k in ("time_to_1e-6_s", "converged", "pcg_iters", "ipm_iters_max")}
        d[form]["frac"] = ln["roofline"]["frac"]
    out["c3_first32_n_le_1024"] = d
    return out


def run_other(args):
    """Time-to-1e-6 of the other configurations, plain FP64 against mixed
    (and batched), on one GPU.  One JSON line per form; the median of
    `--steps` solves after `--warmup` (wall time of ipm_solve, which ends with
    the status read back on the host)."""
    import numpy as np
    import torch
    import qpgen
    import paper_2308_00637_gb300 as kq
    from paper_2308_00637_gb300 import build as kqbuild
    torch.cuda.set_device(0)
    kqbuild.build()
    kq.load()
    steps, warm = max(1, args.steps), max(0, args.warmup)

    def emit(d):
        print(json.dumps(d), flush=True)

    if args.workload in ("c0", "c2", "c4"):
        qp = {"c0": qpgen.config0, "c2": qpgen.config2, "c4": qpgen.config4}[args.workload]()
        for prec, name in ((kq.KQ_PREC_F64, "f64"), (kq.KQ_PREC_MIXED, "mixed")):
            h = kq.create_from(qp, device_tensors=True)
            opts = kq.default_ipm_opts(precision=prec)
            x = np.zeros(qp.n)
            ts, st = [], None
            for k in range(warm + steps):
                _, st = kq.ipm_solve(h, opts, x=x)
                if k >= warm:
                    ts.append(st.time_s)
            d = {"workload": args.workload, "form": name, "time_to_1e-6_s": float(np.median(ts)),
                 "ipm_iters": st.ipm_iters, "pcg_iters": int(st.pcg_iters),
                 "pcg_iters_f64": int(st.pcg_iters_f64), "pcg_kernel_ms": st.pcg_kernel_ms,
                 "objective": qp.objective(x), "n": qp.n}
            if args.workload == "c4":
                gbar = qpgen.config4_directions(qp, 1)[0]
                po = kq.default_pcg_opts(tol=1e-7, precision=prec)
                tb = []
                for k in range(warm + steps):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    kq.qp_backward(h, gbar, grad_p=np.zeros(qp.n), grad_lA=np.zeros(qp.m),
                                   grad_uA=np.zeros(qp.m), opts=po)
                    torch.cuda.synchronize()
                    if k >= warm:
                        tb.append(time.perf_counter() - t0)
                d["backward_s"] = float(np.median(tb))
                d["backward_over_forward"] = d["backward_s"] / d["time_to_1e-6_s"]
            emit(d)
            kq.qp_destroy(h)
        return 0

    nqp = args.nqp if args.nqp > 0 else (128 if args.workload == "batch128" else 512)
    hi = 1024 if args.workload == "batch128" else 4096
    sizes = qpgen.batch_sizes(nqp, 64, hi, size_seed=5 if args.workload == "batch128" else 0)
    qps = [qpgen.batch_qp(k, n, light=True) for k, n in enumerate(sizes)]
    peak, peak_src = read_peaks()
    forms = {"mixed-graph": (kq.KQ_PREC_MIXED, 1, "batched mixed, graph"),
             "f64-graph": (kq.KQ_PREC_F64, 1, "batched f64, graph"),
             "mixed-host": (kq.KQ_PREC_MIXED, 0, "batched mixed, host-driven"),
             "f64-host": (kq.KQ_PREC_F64, 0, "batched f64, host-driven")}
    pick = list(forms) if args.batch_form == "all" else [args.batch_form]
    for key in pick:
        prec, graph, name = forms[key]
        emit(batch_line(kq, qps, prec, graph, peak, peak_src,
                        {"workload": args.workload, "form": name, "nqp": nqp,
                         "sum_4n2_bytes": sum(batch_bytes_per_product(q) for q in qps)},
                        ipm_maxit=args.ipm_maxit))
    if args.sequential:
        tot, its = 0.0, 0
        for q in qps:
            _, st, _ = kq.solve(q, kq.default_ipm_opts(precision=kq.KQ_PREC_F64))
            tot += st.time_s
            its += int(st.pcg_iters)
        emit({"workload": args.workload, "form": "one at a time f64", "time_to_1e-6_s": tot,
              "pcg_iters": its, "nqp": nqp})
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"])
    ap.add_argument("--mode", default="solve", choices=["solve", "pcg"])
    ap.add_argument("--pcg-iters", type=int, default=200)
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the other configurations' record on the benchmark line")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--warm-start", type=int, default=0,
                    help="1: each Newton solve's PCG starts from the previous direction "
                         "(opts.warm_start); 0: from zero, as the paper")
    ap.add_argument("--workload", default="c1",
                    choices=["c1", "c0", "c2", "c4", "batch128", "batch512"],
                    help="c1 (default) is the benchmark; the others print one timing line "
                         "per form (plain FP64 / mixed / batched) on the other configurations")
    ap.add_argument("--nqp", type=int, default=0,
                    help="batch workloads: number of QPs (default 128 / 512)")
    ap.add_argument("--batch-form", default="all",
                    choices=["all", "mixed-graph", "f64-graph", "mixed-host", "f64-host"],
                    help="batch workloads: which form(s) to run")
    ap.add_argument("--ipm-maxit", type=int, default=200,
                    help="batch workloads: stop after this many lock-step IPM iterations "
                         "(the line then gives their cost, not a time-to-1e-6)")
    ap.add_argument("--sequential", action="store_true",
                    help="batch workloads: also time plain FP64 one QP at a time")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c1":
        return run_other(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import qpgen
    import paper_2308_00637_gb300 as kq
    from paper_2308_00637_gb300 import build as kqbuild
    if rank == 0:
        kqbuild.build()
    if dist is not None:
        dist.barrier()
    kq.load()

    qp = qpgen.config1()
    prec = kq.KQ_PREC_MIXED if args.precision == "mixed" else kq.KQ_PREC_F64
    opts = kq.default_ipm_opts(precision=prec, warm_start=int(args.warm_start))
    h = kq.create_from(qp, device_tensors=True)
    n, m = h.n, h.m
    dev = {k: torch.zeros(s, dtype=torch.float64, device="cuda")
           for k, s in (("x", n), ("lam_lA", m), ("lam_uA", m), ("lam_lx", n), ("lam_ux", n))}

    if args.mode == "pcg":
        # one Newton system at the initial point, fixed iteration count (profiling)
        rhs = torch.zeros(h.nkp, dtype=torch.float64, device="cuda")
        sol = torch.zeros_like(rhs)
        kq.qp_residuals(h, rhs=rhs)
        po = kq.default_pcg_opts(tol=1e-30, maxit=args.pcg_iters, precision=prec,
                                 refine_steps=1 if prec else 0, inner_tol=1e-30)
        res = []
        for _ in range(max(1, args.steps)):
            rc, st = kq.kkt_pcg_solve(h, rhs, sol, po)
            res.append(st.as_dict())
        torch.cuda.synchronize()
        last = res[-1]
        us = 1e3 * last["kernel_ms"] / max(1, last["iters"] + last["passes"])
        print(json.dumps({"mode": "pcg", "iters": last["iters"], "kernel_ms": last["kernel_ms"],
                          "us_per_product": us, "kv_gbs": algo_bytes(qp) / (us * 1e-6) / 1e9,
                          "env": {k: os.environ.get(k) for k in ("KQ_CHUNK", "KQ_STAGES",
                                                                 "KQ_COPY_PIECE")}}))
        return 0

    def solve():
        return kq.ipm_solve(h, opts, **dev, allow=(kq.KQ_OK,))[1]

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    stats = []
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(solve())
        e1.record(stream)
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms_total = e0.elapsed_time(e1)
    t_step = ms_total / 1e3 / args.steps
    t_step = max_over_ranks(t_step, dist, "cuda")
    s0 = stats[-1]
    prod = sum(s.pcg_products for s in stats)
    kms = sum(s.pcg_kernel_ms for s in stats)
    launches = sum(s.pcg_launches for s in stats)
    # the dominant kernel: the FP32 passes in mixed precision (register-streamed
    # CSR), the FP64 launches in plain FP64
    if prec == kq.KQ_PREC_MIXED:
        prod_dom = prod - sum(s.pcg_products_f64 for s in stats)
        kms_dom = kms - sum(s.pcg_kernel_ms_f64 for s in stats)
        launches_dom = launches - sum(s.pcg_launches_f64 for s in stats)
        kname = "pcg_kernel<OpCsrRows, float> (persistent FP32 PCG pass)"
    else:
        prod_dom, kms_dom, launches_dom = prod, kms, launches
        kname = "pcg_kernel<OpCsrStaged, double> (persistent FP64 PCG solve)"
    abytes = algo_bytes(qp)
    achieved = prod_dom * abytes / (kms_dom * 1e-3) / 1e9
    peak, peak_src = read_peaks()
    # DRAM bytes of the dominant kernel from the committed ncu capture (null once
    # the kernel source has changed since): per K*v product, and per launch of
    # this run (products per launch of the timed region)
    traffic = traffic_pp = None
    try:
        tr = json.load(open(TRAFFIC_FILE))
        if tr.get("kernel_hash") == kernel_source_hash() and tr.get("precision") == args.precision:
            traffic_pp = tr["dram_bytes_per_product"]
            traffic = traffic_pp * (prod_dom / max(1, launches_dom))
    except Exception:
        traffic = traffic_pp = None
    # accuracy of the result (original units)
    x = dev["x"].cpu().numpy()
    out = {k: v.cpu().numpy() for k, v in dev.items()}
    met = dose_kkt(qp, x, out["lam_lA"], out["lam_uA"], out["lam_lx"], out["lam_ux"])

    # ---- e2e: host buffers through the public API, copies inside the timed region
    host_in = [qp.P.data, qp.P.indices, qp.P.indptr, qp.w, qp.p, qp.a_rows, qp.lA, qp.uA,
               qp.lx, qp.ux]
    h2d = int(sum(np.asarray(a).nbytes for a in host_in))
    hout = {k: np.zeros(v.numel()) for k, v in dev.items()}
    d2h = int(sum(a.nbytes for a in hout.values()))
    kq.qp_destroy(h)
    torch.cuda.synchronize()
    e2e_times = []
    for _ in range(max(1, args.e2e_steps)):
        t0 = time.perf_counter()
        h2 = kq.create_from(qp)          # host numpy buffers -> device copies
        kq.ipm_solve(h2, opts, **hout)
        kq.qp_destroy(h2)
        torch.cuda.synchronize()
        e2e_times.append(time.perf_counter() - t0)
    e2e = sum(e2e_times) / len(e2e_times)
    e2e = max_over_ranks(e2e, dist, "cuda")

    # ---- plain-FP64 form on the same problem, for the comparison
    cmp = None
    if not args.no_compare and rank == 0:
        other = kq.KQ_PREC_F64 if prec == kq.KQ_PREC_MIXED else kq.KQ_PREC_MIXED
        h3 = kq.create_from(qp, device_tensors=True)
        torch.cuda.synchronize()
        ec0, ec1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ec0.record(stream)
        rc3, s3 = kq.ipm_solve(h3, kq.default_ipm_opts(precision=other), **dev,
                               allow=(kq.KQ_OK, kq.KQ_ERR_IPM_MAXIT))
        ec1.record(stream)
        torch.cuda.synchronize()
        cmp = {"precision": "f64" if other == kq.KQ_PREC_F64 else "mixed",
               "time_s": ec0.elapsed_time(ec1) / 1e3, "status": int(rc3),
               "ipm_iters": s3.ipm_iters, "pcg_iters": int(s3.pcg_iters),
               "pcg_kernel_ms": s3.pcg_kernel_ms,
               "kv_gbs": s3.pcg_products * abytes / (s3.pcg_kernel_ms * 1e-3) / 1e9}
        kq.qp_destroy(h3)

    others = None
    if rank == 0 and not args.no_others:
        try:
            others = other_configs(kq, qpgen)
        except Exception as e:   # reported, not fatal
            others = {"error": str(e)[-300:]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline_line()
        except Exception as e:   # reported, not fatal
            cpu = {"error": str(e)[-300:]}

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-matvec/f64" if prec == kq.KQ_PREC_MIXED else "f64",
            "data": "synthetic (seeded generator, seed 1)",
            "config": dict(CONFIG, rows=qp.P.shape[0], n=qp.n, nnz=qp.P.nnz, dose_limit_rows=m,
                           precision=args.precision, warm_start=bool(args.warm_start),
                           parallelism="replicas" if world > 1 else "single-gpu"),
            "ipm_iters": s0.ipm_iters, "pcg_iters": int(s0.pcg_iters),
            "pcg_products": int(s0.pcg_products), "pcg_iters_f64": int(s0.pcg_iters_f64),
            "pcg_maxit_hits": s0.pcg_maxit_hits,
            "pcg_iters_per_s": s0.pcg_iters / t_step,
            "kkt_rel": met["kkt_rel"], "objective": met["objective"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "peak_source": peak_src,
                         "kernel": kname, "products": int(prod_dom),
                         "launches": int(launches_dom), "traffic_per_product": traffic_pp,
                         "kernel_ms": kms_dom,
                         "algorithmic_bytes_per_product": abytes,
                         "algorithmic_bytes_per_launch": abytes * prod_dom / max(1, launches_dom),
                         "note": ALGO_BYTES_NOTE,
                         "stored_bytes_per_product": stored_bytes(qp) if prec == kq.KQ_PREC_MIXED
                         else abytes},
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(sum(s.kernel_launches for s in stats)),
            "clocks": clk.summary(),
            "compare": cmp,
            "other_configs": others,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
