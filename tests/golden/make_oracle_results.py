"""Write tests/golden/oracle_results.json: FP64 oracle solves of the workloads
that are too slow to re-solve inside the GPU tests.

Calls only the oracle (oracle/) on the seeded generators (qpgen/); nothing here
touches the CUDA path.  Stored per problem: the oracle's status, IPM
iterations, final mu, objective, acceptance metrics (original units), and x
at a seeded sample of indices (to report the distance of another solution).

    python tests/golden/make_oracle_results.py [--only NAME ...]

Workloads:
  c1               dose-shaped QP, P 200k x 20k, 2e7 nnz, 10k dose-limit rows
                   (banded-Schur direct Newton solves; about 4 min on 8 cores)
  c3_subset        QPs 5, 9, 10, 12 and 26 of the 512-QP batch (n = 2850,
                   3126, 1904, 2264, 4048: the four largest of the first 16 and
                   the largest of the batch), bf16-rounded H, f32-rounded A
  c2_mu1e-6        linear SVM dual at the paper's mu_tol
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import qpgen  # noqa: E402
from oracle.metrics import full_multipliers  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_results.json")
C3_SUBSET = [5, 9, 10, 12, 26]


def record(qp, res, t):
    lA, uA, lx, ux, le = full_multipliers(res.scaled, res.lam, qp)
    met = oracle.kkt_metrics(qp, res.x, lA, uA, lx, ux, le)
    idx = np.sort(np.random.default_rng(123).permutation(qp.n)[:min(qp.n, 200)])
    return {"status": res.status, "iters": int(res.iters), "mu": float(res.mu),
            "objective": float(met["objective"]), "primal_rel": met["primal_rel"],
            "dual_rel": met["dual_rel"], "compl_rel": met["compl_rel"],
            "x_inf": float(np.max(np.abs(res.x))), "x_idx": idx.tolist(),
            "x_at_idx": [float(v) for v in res.x[idx]], "solve_s": t}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args()
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    todo = args.only or ["c1", "c3_subset", "c2_mu1e-6"]
    if "c1" in todo:
        qp = qpgen.config1()
        t0 = time.perf_counter()
        res = oracle.ipm_solve(qp)
        data["c1"] = record(qp, res, time.perf_counter() - t0)
        print("c1", data["c1"]["objective"], data["c1"]["iters"], flush=True)
    if "c3_subset" in todo:
        sizes = qpgen.batch_sizes(512, 64, 4096)
        out = {}
        for k in C3_SUBSET:
            qp = qpgen.batch_qp(k, sizes[k])
            t0 = time.perf_counter()
            res = oracle.ipm_solve(qp)
            out[str(k)] = dict(record(qp, res, time.perf_counter() - t0), n=sizes[k])
            print("c3", k, sizes[k], out[str(k)]["objective"], out[str(k)]["iters"], flush=True)
        data["c3_subset"] = out
    if "c2_mu1e-6" in todo:
        qp = qpgen.config2()
        t0 = time.perf_counter()
        res = oracle.ipm_solve(qp)
        data["c2_mu1e-6"] = record(qp, res, time.perf_counter() - t0)
    data["_about"] = ("FP64 oracle (Algorithm 1 with direct Newton solves) on the seeded "
                      "workloads; written by tests/golden/make_oracle_results.py")
    json.dump(data, open(OUT, "w"), indent=1)


if __name__ == "__main__":
    main()
