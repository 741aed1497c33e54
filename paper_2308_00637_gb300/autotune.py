"""Autotuner of the batched dense K*v products (per size bucket k = floor(log2 n)).

For one representative QP per bucket it times one product on teams of 1, 2,
4, ... CTAs (``qp_batch_time_product``) and, for n >= 128, with and without
the column-blocked A' pass.  Per bucket it keeps

* ``team_cap``  -- the smallest team within 10 % of the fastest: more CTAs
  than that are better spent on other QPs of the batch;
* ``t_prod_us`` -- one product on one CTA: the scheduler's cost of the QP per
  PCG iteration (instead of its bytes);

and one ``colpass_min_n`` -- the smallest bucket from which the column pass
wins in every tuned bucket above it.  Tables are cached as JSON, keyed by GPU
name, storage types and precision; ``apply_tuning`` installs one in a batch
(``qp_batch_set_tuning``).  The selection rules are plain functions of the
timings, so they are tested without a GPU.
"""
from __future__ import annotations

import ctypes as C
import json
import math
import os
from typing import Callable, Dict, Iterable, List, Optional

TEAMS = (1, 2, 4, 8, 16, 32, 64, 128)
NEAR_BEST = 1.10
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "kktqp", "autotune.json")


def bucket_of(n: int) -> int:
    """floor(log2 n), the size bucket the library uses."""
    return max(0, int(math.floor(math.log2(max(1, int(n))))))


def choose_team(times: Dict[int, float]) -> int:
    """Smallest team whose time is within NEAR_BEST of the fastest."""
    best = min(times.values())
    return min(t for t, ms in times.items() if ms <= NEAR_BEST * best)


def choose_colpass(on_off: Dict[int, tuple]) -> int:
    """on_off[k] = (ms with the column pass, ms without) per bucket k: the
    threshold n = 2^k of the smallest bucket from which the column pass wins
    in every tuned bucket above; no win -> beyond every tuned bucket."""
    ks = sorted(on_off)
    if not ks:
        return 512
    thr = ks[-1] + 1
    for k in reversed(ks):
        on, off = on_off[k]
        if on < off:
            thr = k
        else:
            break
    return 1 << thr


def table_arrays(table: dict):
    """(team_cap, t_prod_us) lists over buckets 0..max, each untuned bucket
    filled from the nearest tuned one."""
    tuned = {int(k): v for k, v in table["buckets"].items()}
    nb = max(tuned) + 1
    caps, times = [], []
    for k in range(nb):
        near = min(tuned, key=lambda t: (abs(t - k), t))
        caps.append(int(tuned[near]["team_cap"]))
        # scale the one-CTA time by the work (about n^2) when borrowing a bucket
        times.append(float(tuned[near]["t_prod_us"]) * 4.0 ** (k - near))
    return caps, times


def cache_key(gpu: str, hdtype: int, adtype: int, precision: int) -> str:
    return f"{gpu}|H{hdtype}|A{adtype}|prec{precision}"


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path: str, data: dict) -> None:
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


# ---------------------------------------------------------------- GPU side
def _lib():
    from . import _batch_lib
    lib = _batch_lib()
    if not hasattr(lib, "_tune_sigs"):
        P = C.c_void_p
        lib.qp_batch_time_product.restype = C.c_int
        lib.qp_batch_time_product.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                              C.POINTER(C.c_double)]
        lib.qp_batch_set_tuning.restype = C.c_int
        lib.qp_batch_set_tuning.argtypes = [P, C.c_int, C.POINTER(C.c_int),
                                            C.POINTER(C.c_double), C.c_int]
        lib._tune_sigs = True
    return lib


def time_product(batch, i: int, team: int, precision: int, colpass_min_n: int = 0,
                 reps: int = 5) -> float:
    from . import KQ_OK, KQError
    lib = _lib()
    ms = C.c_double()
    rc = lib.qp_batch_time_product(batch.b, int(i), int(team), int(precision),
                                   int(colpass_min_n), int(reps), C.byref(ms))
    if rc != KQ_OK:
        raise KQError(rc, lib.qp_batch_last_error(batch.b).decode())
    return ms.value


def apply_tuning(batch, table: Optional[dict]) -> None:
    """Install a table (None restores the default scheduling)."""
    from . import KQ_OK, KQError
    lib = _lib()
    if table is None:
        rc = lib.qp_batch_set_tuning(batch.b, 0, None, None, 0)
    else:
        caps, times = table_arrays(table)
        ca = (C.c_int * len(caps))(*caps)
        ta = (C.c_double * len(times))(*times)
        rc = lib.qp_batch_set_tuning(batch.b, len(caps), ca, ta, int(table["colpass_min_n"]))
    if rc != KQ_OK:
        raise KQError(rc, lib.qp_batch_last_error(batch.b).decode())


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name().replace("|", " ")
    except Exception:
        return "gpu"


def autotune(sample_qps: Iterable, precision: int, reps: int = 5,
             cache: Optional[str] = DEFAULT_CACHE, force: bool = False,
             timer: Optional[Callable] = None) -> dict:
    """Tune the buckets of `sample_qps` (one representative, the largest, per
    bucket) and return the table; cached tables are reused unless `force`."""
    from . import qp_create_batch, qp_batch_destroy, KQ_BF16, KQ_F32, KQ_F64
    qps = list(sample_qps)
    rep: Dict[int, object] = {}
    for q in qps:
        k = bucket_of(q.n)
        if k not in rep or q.n > rep[k].n:
            rep[k] = q
    q0 = qps[0]
    hdt = KQ_BF16 if (q0.meta or {}).get("H_bf16_bits") is not None else KQ_F64
    adt = KQ_F32 if (q0.meta or {}).get("a_f32", False) else KQ_F64
    key = cache_key(_gpu_name(), hdt, adt, precision)
    data = load_cache(cache) if cache else {}
    if not force and key in data and all(str(k) in data[key]["buckets"] for k in rep):
        out = dict(data[key])
        out["from_cache"] = True
        return out
    ks = sorted(rep)
    b = qp_create_batch([rep[k] for k in ks])
    try:
        import torch
        sms = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        sms = 152
    tm = timer or (lambda i, team, cp: time_product(b, i, team, precision, cp, reps))
    buckets, on_off = {}, {}
    for i, k in enumerate(ks):
        q = rep[k]
        rows = q.n + q.m + q.me
        teams = [t for t in TEAMS if t <= min(sms, max(1, -(-rows // 32)))]
        times = {t: tm(i, t, 0) for t in teams}
        cap = choose_team(times)
        buckets[str(k)] = {"n": q.n, "team_cap": cap, "t_prod_us": 1e3 * times[1],
                           "times_ms": {str(t): v for t, v in times.items()}}
        if q.n >= 128 and q.m > 0:
            on_off[k] = (tm(i, cap, q.n), tm(i, cap, q.n + 1))
    qp_batch_destroy(b)
    table = {"buckets": buckets, "colpass_min_n": choose_colpass(on_off), "precision": precision,
             "key": key, "reps": reps}
    if cache:
        data = load_cache(cache)
        old = data.get(key, {}).get("buckets", {})
        old.update(buckets)
        table["buckets"] = old
        data[key] = table
        save_cache(cache, data)
    table["from_cache"] = False
    return table
