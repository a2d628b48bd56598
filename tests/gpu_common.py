"""Helpers shared by the GPU parity tests: run a workload through the C ABI and compare with the
FP64 oracle.  The tolerance is the one the force step is specified to: median relative error
<= 1e-5 and 99th percentile <= 1e-4 for accelerations, densities and du/dt, the relative error
being |got - ref| / |ref|.

Every comparison is also appended as one JSON line to the file named by the environment
variable EVOL_PARITY_REPORT (when set), so that a GPU run leaves a record of the errors."""
from __future__ import annotations

import json
import os

import numpy as np

MEDIAN_TOL = 1e-5
P99_TOL = 1e-4
# A set mismatch is explained if the oracle saw a decision closer to its threshold than this,
# relative to (threshold + the particle's coordinate scale).  The GPU takes each opening and
# near decision in FP32 on float positions, centres of mass taken relative to node centres,
# float box bounds and float lengths: its error is a few FP32 ulps (u = 6e-8) of the coordinate
# scale plus the lengths' own error relative to the threshold (h and eps agree with the oracle
# to about 1e-7), which stays below 16 u = 1e-6.
EXPLAIN_MARGIN = 1e-6
# Below this fraction of the sum of its terms' magnitudes a sum is dominated by cancellation;
# such particles are judged by |d| / sum |terms| (and counted) instead of |d| / |ref|.
CANCEL_FLOOR = 1e-2


def report(record: dict):
    """Print one comparison record and append it to $EVOL_PARITY_REPORT."""
    import inspect
    caller = next((f.function for f in inspect.stack() if f.function.startswith("test_")), None)
    record = {"test": caller, **record}
    print(json.dumps(record))
    path = os.environ.get("EVOL_PARITY_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(record) + "\n")


def run_gpu(w, params=None, check=True, precision=0, api="step", max_n=None):
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet

    build.build()
    p = params or w.params
    ds = DeviceSet(w, p, precision=precision)
    ctx = E.evol_create(max_n or max(w.n, 1), torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_set_check_mode(ctx, check)
        if api == "step":
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        else:
            E.evol_build_tree(ctx, ds.particles, ds.params)
            if p.sph and w.n_gas > 0:
                E.evol_sph_density(ctx, ds.particles, ds.params, ds.outputs)
            if p.gravity:
                E.evol_gravity(ctx, ds.particles, ds.params, ds.outputs)
            if p.sph and w.n_gas > 0:
                E.evol_sph_forces(ctx, ds.particles, ds.params, ds.outputs)
        rc = E.evol_sync(ctx, raise_on_error=False)
        res = ds.numpy()
        res["status"] = rc
        res["keys"] = E.evol_get_debug(ctx, E.EVOL_DBG_KEYS, np.uint64)
        res["perm"] = E.evol_get_debug(ctx, E.EVOL_DBG_PERM, np.int32)
        res["cube"] = E.evol_get_debug(ctx, E.EVOL_DBG_CUBE, np.float64)
        nd = E.evol_get_debug(ctx, E.EVOL_DBG_NODES, np.int32)
        nn = nd.size // 5
        res["nodes"] = dict(zip(("begin", "end", "level", "next", "nchild"), nd.reshape(5, nn)))
        res["moments"] = E.evol_get_debug(ctx, E.EVOL_DBG_MOMENTS, np.float32).reshape(nn, 20)
        if check:
            res["hashes"] = E.evol_get_debug(ctx, E.EVOL_DBG_HASHES, np.uint64).reshape(-1, 3)
            res["counts"] = E.evol_get_debug(ctx, E.EVOL_DBG_COUNTS, np.int32).reshape(-1, 3)
        res["diag"] = E.evol_get_diagnostics(ctx)
        if getattr(p, "sph", 0) and w.n_gas > 0 and (getattr(p, "visc_form", 0) or getattr(p, "balsara", 0) or
                                                     getattr(p, "variable_alpha", 0) or getattr(p, "conduction", 0)):
            res["dbg_diss"] = E.evol_get_debug(ctx, E.EVOL_DBG_DISS, np.float32).reshape(5, w.n).astype(np.float64)
    finally:
        E.evol_destroy(ctx)
    return res


def rel_stats(got, ref, sel=None):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if sel is not None:
        got, ref = got[sel], ref[sel]
    if got.ndim == 2:
        err = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    else:
        err = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    return float(np.median(err)), float(np.percentile(err, 99)), err


def assert_tol(name, got, ref, sel=None, med=MEDIAN_TOL, p99=P99_TOL, scale=None):
    """Plain relative error |got - ref| / |ref| must meet the median and p99 tolerances.

    With `scale` (the oracle's sum of the magnitudes of the individual contributions to each
    result), particles whose |ref| is below CANCEL_FLOOR of their scale -- sums dominated by
    cancellation, e.g. the acceleration at the centre of a sphere -- are taken out of the plain
    statistics and judged by |got - ref| / scale against the same tolerances; their number and
    that error are reported.  The plain relative error over all particles is reported too."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    sc = None if scale is None else np.asarray(scale, np.float64)
    if sel is not None:
        got, ref = got[sel], ref[sel]
        sc = None if sc is None else sc[sel]
    if got.ndim == 2:
        d, r = np.linalg.norm(got - ref, axis=1), np.linalg.norm(ref, axis=1)
    else:
        d, r = np.abs(got - ref), np.abs(ref)
    plain = d / np.maximum(r, 1e-300)
    floor = np.zeros(len(d), bool) if sc is None else r < CANCEL_FLOOR * sc
    judged = plain[~floor]
    m, p = (float(np.median(judged)), float(np.percentile(judged, 99))) if judged.size else (0.0, 0.0)
    rec = {"quantity": name, "n": int(len(d)), "median": m, "p99": p,
           "all_median": float(np.median(plain)) if len(d) else 0.0,
           "all_p99": float(np.percentile(plain, 99)) if len(d) else 0.0,
           "max": float(judged.max()) if judged.size else 0.0, "n_floor": int(floor.sum())}
    ok = m <= med and p <= p99
    if floor.any():
        fe = d[floor] / sc[floor]
        fm, fp = float(np.median(fe)), float(np.percentile(fe, 99))
        rec.update(floor_median=fm, floor_p99=fp)
        ok = ok and fm <= med and fp <= p99
    report(rec)
    assert ok, f"{name}: {rec}"
    return m, p


def acc(res):
    return np.stack([res["ax"], res["ay"], res["az"]], 1)


def set_mismatches(gpu_hash, ora, margin_key="margin", active=None):
    """Particles whose interaction-set hashes differ, and how many of them the oracle's own
    decision margins explain (a decision within EXPLAIN_MARGIN of its threshold).  The counts
    are reported."""
    oh = np.stack([ora["hfar"], ora["hnear"], ora["hsph"]], 1)
    bad = np.any(gpu_hash != oh, axis=1)
    if active is not None:
        bad &= active
    idx = np.flatnonzero(bad)
    mg = ora[margin_key][idx]
    explained = mg < EXPLAIN_MARGIN
    report({"quantity": "interaction_sets", "n": int(len(gpu_hash)), "mismatches": int(len(idx)),
            "explained": int(explained.sum()), "largest_margin": float(mg.max()) if len(idx) else None})
    return idx, int(explained.sum())
