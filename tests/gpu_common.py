"""Helpers shared by the GPU parity tests: run a workload through the C ABI and compare with the
FP64 oracle.  The tolerance is the one the force step is specified to: median relative error
<= 1e-5 and 99th percentile <= 1e-4 for accelerations, densities and du/dt."""
from __future__ import annotations

import numpy as np

MEDIAN_TOL = 1e-5
P99_TOL = 1e-4
EXPLAIN_MARGIN = 1e-5      # a set mismatch is explained if the oracle saw a decision this close


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
    """Relative error |got - ref| / |ref|; with `scale` (the oracle's sum of the magnitudes of the
    individual contributions) the error of a sum with cancellation is taken relative to
    max(|ref|, scale * 1e-2): a result that is less than 1% of its own terms is judged on
    the terms' scale."""
    if scale is None:
        m, p, _ = rel_stats(got, ref, sel)
    else:
        got = np.asarray(got, np.float64)
        ref = np.asarray(ref, np.float64)
        sc = np.asarray(scale, np.float64)
        if sel is not None:
            got, ref, sc = got[sel], ref[sel], sc[sel]
        if got.ndim == 2:
            d, r = np.linalg.norm(got - ref, axis=1), np.linalg.norm(ref, axis=1)
        else:
            d, r = np.abs(got - ref), np.abs(ref)
        err = d / np.maximum(np.maximum(r, 1e-2 * sc), 1e-300)
        m, p = float(np.median(err)), float(np.percentile(err, 99))
    assert m <= med and p <= p99, f"{name}: median {m:.3g} (tol {med}), p99 {p:.3g} (tol {p99})"
    return m, p


def acc(res):
    return np.stack([res["ax"], res["ay"], res["az"]], 1)


def set_mismatches(gpu_hash, ora, margin_key="margin", active=None):
    """Particles whose interaction-set hashes differ, and how many of them the oracle's own
    decision margins explain (a decision within EXPLAIN_MARGIN of its threshold)."""
    oh = np.stack([ora["hfar"], ora["hnear"], ora["hsph"]], 1)
    bad = np.any(gpu_hash != oh, axis=1)
    if active is not None:
        bad &= active
    idx = np.flatnonzero(bad)
    explained = ora[margin_key][idx] < EXPLAIN_MARGIN
    return idx, int(explained.sum())
