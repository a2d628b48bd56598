"""The autotuner picks one of the candidate leaf sizes by timing; the step with the chosen leaf
size still matches the oracle run with the same leaf size (theta and N_nei untouched)."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, run_gpu

pytestmark = pytest.mark.gpu


def test_autotune_returns_candidate_and_parity_holds():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.hernquist_gas(n_dm=1 << 14, n_gas=1 << 13, seed=3)
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        best, ms = E.evol_autotune(ctx, ds.particles, ds.params, ds.outputs, candidates=[4, 8, 16], reps=2)
    finally:
        E.evol_destroy(ctx)
    assert best in (4, 8, 16)
    assert all(v > 0 for v in ms.values())
    assert ds.params.theta == w.params.theta and ds.params.n_nei_sph == w.params.n_nei_sph
    p = W.Params(theta=w.params.theta, leaf_size=best)
    g = run_gpu(w, p, check=False)
    o = oracle.force_step(w, params=p)
    assert_tol("acc", acc(g), np.stack([o["ax"], o["ay"], o["az"]], 1), scale=o["aabs"])


def test_length_group_autotune_returns_candidate_and_rejects_bad_sizes():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.hernquist_gas(n_dm=1 << 14, n_gas=1 << 13, seed=3, params=W.Params(theta=0.5, leaf_size=16))
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        best, ms = E.evol_autotune_length_group(ctx, ds.particles, ds.params, ds.outputs, candidates=[4, 8, 16],
                                                reps=2)
        ds.params.length_group = 33
        with pytest.raises(E.EvolError) as ei:
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert ei.value.code == E.EVOL_EINVAL
    finally:
        E.evol_destroy(ctx)
    assert best in (4, 8, 16)
    assert all(v > 0 for v in ms.values())


@pytest.mark.parametrize("lg", [1, 4, 16, 32])
def test_length_group_changes_cost_not_results(lg):
    # every group size gives the oracle's lengths, densities and forces
    w = W.hernquist_gas(n_dm=1 << 13, n_gas=1 << 12, seed=8, params=W.Params(theta=0.5, leaf_size=16, length_group=lg))
    o = oracle.force_step(w)
    g = run_gpu(w, check=False)
    assert g["status"] == 0
    ng = w.n_gas
    assert_tol("h", g["h"], o["h"][:ng])
    assert_tol("rho", g["rho"], o["rho"][:ng])
    assert_tol("eps", g["eps"], o["eps"])
    assert_tol("acc", acc(g), np.stack([o["ax"], o["ay"], o["az"]], 1), scale=o["aabs"])


def test_batched_autotune_picks_candidates_and_parity_holds():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.ensemble(6, seed=9, log2_min=9.0, log2_max=12.0)
    offs = [int(v) for v in w.sys_offsets]
    ds = DeviceSet(w)
    h0, e0 = ds.inp["h"].clone(), ds.inp["eps"].clone()
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        leaf, ms = E.evol_autotune_batched(ctx, offs, ds.particles, ds.params, ds.outputs,
                                           which=E.EVOL_TUNE_LEAF_SIZE, candidates=[8, 16], reps=2)
        ds.params.leaf_size = leaf
        grp, msg = E.evol_autotune_batched(ctx, offs, ds.particles, ds.params, ds.outputs,
                                           which=E.EVOL_TUNE_LENGTH_GROUP, candidates=[4, 16], reps=2)
        # the caller's starting lengths are back after tuning
        assert torch.equal(ds.inp["h"], h0) and torch.equal(ds.inp["eps"], e0)
        for bad in (dict(which=2), dict(which=E.EVOL_TUNE_LENGTH_GROUP, candidates=[33]),
                    dict(which=E.EVOL_TUNE_LEAF_SIZE, candidates=[0])):
            with pytest.raises(E.EvolError) as ei:
                E.evol_autotune_batched(ctx, offs, ds.particles, ds.params, ds.outputs, reps=1, **bad)
            assert ei.value.code == E.EVOL_EINVAL
        with pytest.raises(E.EvolError) as ei:
            E.evol_autotune_batched(ctx, [0, 10, 5, w.n], ds.particles, ds.params, ds.outputs, reps=1)
        assert ei.value.code == E.EVOL_EINVAL
        ds.params.length_group = grp
        E.evol_step_batched(ctx, offs, ds.particles, ds.params, ds.outputs)
        assert E.evol_sync(ctx, raise_on_error=False) == 0
        g = ds.numpy()
    finally:
        E.evol_destroy(ctx)
    assert leaf in (8, 16) and grp in (4, 16)
    assert all(v > 0 for v in list(ms.values()) + list(msg.values()))
    p = W.Params(theta=w.params.theta, n_nei_sph=w.params.n_nei_sph, n_nei_grav=w.params.n_nei_grav, leaf_size=leaf)
    for k in range(len(offs) - 1):
        b, e = offs[k], offs[k + 1]
        ws = W.Workload("sys", **{key: np.ascontiguousarray(v[b:e]) for key, v in w.arrays().items()},
                        n_gas=e - b, params=p)
        o = oracle.force_step(ws)
        assert_tol("acc", acc(g)[b:e], np.stack([o["ax"], o["ay"], o["az"]], 1), scale=o["aabs"])
        assert_tol("rho", g["rho"][b:e], o["rho"])
