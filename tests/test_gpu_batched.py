"""Batched ensemble: independent systems of uneven N in one step.  Each system's keys and
nodes must equal the oracle's tree of that system alone (bit for bit), its forces must match
the oracle per system, and a batch of one system must reproduce evol_step exactly."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol

pytestmark = pytest.mark.gpu


def _run_batched(w, offsets, precision=0):
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    ds = DeviceSet(w, precision=precision)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_step_batched(ctx, offsets, ds.particles, ds.params, ds.outputs)
        rc = E.evol_sync(ctx, raise_on_error=False)
        res = ds.numpy()
        res["status"] = rc
        res["keys"] = E.evol_get_debug(ctx, E.EVOL_DBG_KEYS, np.uint64)
        res["perm"] = E.evol_get_debug(ctx, E.EVOL_DBG_PERM, np.int32)
        nd = E.evol_get_debug(ctx, E.EVOL_DBG_NODES, np.int32)
        nn = nd.size // 5
        res["nodes"] = dict(zip(("begin", "end", "level", "next", "nchild"), nd.reshape(5, nn)))
    finally:
        E.evol_destroy(ctx)
    return res


def _sub(w, b, e):
    a = {k: np.ascontiguousarray(v[b:e]) for k, v in w.arrays().items()}
    return W.Workload("sys", **a, n_gas=e - b, params=w.params)


def test_batched_systems_match_oracle_per_system():
    w = W.ensemble(9, seed=5, log2_min=8.0, log2_max=11.5)
    w.vx[:] = np.random.default_rng(6).normal(0, 0.1, w.n).astype(np.float32)
    offs = [int(v) for v in w.sys_offsets]
    g = _run_batched(w, offs)
    assert g["status"] == 0
    nodes_seen = 0
    for k in range(len(offs) - 1):
        b, e = offs[k], offs[k + 1]
        ws = _sub(w, b, e)
        o = oracle.force_step(ws)
        t = o["tree"]
        # sorted positions of system k are [b, e); permutation maps into the caller's indices
        assert np.array_equal(g["perm"][b:e] - b, t.perm())
        assert np.array_equal(g["keys"][b:e], t.keys()[t.perm()])
        on = t.nodes()
        nn = t.nnodes
        sl = slice(nodes_seen, nodes_seen + nn)
        assert np.array_equal(g["nodes"]["begin"][sl] - b, on["begin"])
        assert np.array_equal(g["nodes"]["end"][sl] - b, on["end"])
        assert np.array_equal(g["nodes"]["level"][sl], on["level"])
        assert np.array_equal(g["nodes"]["nchild"][sl], on["nchild"])
        assert np.array_equal(g["nodes"]["next"][sl] - nodes_seen, on["next"])
        nodes_seen += nn
        a_ref = np.stack([o["ax"], o["ay"], o["az"]], 1)
        assert_tol("acc", acc(g)[b:e], a_ref, scale=o["aabs"])
        assert_tol("rho", g["rho"][b:e], o["rho"])
        assert_tol("dudt", g["dudt"][b:e], o["dudt"], scale=o["duabs"])
    assert nodes_seen == g["nodes"]["begin"].size


@pytest.mark.slow
def test_batched_fullsize_ensemble_sampled():
    # the 64-sphere ensemble of the batched benchmark (N_k from 2^10 to 2^17, 1.76 M particles):
    # every system's keys and nodes bit-exact, and a seeded sample of each system's particles
    # against the oracle run on that system alone (all its lengths solved, forces on the sample)
    # at the leaf and length-solve group sizes the batched autotuner picks for it on GB300
    p = W.Params(theta=0.5, n_nei_sph=50.0, n_nei_grav=50.0, leaf_size=16, length_group=16)
    w = W.ensemble(64, seed=5, params=p)
    w.vx[:] = np.random.default_rng(7).normal(0, 0.1, w.n).astype(np.float32)
    offs = [int(v) for v in w.sys_offsets]
    assert max(np.diff(offs)) > 1 << 16
    g = _run_batched(w, offs)
    assert g["status"] == 0
    nodes_seen = 0
    cols = {k: ([], []) for k in ("acc", "rho", "h", "eps", "dudt")}
    scales = {"acc": [], "dudt": []}
    for k in range(len(offs) - 1):
        b, e = offs[k], offs[k + 1]
        ws = _sub(w, b, e)
        idx = W.sample_indices(e - b, 48, seed=100 + k)
        o = oracle.force_step(ws, idx=idx)
        t = o["tree"]
        assert np.array_equal(g["perm"][b:e] - b, t.perm())
        assert np.array_equal(g["keys"][b:e], t.keys()[t.perm()])
        on = t.nodes()
        sl = slice(nodes_seen, nodes_seen + t.nnodes)
        for key in ("begin", "end"):
            assert np.array_equal(g["nodes"][key][sl] - b, on[key]), (k, key)
        assert np.array_equal(g["nodes"]["level"][sl], on["level"])
        assert np.array_equal(g["nodes"]["nchild"][sl], on["nchild"])
        assert np.array_equal(g["nodes"]["next"][sl] - nodes_seen, on["next"])
        nodes_seen += t.nnodes
        gi = b + idx
        cols["acc"][0].append(acc(g)[gi])
        cols["acc"][1].append(np.stack([o["ax"], o["ay"], o["az"]], 1)[idx])
        scales["acc"].append(o["aabs"][idx])
        for q in ("rho", "h", "eps", "dudt"):
            cols[q][0].append(g[q][gi])
            cols[q][1].append(o[q][idx])
        scales["dudt"].append(o["duabs"][idx])
    assert nodes_seen == g["nodes"]["begin"].size
    for q, (gv, ov) in cols.items():
        sc = np.concatenate(scales[q]) if q in scales else None
        assert_tol(q, np.concatenate(gv), np.concatenate(ov), scale=sc)


def test_batch_of_one_equals_step():
    from gpu_common import run_gpu
    w = W.evrard_sphere(3000, seed=22, sigma_v=0.1)
    g1 = run_gpu(w, check=False)
    g2 = _run_batched(w, [0, w.n])
    for k in ("ax", "ay", "az", "pot", "rho", "dudt", "h", "eps"):
        assert np.array_equal(g1[k], g2[k]), k


def test_batched_rejects_bad_offsets():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.evrard_sphere(500, seed=23)
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        for offs in ([0, 200, 100, 500], [0, 200, 499], [1, 500]):
            with pytest.raises(E.EvolError) as ei:
                E.evol_step_batched(ctx, offs, ds.particles, ds.params, ds.outputs)
            assert ei.value.code == E.EVOL_EINVAL
    finally:
        E.evol_destroy(ctx)


def test_batched_offsets_restaged_after_other_steps():
    # repeated steps of one batch skip staging their offsets; a single-system step or a batch with
    # other offsets in between must not leave stale offsets behind
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.ensemble(5, seed=12, log2_min=8.0, log2_max=10.0)
    offs = [int(v) for v in w.sys_offsets]
    merged = [offs[0]] + offs[2:]                 # systems 0 and 1 as one
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    keys = ("ax", "ay", "az", "pot", "rho", "h", "eps")
    try:
        def batched(o):
            ds.reset_lengths()
            E.evol_step_batched(ctx, o, ds.particles, ds.params, ds.outputs)
            assert E.evol_sync(ctx, raise_on_error=False) == 0
            return ds.numpy()
        g1 = batched(offs)
        g2 = batched(offs)                        # offsets not staged again
        ds.reset_lengths()
        E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert E.evol_sync(ctx, raise_on_error=False) == 0
        g3 = batched(offs)                        # after a single-system step
        gm = batched(merged)
        g4 = batched(offs)                        # after a batch with other offsets
    finally:
        E.evol_destroy(ctx)
    for g in (g2, g3, g4):
        for k in keys:
            assert np.array_equal(g[k], g1[k]), k
    assert not np.array_equal(gm["ax"], g1["ax"])
