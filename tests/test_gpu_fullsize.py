"""Parity at the full sizes of the benchmark and the paper-shaped configurations, in the launch
configuration bench.py times (evol_step, default leaf size).  The oracle solves every particle's
lengths (they enter its neighbours' forces) and computes the force pass for a seeded sample of
particles; the GPU results of those particles are compared one by one."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, run_gpu, set_mismatches

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SAMPLE = 3000


def _check(w, precision=0, sample=SAMPLE):
    p = w.params
    g = run_gpu(w, p, check=True, precision=precision)
    assert g["status"] == 0
    idx = W.sample_indices(w.n, sample, seed=77)
    o = oracle.force_step(w, params=p, idx=idx)
    t = o["tree"]
    # structure at full size: bit-exact
    perm = t.perm()
    assert np.array_equal(g["perm"], perm)
    assert np.array_equal(g["keys"], t.keys()[perm])
    nd = t.nodes()
    for k in ("begin", "end", "level", "next", "nchild"):
        assert np.array_equal(g["nodes"][k], nd[k]), k
    ng = w.n_gas
    gas_idx = idx[idx < ng]
    if p.sph and ng:
        assert_tol("h", g["h"][gas_idx], o["h"][gas_idx])
        assert_tol("rho", g["rho"][gas_idx], o["rho"][gas_idx])
    if p.gravity and p.adaptive_softening:
        assert_tol("eps", g["eps"][idx], o["eps"][idx])
    a_ref = np.stack([o["ax"], o["ay"], o["az"]], 1)
    sel = idx if p.gravity else gas_idx
    assert_tol("acc", acc(g)[sel], a_ref[sel], scale=o["aabs"][sel])
    if p.gravity:
        assert_tol("pot", g["pot"][idx], o["pot"][idx])
    if p.sph and ng and np.any(w.vx[:ng] != 0):
        assert_tol("dudt", g["dudt"][gas_idx], o["dudt"][gas_idx], scale=o["duabs"][gas_idx])
    # interaction sets of the sampled particles
    sub = {k: o[k][idx] for k in ("hfar", "hnear", "hsph", "margin")}
    bad, explained = set_mismatches(g["hashes"][idx], sub)
    assert len(bad) == explained, f"{len(bad)} set mismatches, {explained} explained"
    return g, o


def test_fullsize_mixed_species_plain():
    w = W.hernquist_gas(n_dm=1 << 21, n_gas=1 << 20, seed=3)
    w.vx[: w.n_gas] = np.random.default_rng(5).normal(0, 0.1, w.n_gas).astype(np.float32)
    _check(w, precision=0)


def test_fullsize_mixed_species_mixed_precision():
    w = W.hernquist_gas(n_dm=1 << 21, n_gas=1 << 20, seed=3)
    _check(w, precision=1)


def test_fullsize_plummer():
    w = W.plummer(1 << 20, seed=2, params=W.Params(theta=0.6, sph=0, n_nei_grav=32.0, leaf_size=8))
    _check(w)


def test_fullsize_shock_tube():
    w = W.shock_tube(seed=4)
    w.vx[:] = np.where(w.x < 0.5, 0.2, -0.2).astype(np.float32)
    _check(w)
