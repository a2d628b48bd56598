"""Periodic gravity by the Ewald method (Sect. 4.3) on the GPU against the FP64 oracle, through the
C ABI: nearest images, the tabulated correction on every pair and far node, the periodic
potential; a grid-aligned lattice against its closed form."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, run_gpu, set_mismatches

pytestmark = pytest.mark.gpu

MADELUNG_SC = 2.8372974794806


def _box(n, seed, L=1.0, gas=0, sigma_v=0.0, **kw):
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, L, (n, 3))
    # a clustered part so that the tree has depth: half the particles in three Gaussian clumps
    k = n // 2
    centres = rng.uniform(0.1, 0.9, (3, 3)) * L
    P[:k] = np.mod(centres[rng.integers(0, 3, k)] + rng.normal(0, 0.05 * L, (k, 3)), L)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    v = rng.normal(0, sigma_v, (n, 3)) if sigma_v > 0 else np.zeros((n, 3))
    m = np.full(n, 1.0 / n)
    base = dict(theta=0.5, gravity=1, sph=1 if gas else 0, adaptive_softening=1, n_nei_grav=32.0,
                n_nei_sph=40.0, leaf_size=8, periodic_mask=7, periodic_lo=(0, 0, 0), periodic_hi=(L, L, L))
    base.update(kw)
    u = np.full(n, 0.5)
    h = np.full(n, 0.05 * L)
    return W.Workload("box", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(v[:, 0]), f(v[:, 1]), f(v[:, 2]), f(m), f(u), f(h),
                      f(h), n_gas=gas, params=W.Params(**base))


def _compare(w, precision=0):
    g = run_gpu(w, w.params, check=True, precision=precision)
    assert g["status"] == 0, g["status"]
    o = oracle.force_step(w)
    idx, explained = set_mismatches(g["hashes"], o)
    assert len(idx) == explained
    assert_tol("eps", g["eps"], o["eps"])
    assert_tol("acc", acc(g), np.stack([o["ax"], o["ay"], o["az"]], 1), scale=o["aabs"])
    assert_tol("pot", g["pot"], o["pot"])
    if w.n_gas and np.any(w.vx != 0):
        assert_tol("dudt", g["dudt"], o["dudt"][: w.n_gas], scale=o["duabs"][: w.n_gas])
    return g, o


def test_periodic_box_gravity():
    _compare(_box(4096, 91))


def test_periodic_box_gravity_mixed_precision_and_direct_sum():
    _compare(_box(3000, 92), precision=1)
    _compare(_box(2000, 93, theta=0.0))


def test_periodic_box_with_gas():
    _compare(_box(4096, 94, gas=2048, sigma_v=0.1))


def test_periodic_lattice_closed_form():
    n, L = 8, 2.0
    g1 = (np.arange(n) + 0.5) * (L / n)
    P = np.stack(np.meshgrid(g1, g1, g1, indexing="ij"), -1).reshape(-1, 3)
    N = len(P)
    eps = 0.2 * L / n
    f = lambda a: np.ascontiguousarray(a, np.float32)
    z = np.zeros(N)
    p = W.Params(theta=0.5, gravity=1, sph=0, adaptive_softening=0, leaf_size=8, periodic_mask=7,
                 periodic_lo=(0, 0, 0), periodic_hi=(L, L, L))
    w = W.Workload("lattice", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(z), f(z), f(z), f(np.full(N, 1.0 / N)), f(z),
                   f(np.full(N, eps)), f(np.full(N, eps)), n_gas=0, params=p)
    g = run_gpu(w, p, check=False)
    assert g["status"] == 0
    m = 1.0 / N
    expect = m * (MADELUNG_SC / (L / n) - 1.4 / eps)
    assert_tol("lattice_pot", g["pot"], np.full(N, expect))
    assert np.abs(acc(g)).max() < 1e-4 * m / (L / n) ** 2


def test_periodic_gravity_arguments():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    import dataclasses
    build.build()
    w = _box(500, 95)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        for kw in (dict(periodic_mask=3), dict(periodic_hi=(1.0, 1.0, 0.5))):
            ds = DeviceSet(w, dataclasses.replace(w.params, **kw))
            with pytest.raises(E.EvolError) as ei:
                E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
            assert ei.value.code == E.EVOL_EINVAL, kw
    finally:
        E.evol_destroy(ctx)
