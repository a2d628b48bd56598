"""GPU vs FP64 oracle parity of the standard SPH scheme (Sect. 3: N gas particles inside 2h, no
grad-h terms), through the C ABI, with the same tolerances and set checks as the n-h scheme."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import assert_tol, run_gpu
from test_gpu_parity import _compare
from test_gpu_dissipation import ALL, _check

pytestmark = pytest.mark.gpu


def test_standard_scheme_evrard():
    w = W.evrard_sphere(4096, seed=1, sigma_v=0.1, params=W.Params(theta=0.5, leaf_size=8, sph_scheme=1))
    g, o = _compare(w)
    assert np.all(g["omega"] == 1.0) and np.all(g["zeta"] == 0.0)


def test_standard_scheme_mixed_species_and_neighbour_counts():
    for N in (16, 64):
        w = W.hernquist_gas(n_dm=1 << 14, n_gas=1 << 13, seed=3,
                            params=W.Params(theta=0.5, leaf_size=16, sph_scheme=1, n_nei_sph=float(N)))
        w.vx[:] = np.random.default_rng(5).normal(0, 0.1, w.n).astype(np.float32)
        _compare(w)


def test_standard_scheme_periodic_shock_tube():
    w = W.shock_tube(seed=4, left=(40, 8, 8), right=(25, 5, 5))
    w.params = dataclasses.replace(w.params, sph_scheme=1)
    w.vx[:] = np.where(w.x < 0.5, 0.2, -0.2).astype(np.float32)
    _compare(w)


def test_standard_scheme_with_all_dissipation_variants():
    w = W.evrard_sphere(4096, seed=101, sigma_v=0.1, params=W.Params(theta=0.5, leaf_size=8, sph_scheme=1))
    _check(W.with_dissipation(w, seed=7, **ALL))


def test_standard_scheme_bad_neighbour_number_and_too_few_particles():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.evrard_sphere(200, seed=2, params=W.Params(theta=0.5, leaf_size=8, sph_scheme=1, n_nei_sph=400.0))
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        ds = DeviceSet(w)
        with pytest.raises(E.EvolError) as ei:
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert ei.value.code == E.EVOL_EINVAL
        # 40 gas particles cannot give 50 neighbours: the step completes and reports it
        w2 = W.evrard_sphere(40, seed=3, params=W.Params(theta=0.5, leaf_size=8, sph_scheme=1, n_nei_sph=50.0))
        ds2 = DeviceSet(w2)
        E.evol_step(ctx, ds2.particles, ds2.params, ds2.outputs)
        assert E.evol_sync(ctx, raise_on_error=False) == E.EVOL_ENOCONV
    finally:
        E.evol_destroy(ctx)
