"""GPU vs FP64 oracle parity, through the C ABI, at sizes the oracle finishes in seconds.

Integer structure (cube, keys, permutation, nodes) must be bit-exact.  Opening / neighbour
decisions are compared as per-particle set hashes: every mismatch must be explained by an
oracle decision within 1e-5 of its threshold.  Floating results must meet median <= 1e-5 and
p99 <= 1e-4 relative error against the oracle; accelerations and du/dt, which are sums with
cancellation, are judged relative to max(|ref|, 1% of the sum of their terms' magnitudes)."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, rel_stats, run_gpu, set_mismatches

pytestmark = pytest.mark.gpu


def _structure(g, o):
    t = o["tree"]
    c, s = t.cube()
    assert np.array_equal(g["cube"], np.concatenate([c, [s]]))
    perm = t.perm()
    assert np.array_equal(g["perm"], perm)
    assert np.array_equal(g["keys"], t.keys()[perm])
    on = t.nodes()
    for k in ("begin", "end", "level", "next", "nchild"):
        assert np.array_equal(g["nodes"][k], on[k]), k
    mo = t.moments()
    gm = g["moments"]
    assert np.allclose(gm[:, 0], mo["M"], rtol=2e-6)
    assert np.allclose(gm[:, 11:14], mo["bmin"], rtol=0, atol=0)
    assert np.allclose(gm[:, 14:17], mo["bmax"], rtol=0, atol=0)
    scale = np.abs(mo["com"]).max()
    assert np.abs(gm[:, 1:4] - mo["com"]).max() <= 2e-6 * scale


def _sets(g, o, n_active=None):
    idx, explained = set_mismatches(g["hashes"], o)
    assert len(idx) == explained, f"{len(idx)} interaction-set mismatches, {explained} explained at threshold"
    return len(idx)


def _compare(w, params=None, precision=0, api="step", med=1e-5, p99=1e-4):
    p = params or w.params
    g = run_gpu(w, p, check=True, precision=precision, api=api)
    assert g["status"] == 0, g["status"]
    o = oracle.force_step(w, params=p)
    _structure(g, o)
    ng = w.n_gas
    if p.sph and ng:
        assert_tol("h", g["h"], o["h"][:ng], med=med, p99=p99)
        assert_tol("rho", g["rho"], o["rho"][:ng], med=med, p99=p99)
        assert_tol("omega", g["omega"], o["omega"][:ng], med=med, p99=p99)
    if p.gravity and p.adaptive_softening:
        assert_tol("eps", g["eps"], o["eps"], med=med, p99=p99)
    a_ref = np.stack([o["ax"], o["ay"], o["az"]], 1)
    if p.gravity or p.sph:
        sel = None if p.gravity else np.arange(ng)
        assert_tol("acc", acc(g), a_ref, sel=sel, med=med, p99=p99, scale=o["aabs"])
    if p.gravity:
        assert_tol("pot", g["pot"], o["pot"], med=med, p99=p99)
    if p.sph and ng and np.any(w.vx != 0):
        assert_tol("dudt", g["dudt"], o["dudt"][:ng], med=med, p99=p99, scale=o["duabs"][:ng])
    if api == "step":
        _sets(g, o)
    return g, o


def test_c1_evrard_leaf1():
    w = W.evrard_sphere(4096, seed=1, sigma_v=0.1, params=W.Params(theta=0.5, leaf_size=1))
    _compare(w)


def test_c1_evrard_leaf8_ragged():
    w = W.evrard_sphere(4099, seed=101, sigma_v=0.1)
    _compare(w)


def test_c1_zero_velocity_as_specified():
    w = W.evrard_sphere(4096, seed=1)
    g, o = _compare(w)
    # v = 0: du/dt vanishes identically on both sides
    assert np.all(g["dudt"] == 0)


def test_c1_mixed_precision():
    w = W.evrard_sphere(4096, seed=1, sigma_v=0.1)
    _compare(w, precision=1)


def test_c2_plummer_gravity_only():
    for th in (0.4, 0.8):
        w = W.plummer(1 << 15, seed=2, params=W.Params(theta=th, sph=0, n_nei_grav=32.0, leaf_size=8))
        _compare(w)


def test_c3_mixed_species():
    w = W.hernquist_gas(n_dm=1 << 15, n_gas=1 << 14, seed=3)
    w.vx[:] = np.random.default_rng(5).normal(0, 0.1, w.n).astype(np.float32)
    _compare(w)


def test_c4_shock_tube_periodic():
    w = W.shock_tube(seed=4, left=(40, 8, 8), right=(25, 5, 5))
    w.vx[:] = np.where(w.x < 0.5, 0.2, -0.2).astype(np.float32)    # converging flow: viscosity active
    _compare(w)


def test_separate_calls_match_oracle():
    w = W.evrard_sphere(3000, seed=11, sigma_v=0.1)
    p = W.Params(theta=0.5, leaf_size=8)
    g = run_gpu(w, p, check=False, api="separate")
    assert g["status"] == 0
    # separate calls: gravity walk without the SPH radius, SPH walk without gravity
    og = oracle.force_step(w, params=W.Params(theta=0.5, leaf_size=8, sph=0))
    os_ = oracle.force_step(w, params=W.Params(theta=0.5, leaf_size=8, gravity=0, adaptive_softening=0))
    a_ref = np.stack([og["ax"] + os_["ax"], og["ay"] + os_["ay"], og["az"] + os_["az"]], 1)
    assert_tol("acc", acc(g), a_ref, scale=og["aabs"] + os_["aabs"])
    assert_tol("dudt", g["dudt"], os_["dudt"], scale=os_["duabs"])
    assert_tol("rho", g["rho"], os_["rho"])


def test_direct_sum_theta_zero():
    w = W.evrard_sphere(2048, seed=12, sigma_v=0.1, params=W.Params(theta=0.0, leaf_size=4))
    g, o = _compare(w)
    assert g["diag"][12] == 0      # no far nodes at theta = 0


def test_diagnostics_conservation():
    # SPH terms are pairwise antisymmetric: sum m a_hyd ~ 0 and sum m (v.a_hyd + du/dt) ~ 0
    w = W.evrard_sphere(4096, seed=13, sigma_v=0.2)
    p = W.Params(theta=0.5, gravity=0, adaptive_softening=0, leaf_size=8)
    g = run_gpu(w, p, check=False)
    d = g["diag"]
    m = w.m.astype(np.float64)
    scale = np.sum(m * np.linalg.norm(acc(g), axis=1))
    assert abs(d[3]) < 1e-5 * scale and abs(d[4]) < 1e-5 * scale and abs(d[5]) < 1e-5 * scale
    escale = np.sum(m * np.abs(g["dudt"]))
    assert abs(d[9]) < 1e-5 * escale


# ---- edge cases ---------------------------------------------------------------------------
def test_single_particle_fixed_softening():
    w = W.plummer(1, seed=3, params=W.Params(theta=0.5, sph=0, adaptive_softening=0, leaf_size=1))
    g = run_gpu(w, check=True)
    assert g["status"] == 0
    assert np.all(acc(g) == 0)
    # potential = self term G m phi(0, eps) = -7/5 m / eps
    assert np.isclose(g["pot"][0], -1.4 * w.m[0] / w.eps[0], rtol=1e-6)


def test_identical_particles_chain():
    n = 40
    w = W.plummer(n, seed=3, params=W.Params(theta=0.5, sph=0, adaptive_softening=0, leaf_size=1))
    for k in ("x", "y", "z"):
        getattr(w, k)[:] = 0.125
    g = run_gpu(w, check=False)
    assert g["status"] == 0
    o = oracle.force_step(w)
    _structure(g, o)
    assert np.all(acc(g) == 0)


def test_too_few_particles_reports_noconv():
    w = W.evrard_sphere(4, seed=3)
    g = run_gpu(w, check=False)
    from paper_0912_1786_gb300 import evol as E
    assert g["status"] == E.EVOL_ENOCONV


def test_bad_arguments_rejected():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.evrard_sphere(256, seed=3)
    ds = DeviceSet(w)
    ctx = E.evol_create(128, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(E.EvolError) as ei:
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)      # n > capacity
        assert ei.value.code == E.EVOL_ENOMEM
    finally:
        E.evol_destroy(ctx)
    ctx = E.evol_create(256, torch.cuda.current_stream().cuda_stream)
    try:
        ds.params.periodic_mask = 2                                     # periodic gravity: unsupported
        with pytest.raises(E.EvolError) as ei:
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert ei.value.code == E.EVOL_EINVAL
        ds.params.periodic_mask = 0
        with pytest.raises(E.EvolError) as ei:                          # forces before density
            E.evol_sph_forces(ctx, ds.particles, ds.params, ds.outputs)
        assert ei.value.code == E.EVOL_ESTATE
        empty = E.make_particles(0, 0, {})
        E.evol_step(ctx, empty, ds.params, ds.outputs)                  # n = 0: no-op
        assert E.evol_sync(ctx) == 0
    finally:
        E.evol_destroy(ctx)


def test_host_buffer_step_matches_device_step():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    build.build()
    w = W.evrard_sphere(2000, seed=14, sigma_v=0.1)
    g = run_gpu(w, check=False)
    arrs = {k: np.ascontiguousarray(v.copy(), np.float32) for k, v in w.arrays().items()}
    outs = {k: np.zeros(w.n, np.float32) for k in E.OUTPUT_FIELDS}
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_step_host(ctx, E.make_particles(w.n, w.n_gas, arrs), E.make_params(w.params), E.make_outputs(outs))
    finally:
        E.evol_destroy(ctx)
    for k in ("ax", "ay", "az", "pot"):
        assert np.array_equal(outs[k], g[k].astype(np.float32)), k
    assert np.array_equal(outs["dudt"][: w.n_gas], g["dudt"].astype(np.float32))
