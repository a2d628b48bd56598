"""GPU vs FP64 oracle parity, through the C ABI, at sizes the oracle finishes in seconds.

Integer structure (cube, keys, permutation, nodes) must be bit-exact.  Opening / neighbour
decisions are compared as per-particle set hashes: every mismatch must be explained by an
oracle decision within 1e-6 of its threshold (relative to threshold + coordinate scale).
Floating results must meet median <= 1e-5 and p99 <= 1e-4 plain relative error |d|/|ref|
against the oracle; particles whose acceleration or du/dt is below 1% of the sum of its terms'
magnitudes (cancellation) are counted and judged by |d| / sum |terms| instead."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, rel_stats, report, run_gpu, set_mismatches

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
    # quadrupole (traceless, about the centre of mass) on its natural scale M l^2, and delta on l
    l = mo["l"]
    qerr = np.abs(gm[:, 4:10] - mo["Q"]).max(1) / (mo["M"] * l * l)
    derr = np.abs(gm[:, 10] - mo["delta"]) / l
    report({"quantity": "node_Q", "n": int(len(l)), "median": float(np.median(qerr)),
            "p99": float(np.percentile(qerr, 99)), "max": float(qerr.max())})
    report({"quantity": "node_delta", "n": int(len(l)), "median": float(np.median(derr)),
            "p99": float(np.percentile(derr, 99)), "max": float(derr.max())})
    assert np.median(qerr) <= 1e-5 and np.percentile(qerr, 99) <= 1e-4
    assert np.median(derr) <= 1e-5 and np.percentile(derr, 99) <= 1e-4


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
        assert_tol("P", g["P"], o["P"][:ng], med=med, p99=p99)
        assert_tol("c", g["c"], o["c"][:ng], med=med, p99=p99)
        # zeta = m (1 - Omega*) for equal masses: it can vanish, so it is judged on the mass scale
        assert_tol("zeta", g["zeta"], o["zeta"][:ng], med=med, p99=p99, scale=w.m[:ng].astype(np.float64))
    if p.gravity and p.adaptive_softening:
        assert_tol("eps", g["eps"], o["eps"], med=med, p99=p99)
        assert_tol("ups", g["ups"], o["ups"], med=med, p99=p99)
        assert_tol("X", g["X"], o["X"], med=med, p99=p99)
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
        _diagnostics(w, p, g, o)
    return g, o


def _diagnostics(w, p, g, o):
    """The FP64 totals of the step against the same sums of the oracle's results."""
    d = g["diag"]
    m = w.m.astype(np.float64)
    v = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    a = np.stack([o["ax"], o["ay"], o["az"]], 1)
    ng = w.n_gas
    ref = {"sum_mv": (m[:, None] * v).sum(0), "E_kin": 0.5 * float((m * (v * v).sum(1)).sum()),
           "E_th": float((m[:ng] * w.u[:ng].astype(np.float64)).sum()) if ng else 0.0,
           "M": float(m.sum())}
    got = {"sum_mv": np.array(d[0:3]), "E_kin": d[6], "E_th": d[7], "M": d[10]}
    for k in ref:
        sc = np.abs(ref[k]).max() if np.ndim(ref[k]) else abs(ref[k])
        err = float(np.abs(np.asarray(got[k]) - ref[k]).max() / max(sc, 1e-300))
        report({"quantity": "diag_" + k, "err": err})
        assert err <= 1e-12 or sc == 0.0, (k, got[k], ref[k])
    # sum m a: a cancellation sum, judged against sum m |a|
    sma = (m[:, None] * a).sum(0)
    scale = float((m * np.linalg.norm(a, axis=1)).sum())
    err = float(np.abs(np.array(d[3:6]) - sma).max() / scale)
    report({"quantity": "diag_sum_ma", "err": err})
    assert err <= 1e-5
    if p.gravity:
        epot = 0.5 * float((m * o["pot"]).sum())
        err = abs(d[8] - epot) / abs(epot)
        report({"quantity": "diag_E_pot", "err": err})
        assert err <= 1e-5


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


def test_mixed_form_closer_to_oracle_than_plain():
    # the mixed form's FP64 moments and compensated gravity totals must show: on a halo whose
    # particles sum about a thousand far nodes each, its median acceleration and potential errors
    # are below the plain form's
    w = W.hernquist_gas(n_dm=1 << 15, n_gas=1 << 14, seed=3)
    o = oracle.force_step(w)
    a_ref = np.stack([o["ax"], o["ay"], o["az"]], 1)
    med = {}
    for prec in (0, 1):
        g = run_gpu(w, check=False, precision=prec)
        assert g["status"] == 0
        med[prec] = (rel_stats(acc(g), a_ref)[0], rel_stats(g["pot"], o["pot"])[0])
    report({"quantity": "acc_pot_median_plain_vs_mixed", "plain": med[0], "mixed": med[1]})
    assert med[1][0] < med[0][0] and med[1][1] < med[0][1]


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


def test_nan_position_reports_enan():
    # a non-finite input position: the step completes (every loop stays bounded) and reports it
    from paper_0912_1786_gb300 import evol as E
    w = W.evrard_sphere(2048, seed=15, sigma_v=0.1)
    w.x[77] = np.float32(np.nan)
    g = run_gpu(w, check=False)
    assert g["status"] == E.EVOL_ENAN


def test_nonfinite_output_reports_enan():
    # zero internal energy everywhere but one particle at +inf: P and c are infinite there
    from paper_0912_1786_gb300 import evol as E
    w = W.evrard_sphere(2048, seed=16)
    w.u[5] = np.float32(np.inf)
    g = run_gpu(w, check=False)
    assert g["status"] == E.EVOL_ENAN


def test_walk_stack_overflow_reports_eoverflow():
    # the walks check the stack bound before every push: a 32-entry stack overflows on a
    # 4096-particle sphere and the step reports EVOL_EOVERFLOW instead of writing past it
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = W.evrard_sphere(4096, seed=17)
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(E.EvolError):
            E.evol_set_stack_limit(ctx, 31)
        E.evol_set_stack_limit(ctx, 32)
        E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert E.evol_sync(ctx, raise_on_error=False) == E.EVOL_EOVERFLOW
        # restored capacity: the same context runs the step cleanly again
        E.evol_set_stack_limit(ctx, 0)
        ds.reset_lengths()
        E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
        assert E.evol_sync(ctx, raise_on_error=False) == 0
    finally:
        E.evol_destroy(ctx)


@pytest.mark.parametrize("scale", [0.5, 2.0])
def test_length_solve_from_poor_guesses(scale):
    # the solution does not depend on the starting guesses (unique root): guesses off by a factor
    # of two either way converge to the same lengths and forces
    w = W.evrard_sphere(4096, seed=18, sigma_v=0.1)
    w.h[:] = (w.h * scale).astype(np.float32)
    w.eps[:] = (w.eps * scale).astype(np.float32)
    _compare(w)


@pytest.mark.parametrize("n_nei", [60.0, 110.0])
def test_paper_neighbour_numbers(n_nei):
    # the paper's recommended range 60 <= N_nei <= 110 (Sect. 2.1): lists of that many neighbours
    # take the length solve's one-warp-per-particle form
    w = W.evrard_sphere(8192, seed=7, sigma_v=0.1,
                        params=W.Params(theta=0.5, n_nei_sph=n_nei, n_nei_grav=n_nei, leaf_size=16))
    _compare(w)
