"""GPU vs FP64 oracle parity of the dissipation variants (Sect. 3.3.3), through the C ABI: the
signal-velocity viscosity, the Balsara limiter, per-particle alpha with d alpha/dt and the
artificial conductivity with d alpha^u/dt, alone and together, plain and mixed precision, with
and without gravity, periodic, and through the separate-call and host-buffer entry points.

Tolerances as for the standard force step (median <= 1e-5, p99 <= 1e-4 of |d| / |ref|), with the
sums that cancel (accelerations, du/dt, div v, curl v, lap u, the alpha switches) judged by
|d| / (sum of the magnitudes of their terms) where |ref| falls below 1% of that sum."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import acc, assert_tol, run_gpu, set_mismatches

pytestmark = pytest.mark.gpu

ALL = dict(visc_form=1, balsara=1, variable_alpha=1, conduction=1)


def _evrard(**kw):
    w = W.evrard_sphere(4096, seed=101, sigma_v=0.1, params=W.Params(theta=0.5, leaf_size=8))
    return W.with_dissipation(w, seed=7, **kw)


def _check(w, precision=0, api="step", check=True):
    p = w.params
    g = run_gpu(w, p, check=check, precision=precision, api=api)
    assert g["status"] == 0, g["status"]
    o = oracle.force_step(w, params=p)
    ng = w.n_gas
    if check:
        idx, explained = set_mismatches(g["hashes"], o)
        assert len(idx) == explained
    a_ref = np.stack([o["ax"], o["ay"], o["az"]], 1)
    sel = None if p.gravity else np.arange(ng)
    assert_tol("acc", acc(g), a_ref, sel=sel, scale=o["aabs"])
    assert_tol("dudt", g["dudt"], o["dudt"][:ng], scale=o["duabs"][:ng])
    # per-particle flow quantities of the variants (caller order, gas)
    dv, cv, f, vs, lap = g["dbg_diss"][:, :ng]
    flow = np.abs(o["divv_h"][:ng]) + o["curlv_h"][:ng]
    if p.balsara or p.variable_alpha:
        assert_tol("divv_h", dv, o["divv_h"][:ng], scale=flow)
        assert_tol("curlv_h", cv, o["curlv_h"][:ng], scale=flow)
        assert_tol("balsara_f", f, o["balsara_f"][:ng], scale=np.ones(ng))
    assert_tol("vsig", vs, o["vsig"][:ng])
    st = o["state"]
    tau = p.alpha_tau * o["h"][:ng] / o["vsig"][:ng]
    if p.variable_alpha:
        sc = np.abs(st["alpha"][:ng] - p.alpha_min) / tau + p.alpha_source * st["f"][:ng] * np.abs(o["divv_h"][:ng])
        assert_tol("dalpha", g["dalpha"], o["dalpha"][:ng], scale=sc)
    if p.conduction:
        assert_tol("lapu", lap, o["lapu"][:ng], scale=o["lapabs"][:ng])
        srcs = (o["h"][:ng] * o["lapabs"][:ng] / np.sqrt(st["u"][:ng]) if p.cond_source == 0
                else 0.1 * o["h"][:ng] * o["lapabs"][:ng])
        sc = np.abs(st["alpha_u"][:ng] - p.alpha_u_min) / tau + srcs
        assert_tol("dalpha_u", g["dalpha_u"], o["dalpha_u"][:ng], scale=sc)
    return g, o


def test_signal_velocity_viscosity():
    _check(_evrard(visc_form=1))


def test_balsara_limiter_and_variable_alpha():
    _check(_evrard(balsara=1, variable_alpha=1))


def test_all_variants_sound_speed_conduction():
    _check(_evrard(**ALL, cond_vsig=0, cond_source=0))


def test_conduction_pressure_jump_linear_source_monaghan_form():
    _check(_evrard(conduction=1, cond_vsig=1, cond_source=1))


def test_all_variants_mixed_precision():
    _check(_evrard(**ALL), precision=1)


def test_all_variants_separate_calls():
    _check(_evrard(**ALL), api="separate", check=False)


def test_all_variants_with_gravity_and_dark_matter():
    w = W.hernquist_gas(n_dm=1 << 14, n_gas=1 << 13, seed=3)
    w = W.with_dissipation(w, seed=8, sigma_v=0.1, **ALL)
    _check(w)


def test_all_variants_periodic_shock_tube():
    w = W.shock_tube(seed=4, left=(40, 8, 8), right=(25, 5, 5))
    w.vx[:] = np.where(w.x < 0.5, 0.2, -0.2).astype(np.float32)
    w = W.with_dissipation(w, seed=9, u_spread=0.0, **ALL)
    _check(w)


def test_host_buffer_step_carries_the_dissipation_arrays():
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    build.build()
    w = _evrard(**ALL)
    g = run_gpu(w, check=False)
    arrs = {k: np.ascontiguousarray(v.copy(), np.float32) for k, v in w.arrays().items()}
    arrs["alpha"], arrs["alpha_u"] = w.alpha.copy(), w.alpha_u.copy()
    outs = {k: np.zeros(w.n, np.float32) for k in E.OUTPUT_FIELDS}
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_step_host(ctx, E.make_particles(w.n, w.n_gas, arrs), E.make_params(w.params), E.make_outputs(outs))
    finally:
        E.evol_destroy(ctx)
    for k in ("ax", "ay", "az", "dudt", "dalpha", "dalpha_u"):
        ln = w.n_gas if k in ("dudt", "dalpha", "dalpha_u") else w.n
        assert np.array_equal(outs[k][:ln], g[k].astype(np.float32)), k


def test_dissipation_arguments_rejected():
    import dataclasses
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    w = _evrard(**ALL)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        bad = [dict(visc_form=2), dict(cond_vsig=3), dict(cond_source=-1), dict(alpha_tau=0.0),
               dict(balsara_eta=-1.0)]
        for kw in bad:
            ds = DeviceSet(w, dataclasses.replace(w.params, **kw))
            with pytest.raises(E.EvolError) as ei:
                E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
            assert ei.value.code == E.EVOL_EINVAL, kw
        # variable alpha / conduction without their per-particle arrays
        for k in ("alpha", "alpha_u"):
            ds = DeviceSet(w)
            setattr(ds.particles, k, None)
            with pytest.raises(E.EvolError) as ei:
                E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
            assert ei.value.code == E.EVOL_EINVAL, k
        assert E.evol_sync(ctx) == 0
    finally:
        E.evol_destroy(ctx)


def _run_device(w, nsteps, ts=None, kdk_dt=None):
    """evol_run (global step, ts given) or evol_kdk (fixed step kdk_dt); returns the final state
    including alpha and alpha^u, and the last force step's outputs."""
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        if ts is not None:
            ip = E.make_integrator(ts.eta_acc, ts.eta_vel, ts.eta_av, ts.eta_courant, ts.eta_u, ts.dt_min, ts.dt_max,
                                   1, 1)
            t, _ = E.evol_run(ctx, ds.particles, ds.params, ip, ds.outputs, nsteps)
        else:
            E.evol_kdk(ctx, ds.particles, ds.params, ds.outputs, kdk_dt, nsteps)
            t = nsteps * kdk_dt
        assert E.evol_sync(ctx, raise_on_error=False) == 0
        st = {k: v.cpu().numpy().astype(np.float64) for k, v in ds.inp.items()}
        st.update({k: v.cpu().numpy().astype(np.float64) for k, v in ds.out.items()})
    finally:
        E.evol_destroy(ctx)
    return t, st


def test_fixed_step_kdk_decays_the_switches_of_static_gas():
    # closed form (the oracle pins the same scheme): a static periodic lattice, no forces; with
    # x = k dt/2, k = 2c/(0.1 h), alpha - alpha_min ends at (1 - x)^2 (1 - 2x)^(N-1) of its start
    nx = 16
    g = (np.arange(nx) + 0.5) / nx
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(P)
    rng = np.random.default_rng(48)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=40.0, leaf_size=8,
                 periodic_mask=7, periodic_lo=(0, 0, 0), periodic_hi=(1, 1, 1), variable_alpha=1, conduction=1,
                 alpha_min=0.0625, alpha_u_min=0.0)
    u = 0.7
    w = W.Workload("lattice", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), *(f(np.zeros(n)),) * 3, f(np.full(n, 1.0 / n)),
                   f(np.full(n, u)), f(np.full(n, 1.2 / nx)), f(np.full(n, 1.2 / nx)), n_gas=n, params=p)
    w.alpha = f(rng.uniform(0.1, 1.5, n))
    w.alpha_u = f(rng.uniform(0.0, 1.0, n))
    o = oracle.force_step(w)
    k = float(np.median(o["vsig"] / (0.1 * o["h"])))
    dt = 0.2 / k
    _, st = _run_device(w, 3, kdk_dt=dt)
    fac = (1.0 - 0.1) ** 2 * (1.0 - 0.2) ** 2
    assert_tol("alpha_decay", st["alpha"] - 0.0625, (w.alpha.astype(np.float64) - 0.0625) * fac)
    assert_tol("alpha_u_decay", st["alpha_u"], w.alpha_u.astype(np.float64) * fac)


def test_global_step_run_tracks_the_oracle_with_all_variants():
    w = W.with_dissipation(W.evrard_sphere(2048, seed=49, sigma_v=0.1), seed=10, **ALL)
    ts = oracle.TimeStep(eta_acc=0.1, eta_courant=0.2, eta_u=0.2, dt_max=0.05)
    o = oracle.run(w, 3, ts)
    t, g = _run_device(w, 3, ts=ts)
    assert abs(t - sum(o["dts"])) <= 1e-4 * sum(o["dts"])
    X = np.stack([g["x"], g["y"], g["z"]], 1)
    Xo = np.stack([o["x"], o["y"], o["z"]], 1)
    err = np.linalg.norm(X - Xo, axis=1)
    assert np.median(err) < 1e-6 and err.max() < 1e-4, (np.median(err), err.max())
    # the switches after three steps, on the scale of their change
    for k in ("alpha", "alpha_u"):
        a0 = getattr(w, k).astype(np.float64)
        assert_tol(k + "_after_run", g[k] - a0, o[k] - a0, scale=np.abs(o[k] - a0) + 1e-3 * np.abs(a0))
