"""The device integrator (evol_run: global-time-step KDK, Sect. 4.1-4.2) against the FP64 oracle's
global-step loop, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import assert_tol, report

pytestmark = pytest.mark.gpu


def _gpu_run(w, ts, nsteps, predicted=1, predict_lengths=1, params=None):
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    p = params or w.params
    ds = DeviceSet(w, p)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        ip = E.make_integrator(ts.eta_acc, ts.eta_vel, ts.eta_av, ts.eta_courant, ts.eta_u, ts.dt_min, ts.dt_max,
                               predicted, predict_lengths)
        t, dt = E.evol_run(ctx, ds.particles, ds.params, ip, ds.outputs, nsteps)
        assert E.evol_sync(ctx, raise_on_error=False) == 0
        flow = E.evol_get_debug(ctx, E.EVOL_DBG_FLOW, np.float32).reshape(3, w.n).astype(np.float64)
        cnt = E.evol_get_counters(ctx)
        st = {k: ds.inp[k].cpu().numpy().astype(np.float64) for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
        st["ax"], st["ay"], st["az"], st["dudt"] = (ds.out[k].cpu().numpy().astype(np.float64)
                                                    for k in ("ax", "ay", "az", "dudt"))
    finally:
        E.evol_destroy(ctx)
    return t, dt, st, flow, cnt


def _ts(**kw):
    base = dict(eta_acc=0.1, eta_courant=0.2, eta_u=0.2, dt_max=0.05)
    base.update(kw)
    return oracle.TimeStep(**base)


def _flow_close(name, got, ref):
    # a divergence changes sign across the flow: judged against its root-mean-square value
    d = np.abs(got - ref) / np.sqrt(np.mean(ref ** 2))
    rec = {"quantity": name, "median": float(np.median(d)), "p99": float(np.percentile(d, 99))}
    report(rec)
    assert rec["median"] <= 1e-5 and rec["p99"] <= 1e-4, rec


def test_one_step_matches_oracle():
    w = W.evrard_sphere(2048, seed=31, sigma_v=0.1)
    ts = _ts()
    o = oracle.run(w, 1, ts)
    t, dt, g, flow, _ = _gpu_run(w, ts, 1)
    # the step is the minimum over all particles of criteria built from FP32 results
    report({"quantity": "dt", "gpu": t, "oracle": o["dts"][0]})
    assert abs(t - o["dts"][0]) <= 2e-5 * o["dts"][0]
    assert dt == pytest.approx(t, rel=1e-6)
    v0 = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    dv_g = np.stack([g["vx"], g["vy"], g["vz"]], 1) - v0
    dv_o = np.stack([o["vx"], o["vy"], o["vz"]], 1) - v0
    assert_tol("dv", dv_g, dv_o, scale=o["dts"][0] * o["last"]["aabs"])
    # du/dt of the last force step (the change of the FP32 state u itself is below u's own rounding)
    assert_tol("dudt", g["dudt"][: w.n_gas], o["last"]["dudt"][: w.n_gas], scale=o["last"]["duabs"][: w.n_gas])
    # the last force step's velocity divergences and largest |mu| (predicted velocities)
    r = o["last"]
    _flow_close("divv_eps", flow[0], r["divv_eps"])
    _flow_close("divv_h", flow[1][: w.n_gas], r["divv_h"][: w.n_gas])
    assert_tol("mumax", flow[2][: w.n_gas], r["mumax"][: w.n_gas], scale=np.full(w.n_gas, r["mumax"].max()))


def test_several_steps_track_oracle():
    w = W.evrard_sphere(2048, seed=32, sigma_v=0.1)
    ts = _ts()
    o = oracle.run(w, 6, ts)
    t, _, g, _, _ = _gpu_run(w, ts, 6)
    report({"quantity": "time", "gpu": t, "oracle": sum(o["dts"])})
    assert abs(t - sum(o["dts"])) <= 1e-4 * sum(o["dts"])
    X = np.stack([g["x"], g["y"], g["z"]], 1)
    Xo = np.stack([o["x"], o["y"], o["z"]], 1)
    err = np.linalg.norm(X - Xo, axis=1)
    assert np.median(err) < 1e-6 and err.max() < 1e-4, (np.median(err), err.max())


def test_constant_step_equals_fixed_step_kdk():
    # with the step clamped to a constant and no prediction, evol_run is evol_kdk bit for bit
    import torch
    from paper_0912_1786_gb300 import evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    w = W.evrard_sphere(1500, seed=33, sigma_v=0.1)
    ts = _ts(dt_min=1e-3, dt_max=1e-3)
    _, _, g, _, _ = _gpu_run(w, ts, 4, predicted=0, predict_lengths=0)
    ds = DeviceSet(w)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_kdk(ctx, ds.particles, ds.params, ds.outputs, 1e-3, 4)
        E.evol_sync(ctx)
        k = {key: ds.inp[key].cpu().numpy().astype(np.float64) for key in ("x", "y", "z", "vx", "vy", "vz", "u")}
    finally:
        E.evol_destroy(ctx)
    for key in k:
        assert np.array_equal(g[key], k[key]), key


def test_predicted_lengths_cut_newton_iterations():
    # a homologous collapse: the continuity-equation start follows the compression
    w = W.evrard_sphere(4096, seed=34)
    P = np.stack([w.x, w.y, w.z], 1)
    w.vx[:], w.vy[:], w.vz[:] = (np.float32(-0.8) * P[:, a] for a in range(3))
    ts = _ts(eta_acc=0.2, eta_courant=0.3, eta_u=0.3)
    _, _, g0, _, c0 = _gpu_run(w, ts, 3, predict_lengths=0)
    _, _, g1, _, c1 = _gpu_run(w, ts, 3, predict_lengths=1)
    it0, it1 = c0[24] + c0[25], c1[24] + c1[25]
    report({"quantity": "newton_iterations_last_step", "without_prediction": int(it0), "with_prediction": int(it1)})
    assert it1 < 0.85 * it0
    # the starting point changes the cost, not the result
    a0 = np.stack([g0["ax"], g0["ay"], g0["az"]], 1)
    a1 = np.stack([g1["ax"], g1["ay"], g1["az"]], 1)
    assert_tol("acc_prediction_invariance", a1, a0, med=1e-5, p99=1e-4)
