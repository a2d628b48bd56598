"""Leapfrog (Sect. 4.1) on the GPU: one KDK step against the oracle's KDK, and 100 steps of a
small periodic shock tube recorded in a CUDA graph (conservation, density profile)."""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

from gpu_common import assert_tol

pytestmark = pytest.mark.gpu


def _gpu_kdk(w, dt, nsteps, precision=0):
    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet
    build.build()
    ds = DeviceSet(w, precision=precision)
    ctx = E.evol_create(w.n, torch.cuda.current_stream().cuda_stream)
    try:
        E.evol_kdk(ctx, ds.particles, ds.params, ds.outputs, dt, nsteps)
        E.evol_sync(ctx)
        out = {k: ds.inp[k].cpu().numpy().astype(np.float64) for k in ("x", "y", "z", "vx", "vy", "vz", "u")}
        out["diag"] = E.evol_get_diagnostics(ctx)
    finally:
        E.evol_destroy(ctx)
    return out


def _shock(seed=4):
    w = W.shock_tube(seed=seed, left=(40, 8, 8), right=(25, 5, 5))
    w.vx[:] = np.where(w.x < 0.5, 0.1, -0.1).astype(np.float32)
    return w


def test_one_kdk_step_matches_oracle():
    for w, dt in ((_shock(), 5e-4), (W.evrard_sphere(3000, seed=21, sigma_v=0.1), 1e-3)):
        g = _gpu_kdk(w, dt, 1)
        o = oracle.kdk(w, dt, 1)
        v0 = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
        dv_g = np.stack([g["vx"], g["vy"], g["vz"]], 1) - v0
        dv_o = np.stack([o["vx"], o["vy"], o["vz"]], 1) - v0
        # velocity change over one step = dt (a_0 + a_1)/2; judged like accelerations
        assert_tol("dv", dv_g, dv_o, scale=dt * o["last"]["aabs"])
        x_g = np.stack([g["x"], g["y"], g["z"]], 1)
        x_o = np.stack([o["x"], o["y"], o["z"]], 1)
        assert np.max(np.abs(x_g - x_o)) < 1e-6
        ng = w.n_gas
        if ng:
            # u is float32 state (two half kicks, each rounded to float32): allow 1.5 float32 ulps of
            # u on top of the force-level tolerance on the FP64 oracle's increment
            du_g, du_o = g["u"][:ng] - w.u[:ng], o["u"][:ng] - w.u[:ng]
            ulp = np.spacing(np.abs(o["u"][:ng]).astype(np.float32)).astype(np.float64)
            bound = 1e-4 * np.maximum(np.abs(du_o), 1e-2 * dt * o["last"]["duabs"][:ng]) + 1.5 * ulp
            assert np.all(np.abs(du_g - du_o) <= bound), np.max(np.abs(du_g - du_o) / bound)


def test_hundred_steps_shock_tube_graph():
    w = _shock()
    dt, nsteps = 5e-4, 100
    g = _gpu_kdk(w, dt, nsteps)
    m = w.m.astype(np.float64)
    # momentum: pairwise forces conserve it to rounding
    p0 = np.sum(m * w.vx)
    assert abs(np.sum(m * g["vx"]) - p0) < 1e-4 * np.sum(m * np.abs(w.vx))
    # total energy (kinetic + thermal) is conserved up to the leapfrog's O(dt^2) error; that error
    # (about 1e-3 of e0 here) is the integrator's, so the GPU's energy must follow the FP64
    # oracle's own 100 steps
    def energy(vx, vy, vz, u):
        return np.sum(0.5 * m * (vx ** 2 + vy ** 2 + vz ** 2)) + np.sum(m[: w.n_gas] * u[: w.n_gas])

    e0 = energy(w.vx.astype(np.float64), w.vy, w.vz, w.u.astype(np.float64))
    e1 = energy(g["vx"], g["vy"], g["vz"], g["u"])
    o = oracle.kdk(w, dt, nsteps)
    e1_o = energy(o["vx"], o["vy"], o["vz"], o["u"])
    assert abs(e1 - e0) < 2e-3 * e0
    assert abs(e1 - e1_o) < 1e-5 * e0
    # x-binned mass profile against the oracle's 100 steps
    bins = np.linspace(0, 1, 21)
    hg, _ = np.histogram(g["x"], bins, weights=m)
    ho, _ = np.histogram(o["x"], bins, weights=m)
    assert np.sum(np.abs(hg - ho)) < 1e-2 * np.sum(ho)
