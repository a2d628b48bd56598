"""Pins of the oracle's integrator pieces (Sect. 4.1-4.2 and the continuity equation of Sect. 2.1):
the velocity divergence, the viscosity's largest mu, the global time step and the global-step
KDK loop.

* For a homologous flow v = k r the discretised continuity equation gives div v = 3k exactly at
  every particle, whatever the particle distribution: with r dW/dr = -(3 W + eps dW/deps) the sum
  of (v_i - v_j).grad_i W equals -3 k n Upsilon.  A rigid rotation gives exactly 0.
* A uniform lattice at rest feels no force, so only the Courant criterion limits the step:
  dt = eta_C h / (c (1 + 1.2 alpha)).
* With the step clamped to a constant the global-step loop reduces to the fixed-step KDK.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W


def _with_velocity(w, vel):
    w.vx[:], w.vy[:], w.vz[:] = (np.asarray(vel[:, a], np.float32) for a in range(3))
    return w


def _positions(w):
    return np.stack([w.x, w.y, w.z], 1).astype(np.float64)


@pytest.mark.parametrize("k", [0.37, -1.3])
def test_divergence_of_homologous_flow_is_exact(k):
    w = W.hernquist_gas(n_dm=1500, n_gas=800, seed=21)
    P = _positions(w)
    w = _with_velocity(w, k * P)
    r = oracle.force_step(w)
    # the state handed to the oracle is float32: compare with 3k from the velocities actually used
    vx, vy, vz = (getattr(w, a).astype(np.float64) for a in ("vx", "vy", "vz"))
    assert np.allclose(r["divv_eps"], 3 * k, rtol=2e-6, atol=0)
    assert np.allclose(r["divv_h"][: w.n_gas], 3 * k, rtol=2e-6, atol=0)


def test_divergence_of_rigid_rotation_vanishes():
    w = W.evrard_sphere(1200, seed=22)
    P = _positions(w)
    omega = np.array([0.3, -0.8, 0.5])
    w = _with_velocity(w, np.cross(omega, P))
    r = oracle.force_step(w)
    scale = np.linalg.norm(omega)
    assert np.abs(r["divv_eps"]).max() < 1e-5 * scale
    assert np.abs(r["divv_h"]).max() < 1e-5 * scale


def test_largest_mu_of_a_head_on_pair():
    # two gas particles approaching with speed s: |mu| = hbar s r / (r^2 + 0.01 hbar^2) for both
    rr, s, h = 0.375, 2.0, (0.25, 0.3125)
    P = np.array([[0.5 * rr, 0, 0], [-0.5 * rr, 0, 0]])
    v = np.array([[-0.5 * s, 0, 0], [0.5 * s, 0, 0]])
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, leaf_size=1)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    w = W.Workload("pair", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(v[:, 0]), f(v[:, 1]), f(v[:, 2]), f([0.5, 0.75]),
                   f([1.0, 1.0]), f(h), f(h), n_gas=2, params=p)
    st = dict(h=np.asarray(h), rho=np.array([1.0, 3.0]), P=np.zeros(2), c=np.array([0.5, 1.5]), omega=np.ones(2),
              zeta=np.zeros(2))
    r = oracle.force_step(w, params=p, fixed_lengths=st)
    hb = 0.5 * (h[0] + h[1])
    mu = hb * s * rr / (rr * rr + 0.01 * hb * hb)
    assert np.allclose(r["mumax"], mu, rtol=1e-6)


def test_courant_step_of_a_lattice_at_rest():
    nx = 8
    g = (np.arange(nx) + 0.5) / nx
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(P)
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, leaf_size=8, n_nei_sph=40.0,
                 periodic_mask=7, periodic_lo=(0, 0, 0), periodic_hi=(1, 1, 1))
    f = lambda a: np.ascontiguousarray(a, np.float32)
    u = 0.7
    w = W.Workload("lattice", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), *(f(np.zeros(n)),) * 3, f(np.full(n, 1.0 / n)),
                   f(np.full(n, u)), f(np.full(n, 1.2 / nx)), f(np.full(n, 1.2 / nx)), n_gas=n, params=p)
    r = oracle.force_step(w)
    ts = oracle.TimeStep(eta_acc=0.1, eta_courant=0.2, eta_u=0.1)
    crit = oracle.timestep_criteria(w, r, w.vx, w.vy, w.vz, w.u, ts)
    c = np.sqrt(p.gamma * (p.gamma - 1) * float(np.float32(u)))     # the oracle's input u is float32
    expect = 0.2 * r["h"] / (c * (1 + 1.2 * p.alpha))
    assert np.allclose(crit["courant"], expect, rtol=1e-12, atol=0)
    # forces vanish on the symmetric lattice, so no other criterion is finite-and-smaller
    assert oracle.global_timestep(crit, ts) == pytest.approx(float(expect.min()), rel=1e-9)


def test_global_step_loop_reduces_to_fixed_step_kdk():
    w = W.evrard_sphere(600, seed=23, sigma_v=0.1)
    ts = oracle.TimeStep(dt_min=2e-3, dt_max=2e-3)
    a = oracle.run(w, 3, ts, predicted=False)
    b = oracle.kdk(w, 2e-3, 3)
    assert a["dts"] == [2e-3] * 3
    for k in ("x", "y", "z", "vx", "vy", "vz", "u"):
        assert np.array_equal(a[k], b[k]), k


def _energy(w, st, r):
    m = w.m.astype(np.float64)
    v2 = st["vx"] ** 2 + st["vy"] ** 2 + st["vz"] ** 2
    return 0.5 * np.sum(m * v2) + np.sum(m[: w.n_gas] * st["u"][: w.n_gas]) + 0.5 * np.sum(m * r["pot"])


def test_global_step_loop_conserves_energy_in_a_collapse():
    # cold self-gravitating gas sphere (the adiabatic-collapse set-up of Sect. 5.8.2): the total
    # energy stays within a few 1e-4 over 25 global steps
    w = W.evrard_sphere(1000, seed=24)
    p = W.Params(theta=0.5, leaf_size=8)
    ts = oracle.TimeStep(eta_acc=0.2, eta_courant=0.2, eta_u=0.2)
    r0 = oracle.force_step(w, params=p)
    e0 = _energy(w, {"vx": w.vx.astype(float), "vy": w.vy.astype(float), "vz": w.vz.astype(float),
                     "u": w.u.astype(float)}, r0)
    out = oracle.run(w, 25, ts, params=p)
    import copy
    cur = copy.copy(w)
    cur.x, cur.y, cur.z = (np.ascontiguousarray(out[k], np.float32) for k in ("x", "y", "z"))
    r1 = oracle.force_step(cur, params=p)
    e1 = _energy(w, out, r1)
    assert sum(out["dts"]) > 0.02
    assert abs(e1 - e0) < 5e-4 * abs(e0), (e0, e1, sum(out["dts"]))
