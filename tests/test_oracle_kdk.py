"""Pins of the oracle's leapfrog (Sect. 4.1): second-order accuracy on a two-body orbit and
time reversibility; exact conservation of linear momentum by the pairwise SPH forces."""
import numpy as np

import oracle
from paper_0912_1786_gb300 import workloads as W


def _two_body(dt):
    # circular orbit of two equal point masses (softening far below the separation)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    m = np.array([0.5, 0.5])
    x = np.array([-0.5, 0.5]); vy = np.array([-0.5, 0.5]) * np.sqrt(0.5)   # v^2 = G m_other / (2 * sep) ... circular
    w = W.Workload("2b", f(x), f(np.zeros(2)), f(np.zeros(2)), f(np.zeros(2)), f(vy), f(np.zeros(2)), f(m),
                   f(np.zeros(2)), f(np.full(2, 1e-3)), f(np.full(2, 1e-3)), n_gas=0,
                   params=W.Params(theta=0.5, sph=0, adaptive_softening=0, leaf_size=1))
    return w


def test_leapfrog_two_body_second_order():
    # separation 1, G = 1, masses 1/2: circular speed of each body about the centre = sqrt(G m_other / (4 r)) * ...
    # the exact circular solution: omega^2 = G (m1 + m2) / d^3 = 1, v = omega * d/2 = 0.5
    errs = []
    T = 1.0
    for dt in (0.02, 0.01):
        w = _two_body(dt)
        w.vy[:] = np.array([-0.5, 0.5], np.float32)
        r = oracle.kdk(w, dt, int(round(T / dt)))
        ang = T   # omega = 1
        exact = np.array([-0.5 * np.cos(ang), 0.5 * np.cos(ang)])
        errs.append(abs(r["x"][1] - exact[1]))
    # second order: halving dt divides the error by ~4
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_leapfrog_time_reversible():
    # gravity only (adaptive softening): the leapfrog is time reversible; artificial viscosity
    # would not be (it switches on only for approaching pairs)
    w = W.plummer(300, seed=4, params=W.Params(theta=0.5, sph=0, n_nei_grav=32.0, leaf_size=4))
    fwd = oracle.kdk(w, 1e-3, 5)
    w2 = W.Workload("rev", *(np.ascontiguousarray(fwd[k], np.float32) for k in ("x", "y", "z")),
                    *(np.ascontiguousarray(-fwd[k], np.float32) for k in ("vx", "vy", "vz")),
                    w.m, np.ascontiguousarray(fwd["u"], np.float32), w.h, w.eps, n_gas=w.n_gas, params=w.params)
    back = oracle.kdk(w2, 1e-3, 5)
    # back to the start up to the float32 rounding of the restart state
    assert np.max(np.abs(back["x"] - w.x)) < 1e-5
    assert np.max(np.abs(-back["vx"] - w.vx)) < 1e-4


def test_leapfrog_sph_momentum_conserved():
    w = W.shock_tube(seed=4, left=(20, 4, 4), right=(13, 3, 3))
    w.vx[:] = np.where(w.x < 0.5, 0.2, -0.2).astype(np.float32)
    r = oracle.kdk(w, 2e-4, 5)
    m = w.m.astype(np.float64)
    p0 = (m * w.vx.astype(np.float64)).sum()
    p1 = (m * r["vx"]).sum()
    assert abs(p1 - p0) < 1e-9 * np.sum(m * np.abs(w.vx))
