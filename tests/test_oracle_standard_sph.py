"""Pins of the oracle's "standard SPH scheme" (Sect. 3, the alternative to the n-h relation): h such
that a fixed number N of gas particles, the particle itself included, lies inside the kernel
support r < 2h, with the grad-h terms dropped.

* h against a brute-force sort of all pair distances: h = (r_(N) + r_(N+1)) / 4, and exactly N
  particles inside 2h.
* n and rho against brute-force kernel sums at that h (W itself is pinned by its own tests).
* Omega* = 1 and zeta = 0; the result does not depend on the starting guess.
* The SPH forces built on it still conserve momentum and energy pairwise.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

K = oracle.kernels


def _cloud(seed, n=300, n_dm=0):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, 0.3, (n + n_dm, 3)).astype(np.float32).astype(np.float64)
    m = (np.where(np.arange(n + n_dm) % 3 == 0, 2.5, 1.0) / (n + n_dm)).astype(np.float32).astype(np.float64)
    u = rng.uniform(0.5, 1.5, n + n_dm)
    v = rng.normal(0, 0.3, (n + n_dm, 3)).astype(np.float32).astype(np.float64)
    return P, m, u, v


def _wl(P, m, u, v, n_gas, **kw):
    f = lambda a: np.ascontiguousarray(a, np.float32)
    base = dict(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=32.0, leaf_size=4, sph_scheme=1)
    base.update(kw)
    n = len(m)
    return W.Workload("t", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(v[:, 0]), f(v[:, 1]), f(v[:, 2]), f(m), f(u),
                      f(np.full(n, 0.1)), f(np.full(n, 0.1)), n_gas=n_gas, params=W.Params(**base))


@pytest.mark.parametrize("N", [8, 32, 50])
def test_h_is_the_midpoint_of_the_nth_and_next_distance(N):
    P, m, u, v = _cloud(61, n=300, n_dm=100)
    ng = 300
    w = _wl(P, m, u, v, ng, n_nei_sph=float(N))
    t = oracle.OracleTree(w.x, w.y, w.z, w.m, ng, 4)
    h, nsum, rho, om, zeta = t.solve_lengths(2, float(N), guess=w.h, idx=np.arange(ng))
    Pf = np.stack([w.x, w.y, w.z], 1).astype(np.float64)[:ng]         # gas only
    D = np.linalg.norm(Pf[:, None, :] - Pf[None, :, :], axis=2)
    Ds = np.sort(D, axis=1)
    assert np.allclose(h[:ng], 0.25 * (Ds[:, N - 1] + Ds[:, N]), rtol=1e-14, atol=0)
    assert np.all((D < 2 * h[:ng, None]).sum(1) == N)
    # n and rho: kernel sums over the gas at that h (self term included)
    mg = w.m.astype(np.float64)[:ng]
    Wm = K.W(D, np.broadcast_to(h[:ng, None], D.shape))
    assert np.allclose(nsum[:ng], Wm.sum(1), rtol=1e-13)
    assert np.allclose(rho[:ng], (Wm * mg[None, :]).sum(1), rtol=1e-13)
    assert np.all(om[:ng] == 1.0) and np.all(zeta[:ng] == 0.0)


def test_h_does_not_depend_on_the_guess():
    P, m, u, v = _cloud(62)
    w = _wl(P, m, u, v, len(m))
    t = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, 4)
    h1 = t.solve_lengths(2, 32.0, guess=w.h)[0]
    h2 = t.solve_lengths(2, 32.0, guess=w.h * 7.0)[0]
    h3 = t.solve_lengths(2, 32.0, guess=w.h / 5.0)[0]
    assert np.array_equal(h1, h2) and np.array_equal(h1, h3)


def test_too_few_gas_particles_fail():
    P, m, u, v = _cloud(63, n=20)
    w = _wl(P, m, u, v, len(m))
    t = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, 4)
    with pytest.raises(RuntimeError):
        t.solve_lengths(2, 32.0, guess=w.h)


def test_forces_conserve_momentum_and_energy():
    P, m, u, v = _cloud(64)
    w = _wl(P, m, u, v, len(m), use_tc_gradient=1, alpha=1.0, beta=2.0)
    r = oracle.force_step(w)
    assert np.all(r["omega"] == 1.0) and np.all(r["zeta"] == 0.0)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    mom = (m[:, None] * a).sum(0)
    assert np.all(np.abs(mom) < 1e-13 * (m[:, None] * np.abs(a)).sum())
    e = m * ((v * a).sum(1) + r["dudt"])
    assert abs(e.sum()) < 1e-13 * np.abs(m * (v * a).sum(1)).sum()
