"""Pins of the oracle's periodic gravity (Sect. 4.3: Ewald correction, tabulated and interpolated).

* The correction's own values: g(0) = 2.8372974794806 / L, the Madelung-type constant of a simple
  cubic lattice with a uniform neutralising background (a known number, not computed from the
  series here); at x = (L/2, 0, 0) and at the cube corner the full periodic force vanishes by
  symmetry, so the correction is exactly x / |x|^3 there; f(0) = 0.
* f = -grad g (finite differences of the potential series), the odd/even symmetries, the
  1/L^2 and 1/L scalings, and the table interpolation within its error against the series.
* The force pass: a simple cubic lattice of n^3 equal masses in the periodic cube feels no force,
  and each particle's potential is G m (2.8372974794806 / a - 7 / (5 eps)) (its lattice and the
  background, plus the softened self term), a = L / n; momentum is conserved; the tree with
  theta = 0.5 stays close to the direct sum (theta = 0) with the same corrections.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

MADELUNG_SC = 2.8372974794806


def test_self_image_constant():
    for L in (1.0, 2.5):
        f, g = oracle.ewald([0.0, 0.0, 0.0], L)
        assert abs(g - MADELUNG_SC / L) < 1e-11 / L
        assert np.all(np.abs(f) < 1e-14)


def test_correction_cancels_the_direct_force_where_the_periodic_force_vanishes():
    L = 1.7
    for x in ([L / 2, 0, 0], [0, -L / 2, 0], [L / 2, L / 2, 0], [L / 2, L / 2, L / 2]):
        x = np.array(x)
        f, _ = oracle.ewald(x, L)
        assert np.allclose(f, x / np.linalg.norm(x) ** 3, rtol=1e-10, atol=1e-12)


def test_force_is_minus_gradient_of_potential_and_symmetric():
    rng = np.random.default_rng(81)
    L = 1.3
    for _ in range(6):
        x = rng.uniform(-0.45, 0.45, 3) * L
        f, g = oracle.ewald(x, L)
        h = 1e-5 * L
        fd = np.array([-(oracle.ewald(x + h * e, L)[1] - oracle.ewald(x - h * e, L)[1]) / (2 * h) for e in np.eye(3)])
        assert np.allclose(f, fd, rtol=1e-7, atol=1e-8)
        # odd in its own coordinate, even in the others; g even; axes interchangeable
        for a in range(3):
            xm = x.copy()
            xm[a] = -xm[a]
            fm, gm = oracle.ewald(xm, L)
            assert abs(gm - g) < 1e-12
            for b in range(3):
                assert abs(fm[b] - (-f[b] if b == a else f[b])) < 1e-12
        fp, gp = oracle.ewald(x[[1, 2, 0]], L)
        assert np.allclose(fp, f[[1, 2, 0]], atol=1e-12) and abs(gp - g) < 1e-12
        # scaling with the box
        f1, g1 = oracle.ewald(x / L, 1.0)
        assert np.allclose(f, f1 / L ** 2, rtol=1e-12) and abs(g - g1 / L) < 1e-12


def test_table_interpolation_error():
    rng = np.random.default_rng(82)
    L = 1.0
    worst_f = worst_g = 0.0
    for _ in range(300):
        x = rng.uniform(-0.5, 0.5, 3) * L
        fe, ge = oracle.ewald(x, L)
        ft, gt = oracle.ewald(x, L, exact=False)
        worst_f = max(worst_f, float(np.abs(fe - ft).max()))
        worst_g = max(worst_g, abs(ge - gt))
    # trilinear on a grid of spacing L/128: error ~ spacing^2 |second derivative| / 8, largest near
    # the faces, where |f| reaches 4 / L^2: within 1e-4 of that scale (g: of its 2.84 / L)
    assert worst_f < 4e-4 and worst_g < 3e-4
    # grid points are exact
    fe, ge = oracle.ewald([0.25, 0.125, 0.0], L)
    ft, gt = oracle.ewald([0.25, 0.125, 0.0], L, exact=False)
    assert np.allclose(fe, ft, atol=1e-15) and abs(ge - gt) < 1e-15


def _lattice(n, L, eps):
    g = (np.arange(n) + 0.5) * (L / n)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    N = len(P)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    p = W.Params(theta=0.0, gravity=1, sph=0, adaptive_softening=0, leaf_size=1, periodic_mask=7,
                 periodic_lo=(0, 0, 0), periodic_hi=(L, L, L))
    z = np.zeros(N)
    return W.Workload("lattice", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(z), f(z), f(z), f(np.full(N, 1.0 / N)), f(z),
                      f(np.full(N, eps)), f(np.full(N, eps)), n_gas=0, params=p)


@pytest.mark.parametrize("n, rtol", [(4, 1e-9), (8, 1e-9), (6, 2e-3)])
def test_periodic_lattice_is_in_equilibrium_with_the_madelung_potential(n, rtol):
    # for n = 4 and 8 every pair offset is a table grid point (exact values); for n = 6 the
    # interpolation error of the corrections, summed over the pairs, sets the tolerance
    L = 1.0
    eps = 0.2 * L / n                      # neighbours at a = L/n are beyond 2 eps: unsoftened
    w = _lattice(n, L, eps)
    r = oracle.force_step(w)
    m = 1.0 / n ** 3
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    assert np.abs(a).max() < max(rtol, 1e-12) * 10 * m / (L / n) ** 2
    expect = m * (MADELUNG_SC / (L / n) - 1.4 / eps)
    assert np.allclose(r["pot"], expect, rtol=rtol)


def test_momentum_conserved_and_tree_close_to_direct_sum():
    rng = np.random.default_rng(83)
    N, L = 400, 1.0
    P = rng.uniform(0, L, (N, 3))
    f = lambda a: np.ascontiguousarray(a, np.float32)
    z = np.zeros(N)
    m = np.where(np.arange(N) % 4 == 0, 3.0, 1.0) / N
    base = dict(gravity=1, sph=0, adaptive_softening=1, n_nei_grav=32.0, leaf_size=4, periodic_mask=7,
                periodic_lo=(0, 0, 0), periodic_hi=(L, L, L))
    wd = W.Workload("box", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(z), f(z), f(z), f(m), f(z), f(np.full(N, 0.05)),
                    f(np.full(N, 0.05)), n_gas=0, params=W.Params(theta=0.0, **base))
    d = oracle.force_step(wd)
    ad = np.stack([d["ax"], d["ay"], d["az"]], 1)
    mw = wd.m.astype(np.float64)
    assert np.all(np.abs((mw[:, None] * ad).sum(0)) < 1e-12 * (mw[:, None] * np.abs(ad)).sum())
    wt = W.Workload("box", wd.x, wd.y, wd.z, wd.vx, wd.vy, wd.vz, wd.m, wd.u, wd.h, wd.eps, n_gas=0,
                    params=W.Params(theta=0.5, **base))
    t = oracle.force_step(wt)
    at = np.stack([t["ax"], t["ay"], t["az"]], 1)
    err = np.linalg.norm(at - ad, axis=1) / np.linalg.norm(ad, axis=1)
    assert np.median(err) < 3e-3 and t["nfar"].sum() > 0
