"""Pins of the oracle's force step against what the paper and the mathematics fix.

* The gravitational acceleration with adaptive softening is the gradient of the Lagrangian's
  potential energy (Sect. 2.1, Eqs. Lgrav, dLgravdr); checked by finite differences of the
  total potential energy with the softening lengths re-solved at every displaced configuration.
  This pins the correction term (and its mass-weighted reading for unequal masses).
* The SPH pressure acceleration is minus the gradient of the adiabatic thermal energy, and du/dt
  is the time derivative of the adiabatic u along the flow (Sect. 3, Eqs. dvdt, drhodr,
  dudrho); checked by finite differences with h re-solved.  This pins the grad-h terms, the
  variable-mass factors and the signs.
* Closed forms: Plummer and rho ~ 1/r sphere accelerations; uniform lattice density.
* Conservation: pairwise antisymmetry of the SPH and direct-sum gravity terms.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

K = oracle.kernels


def _wl(P, m, n_gas, v=None, u=None, params=None, h=None, eps=None):
    n = len(m)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    v = np.zeros((n, 3)) if v is None else v
    u = np.zeros(n) if u is None else u
    g = np.full(n, 0.1) if h is None else h
    e = g if eps is None else eps
    return W.Workload("t", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(v[:, 0]), f(v[:, 1]), f(v[:, 2]), f(m), f(u),
                      f(g), f(e), n_gas=n_gas, params=params or W.Params())


def _mixed_cloud(n, seed, n_gas=None):
    rng = np.random.default_rng(seed)
    P = rng.normal(0, 0.3, (n, 3))
    m = (np.where(rng.uniform(size=n) < 0.5, 1.0, 3.0) / n).astype(np.float32).astype(np.float64)
    return P, m


def _displaced(P, i, a, step):
    """Displace particle i along axis a by about +-step, exactly representable in float32;
    returns the two position sets and the exact separation."""
    x0 = np.float32(P[i, a])
    xp = np.float32(x0 + np.float32(step))
    xm = np.float32(x0 - np.float32(step))
    Pp, Pm = P.copy(), P.copy()
    Pp[i, a] = xp
    Pm[i, a] = xm
    return Pp, Pm, float(xp) - float(xm)


GRAV = W.Params(theta=0.0, sph=0, gravity=1, adaptive_softening=1, n_nei_grav=24.0, leaf_size=2)


def _grav_energy(P, m):
    r = oracle.force_step(_wl(P, m, 0, params=GRAV))
    return 0.5 * float(np.sum(m * r["pot"]))


@pytest.mark.parametrize("seed", [21, 22])
def test_adaptive_softening_force_is_energy_gradient(seed):
    P, m = _mixed_cloud(96, seed)
    P = P.astype(np.float32).astype(np.float64)
    base = oracle.force_step(_wl(P, m, 0, params=GRAV))
    a = np.stack([base["ax"], base["ay"], base["az"]], 1)
    for i in (0, 17, 55):
        for ax in range(3):
            Pp, Pm, dx = _displaced(P, i, ax, 2e-4)
            fd = -(_grav_energy(Pp, m) - _grav_energy(Pm, m)) / dx / m[i]
            assert abs(fd - a[i, ax]) < 2e-5 * np.linalg.norm(a[i]), (i, ax, fd, a[i, ax])


def test_correction_term_matters_for_energy_gradient():
    # The check above is sensitive: dropping the correction term (X = 0) breaks it.
    P, m = _mixed_cloud(96, 21)
    P = P.astype(np.float32).astype(np.float64)
    base = oracle.force_step(_wl(P, m, 0, params=GRAV))
    st = dict(base["state"])
    st["X"] = np.zeros_like(st["X"])
    nocorr = oracle.force_step(_wl(P, m, 0, params=GRAV), fixed_lengths=st)
    i, axis = 17, 0
    Pp, Pm, dx = _displaced(P, i, axis, 2e-4)
    fd = -(_grav_energy(Pp, m) - _grav_energy(Pm, m)) / dx / m[i]
    a_full = np.array([base["ax"][i], base["ay"][i], base["az"][i]])
    assert abs(fd - base["ax"][i]) < 2e-5 * np.linalg.norm(a_full)
    assert abs(fd - nocorr["ax"][i]) > 1e-3 * np.linalg.norm(a_full)


SPH = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=24.0, leaf_size=2,
               use_tc_gradient=0, alpha=0.0, beta=0.0)


def _gas(seed, n=120):
    rng = np.random.default_rng(seed)
    P = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32).astype(np.float64)
    m = (np.where(np.arange(n) % 3 == 0, 2.5, 1.0) / n).astype(np.float32).astype(np.float64)  # unequal masses
    u = rng.uniform(0.5, 1.5, n)
    v = rng.normal(0, 0.3, (n, 3)).astype(np.float32).astype(np.float64)
    return P, m, u, v


def _rho(P, m, params=SPH):
    return oracle.force_step(_wl(P, m, len(m), params=params), idx=np.array([0]))["rho"]


@pytest.mark.parametrize("seed", [31, 32])
def test_sph_pressure_force_is_thermal_energy_gradient(seed):
    P, m, u0, _ = _gas(seed)
    g = SPH.gamma
    base = oracle.force_step(_wl(P, m, len(m), u=u0, params=SPH))
    rho0 = base["rho"]
    a = np.stack([base["ax"], base["ay"], base["az"]], 1)

    def U(Pd):
        rho = _rho(Pd, m)
        return float(np.sum(m * u0 * (rho / rho0) ** (g - 1.0)))   # adiabatic u(rho)

    for i in (1, 2, 40, 77):
        for ax in range(3):
            Pp, Pm, dx = _displaced(P, i, ax, 1e-4)
            fd = -(U(Pp) - U(Pm)) / dx / m[i]
            assert abs(fd - a[i, ax]) < 1e-5 * np.linalg.norm(a[i]) + 1e-9, (i, ax, fd, a[i, ax])


def test_sph_dudt_is_adiabatic_rate():
    P, m, u0, v = _gas(33)
    # positions on a 2^-12 grid and velocities on a 2^-8 grid so that x +- v dt is exact in float32
    P = np.round(P * 4096) / 4096
    v = np.round(v * 256) / 256
    g = SPH.gamma
    base = oracle.force_step(_wl(P, m, len(m), v=v, u=u0, params=SPH))
    rho0 = base["rho"]
    dt = 2.0 ** -14
    rp = _rho(P + v * dt, m)
    rm = _rho(P - v * dt, m)
    fd = u0 * ((rp / rho0) ** (g - 1) - (rm / rho0) ** (g - 1)) / (2 * dt)
    scale = np.abs(fd).max()
    assert np.max(np.abs(fd - base["dudt"])) < 1e-5 * scale


def test_grad_h_terms_matter():
    # With the variable-mass factors removed (zeta = 0, Omega* = 1) the energy check fails.
    P, m, u0, _ = _gas(31)
    base = oracle.force_step(_wl(P, m, len(m), u=u0, params=SPH))
    st = dict(base["state"])
    st["zeta"] = np.zeros_like(st["zeta"])
    st["omega"] = np.ones_like(st["omega"])
    bad = oracle.force_step(_wl(P, m, len(m), u=u0, params=SPH), fixed_lengths=st)
    i = 40
    assert abs(bad["ax"][i] - base["ax"][i]) > 1e-3 * abs(base["ax"][i])


def test_sph_conservation_with_viscosity_and_tc_gradient():
    P, m, u0, v = _gas(34, n=200)
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=32.0, leaf_size=4,
                 use_tc_gradient=1, alpha=1.0, beta=2.0)
    r = oracle.force_step(_wl(P, m, len(m), v=v, u=u0, params=p))
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    mom = (m[:, None] * a).sum(0)
    assert np.all(np.abs(mom) < 1e-13 * (m[:, None] * np.abs(a)).sum())
    e = m * ((v * a).sum(1) + r["dudt"])
    assert abs(e.sum()) < 1e-13 * np.abs(m * (v * a).sum(1)).sum()
    assert r["nsph"].sum() > 0


def test_viscous_heating_positive_in_compression():
    # cold gas (P = 0) in homologous collapse v = -x: only viscosity acts; it heats.
    rng = np.random.default_rng(35)
    n = 200
    P = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32).astype(np.float64)
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=32.0, leaf_size=4, alpha=1.0, beta=2.0)
    r = oracle.force_step(_wl(P, np.full(n, 1.0 / n), n, v=-P, u=np.full(n, 1e-8), params=p))
    assert np.all(r["dudt"] >= -1e-12) and r["dudt"].sum() > 0
    # and the viscous force decelerates the collapse (points outward on average)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    assert (a * P).sum() > 0


def test_gravity_direct_sum_conserves_momentum():
    P, m = _mixed_cloud(150, 41)
    r = oracle.force_step(_wl(P, m, 0, params=GRAV))
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    assert np.all(np.abs((m[:, None] * a).sum(0)) < 1e-13 * (m[:, None] * np.abs(a)).sum())


def test_two_distant_particles_newtonian():
    P = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    m = np.array([2.0, 0.5])
    p = W.Params(theta=0.5, sph=0, adaptive_softening=0, leaf_size=1)
    r = oracle.force_step(_wl(P, m, 0, params=p, eps=np.full(2, 0.01)))
    # |a_0| = G m_1 / d^2 towards particle 1, d = 5
    assert np.allclose([r["ax"][0], r["ay"][0]], 0.5 / 25 * np.array([0.6, 0.8]), rtol=1e-14)
    assert np.allclose([r["ax"][1], r["ay"][1]], -2.0 / 25 * np.array([0.6, 0.8]), rtol=1e-14)


def test_tree_converges_to_direct_sum_as_theta_decreases():
    w = W.evrard_sphere(2048, seed=7)
    idx = W.sample_indices(w.n, 256)
    ex = oracle.force_step(w, params=W.Params(theta=0.0, leaf_size=8), idx=idx)
    errs = []
    for th in (0.8, 0.5, 0.3):
        r = oracle.force_step(w, params=W.Params(theta=th, leaf_size=8), idx=idx)
        da = np.sqrt((r["ax"] - ex["ax"]) ** 2 + (r["ay"] - ex["ay"]) ** 2 + (r["az"] - ex["az"]) ** 2)[idx]
        aa = np.sqrt(ex["ax"] ** 2 + ex["ay"] ** 2 + ex["az"] ** 2)[idx]
        errs.append(np.median(da / aa))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 3e-3        # quadrupole tree at theta = 0.5


def _radial_profile(P, a, pot, bins):
    r = np.linalg.norm(P, axis=1)
    ar = (a * P).sum(1) / r
    out = []
    for lo, hi in zip(bins[:-1], bins[1:]):
        s = (r >= lo) & (r < hi)
        out.append((0.5 * (lo + hi), ar[s].mean(), pot[s].mean(), s.sum(), r[s]))
    return out


def test_plummer_closed_form():
    w = W.plummer(1 << 14, seed=2, theta=0.5, params=W.Params(theta=0.5, sph=0, n_nei_grav=32.0, leaf_size=8))
    r = oracle.force_step(w)
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    for _, ar, pot, cnt, rs in _radial_profile(P, a, r["pot"], np.array([0.2, 0.4, 0.7, 1.0, 1.5, 2.5, 4.0])):
        # textbook Plummer (G = M = a = 1): a_r = -r (1 + r^2)^{-3/2}, Phi = -(1 + r^2)^{-1/2}
        an = np.mean(-rs * (1 + rs ** 2) ** -1.5)
        pn = np.mean(-(1 + rs ** 2) ** -0.5)
        assert abs(ar - an) < 0.04 * abs(an) + 3.0 / np.sqrt(cnt) * abs(an), (rs.mean(), ar, an)
        assert abs(pot - pn) < 0.01 * abs(pn), (rs.mean(), pot, pn)


def test_one_over_r_sphere_closed_form():
    # rho ~ 1/r in R = 1 with M = 1: M(<r) = r^2, so a_r = -1 inside the sphere.
    w = W.evrard_sphere(1 << 14, seed=8)
    r = oracle.force_step(w, params=W.Params(theta=0.5, gravity=1, sph=0, leaf_size=8))
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    for rc, ar, _, cnt, _ in _radial_profile(P, a, r["pot"], np.array([0.25, 0.4, 0.55, 0.7, 0.85])):
        assert abs(ar + 1.0) < 0.03 + 3.0 / np.sqrt(cnt), (rc, ar)


def test_uniform_periodic_lattice_density():
    k = 16
    g = (np.arange(k) + 0.5) / k
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    n = P.shape[0]
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=50.0, leaf_size=8,
                 periodic_mask=0b111, periodic_lo=(0, 0, 0), periodic_hi=(1, 1, 1))
    r = oracle.force_step(_wl(P, np.full(n, 1.0 / n), n, u=np.ones(n), params=p, h=np.full(n, 1.2 / k)))
    assert np.max(np.abs(r["rho"] - 1.0)) < 1e-2
    # symmetric lattice: no net pressure force on any particle
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    assert np.abs(a).max() < 1e-9


def test_length_solve_satisfies_defining_relations():
    w = W.evrard_sphere(1024, seed=9)
    t = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, 8)
    h, n, rho, om, zeta = t.solve_lengths(0, 50.0, guess=w.h)
    eta = oracle.eta_from_nnei(50.0)
    # Eq. hn: h = eta n^{-1/3}
    assert np.allclose(h ** 3 * n, eta ** 3, rtol=1e-11)
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    m = w.m.astype(np.float64)
    for i in (0, 100, 777):
        d = np.linalg.norm(P - P[i], axis=1)
        nsum = lambda hh: K.W(d, np.full_like(d, hh)).sum()
        # Eq. densitySPH with the self term
        assert np.isclose(rho[i], (m * K.W(d, np.full_like(d, h[i]))).sum(), rtol=1e-12)
        dh = 1e-6 * h[i]
        dn = (nsum(h[i] + dh) - nsum(h[i] - dh)) / (2 * dh)
        # Omega* = 1 - (dh/dn) sum dW/dh with dh/dn = -h/(3n)
        assert np.isclose(om[i], 1 + h[i] / (3 * n[i]) * dn, rtol=1e-7)
    # equal masses: 1 + zeta/(m Omega*) = 1/Omega* (Sect. 3: reduction to the standard equations)
    assert np.allclose(1 + zeta / (m * om), 1 / om, rtol=1e-12)


def test_length_solve_independent_of_guess_and_fails_without_root():
    w = W.evrard_sphere(512, seed=10)
    t = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, 4)
    h1 = t.solve_lengths(0, 50.0, guess=w.h)[0]
    h2 = t.solve_lengths(0, 50.0, guess=w.h * 7.0)[0]
    assert np.allclose(h1, h2, rtol=1e-12)
    # 4 particles cannot hold 50 kernel-weighted neighbours: F(h) < 0 for every h
    t4 = oracle.OracleTree(w.x[:4], w.y[:4], w.z[:4], w.m[:4], 4, 1)
    with pytest.raises(RuntimeError):
        t4.solve_lengths(0, 50.0)


# ---- Monaghan viscosity (Sect. 3.3.1, Eq. mu_visc) ----------------------------------------------
# Two gas particles on the x axis approach head-on with speed s; the pressure is switched off
# (P = 0 in the force pass's state) so that only the viscosity acts.  With v_ij . r_ij = -s r the
# paper's Pi_ij = (-alpha cbar mu + beta mu^2) / rhobar, mu = hbar v_ij.r_ij / (r^2 + eta^2),
# eta^2 = 0.01 hbar^2, makes the acceleration of particle i a quadratic a(s) = A s + B s^2 whose
# kernel-gradient factor cancels in B/A = beta kappa / (alpha cbar), kappa = hbar r / (r^2 + eta^2).
# From two speeds the tests recover eta^2 and the means independently of the kernel gradient.
_VR = 0.375                 # separation (exact in float32)


def _visc_pair(s, h=(0.25, 0.3125), c=(0.5, 1.5), rho=(1.0, 3.0), m=(0.5, 0.75), alpha=1.0, beta=2.0):
    P = np.array([[0.5 * _VR, 0.0, 0.0], [-0.5 * _VR, 0.0, 0.0]])
    v = np.array([[-0.5 * s, 0.0, 0.0], [0.5 * s, 0.0, 0.0]])
    p = W.Params(theta=0.5, gravity=0, sph=1, adaptive_softening=0, leaf_size=1, alpha=alpha, beta=beta)
    w = _wl(P, np.asarray(m, np.float64), 2, v=v, u=np.full(2, 1.0), params=p, h=np.asarray(h))
    st = dict(h=np.asarray(h, np.float64), rho=np.asarray(rho, np.float64), P=np.zeros(2),
              c=np.asarray(c, np.float64), omega=np.ones(2), zeta=np.zeros(2))
    r = oracle.force_step(w, params=p, fixed_lengths=st)
    return r["ax"][0], r["dudt"][0]


def _quadratic_coeffs(**kw):
    a1, _ = _visc_pair(1.0, **kw)
    a2, _ = _visc_pair(2.0, **kw)
    B = 0.5 * (a2 - 2.0 * a1)
    return a1 - B, B


def test_viscosity_softening_constant_and_means():
    h, c = (0.25, 0.3125), (0.5, 1.5)
    A, B = _quadratic_coeffs(h=h, c=c)
    alpha, beta = 1.0, 2.0
    hbar, cbar = 0.5 * (h[0] + h[1]), 0.5 * (c[0] + c[1])      # arithmetic means of Sect. 3.3.1
    kappa = (B / A) * alpha * cbar / beta
    eta2 = hbar * _VR / kappa - _VR ** 2
    # eta = 0.1 h (Sect. 3.3.1): eta^2 = 0.01 hbar^2; 0.1 hbar^2, a geometric hbar or a cbar taken
    # as max(c_i, c_j) give 0.05, 0.0100-0.0011 shifted, or a 40 % larger kappa respectively
    assert abs(eta2 / hbar ** 2 - 0.01) < 1e-9, eta2 / hbar ** 2
    # the viscous force pushes the approaching particle back (i sits at +x)
    assert A > 0 and B > 0


def test_viscosity_density_mean_is_arithmetic():
    a13, _ = _visc_pair(1.0, rho=(1.0, 3.0))
    a22, _ = _visc_pair(1.0, rho=(2.0, 2.0))
    a11, _ = _visc_pair(1.0, rho=(1.0, 1.0))
    # same arithmetic mean -> same force (a geometric mean would differ by 2/sqrt(3), a harmonic by 4/3)
    assert abs(a13 - a22) <= 1e-14 * abs(a22)
    # Pi ~ 1/rhobar
    assert abs(a11 / a22 - 2.0) < 1e-13


def test_viscosity_sound_speed_mean_is_arithmetic():
    # alpha term only: a ~ cbar, so (c_i, c_j) = (0.5, 1.5) and (1, 1) agree; max(c) would not
    a1, _ = _visc_pair(1.0, c=(0.5, 1.5), beta=0.0)
    a2, _ = _visc_pair(1.0, c=(1.0, 1.0), beta=0.0)
    assert abs(a1 - a2) <= 1e-14 * abs(a2)


def test_viscous_heating_is_half_the_pair_work():
    # du_i/dt = 1/2 m_j Pi_ij v_ij . gradbar W = -1/2 v_ij . a_i(visc): each particle of the pair
    # receives half of the kinetic energy the viscous pair force removes (Eq. thermalvarmass1)
    for s in (0.5, 1.0, 3.0):
        a, du = _visc_pair(s)
        assert abs(du - 0.5 * s * a) <= 1e-13 * abs(du), (s, a, du)
        assert du > 0


def test_viscosity_off_for_receding_pairs():
    a, du = _visc_pair(-1.0)
    assert a == 0.0 and du == 0.0
