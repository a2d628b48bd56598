"""Pins of the oracle's dissipation variants (Sect. 3.3.3): the signal-velocity viscosity, the
Balsara limiter with the curl of v it needs, the per-particle alpha with its switch, and the
artificial conductivity with Brookshaw's Laplacian.

What fixes each value, independently of the oracle's own formulas:

* Curl and divergence of a linear velocity field from one neighbour sum.  With g = dW/dr / r the
  identity r dW/dr = -3 W - h dW/dh makes sum_j r_ij^2 g = -3 n Omega* for any particle set, and a
  cubic lattice makes the second moment sum_j g x_a x_b isotropic at a particle whose whole
  neighbourhood is lattice.  There a rigid rotation v = w x r has |curl v| = 2 |w| and div v = 0, a
  shear v = (k y, 0, 0) has |curl v| = |k|, and a homologous flow v = k r has curl v = 0 anywhere.
* Brookshaw's Laplacian at such a particle, equal masses, exact kernel gradient: for u = x^2 the
  sum is exactly -2 (the printed form uses |grad W|, so it carries the opposite sign of the true
  Laplacian, 2; the source term takes its modulus), for a linear u exactly 0.  The grad-h factor
  (1 + zeta/(m Omega*)) times Omega* is 1 for equal masses, which makes the value exact.
* A head-on pair: the signal-velocity viscosity is quadratic in the approach speed s with the
  ratio of its s^2 and s coefficients 1/(c_i + c_j) (v^sig = 2 cbar - w, w = -s), linear in alpha
  and free of beta; it heats each particle by half the pair work, and is off for receding pairs.
* Static uniform gas: v^sig = 2c, div v = 0, so alpha decays at exactly (alpha - alpha_min) 2c /
  (0.1 h).  Compression with alpha = alpha_min: the decay term vanishes and the source is
  0.75 f 3|k| with f = 1 when the limiter's eta is 0 and the flow has no curl.
* The conductivity moves heat between the particles of each pair only: sum_i m_i du_i/dt = 0, heat
  flows from hot to cold, its pressure-jump signal speed vanishes for equal pressures and scales
  as the square root of the jump.
* Everything on at once still conserves momentum and total energy pairwise.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W

GAMMA = 5.0 / 3.0


def _wl(P, m, v=None, u=None, h=None, params=None, alpha=None, alpha_u=None):
    n = len(m)
    f = lambda a: np.ascontiguousarray(a, np.float32)
    v = np.zeros((n, 3)) if v is None else v
    u = np.ones(n) if u is None else u
    h = np.full(n, 0.1) if h is None else h
    w = W.Workload("t", f(P[:, 0]), f(P[:, 1]), f(P[:, 2]), f(v[:, 0]), f(v[:, 1]), f(v[:, 2]), f(m), f(u),
                   f(h), f(h), n_gas=n, params=params or W.Params())
    w.alpha = None if alpha is None else f(alpha)
    w.alpha_u = None if alpha_u is None else f(alpha_u)
    return w


def _params(**kw):
    base = dict(theta=0.5, gravity=0, sph=1, adaptive_softening=0, n_nei_sph=50.0, leaf_size=8, alpha=1.0,
                beta=2.0)
    base.update(kw)
    return W.Params(**base)


NX = 16


def _lattice(nx=NX):
    g = (np.arange(nx) + 0.5) / nx                       # exact in float32
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    k = np.stack(np.meshgrid(*(np.arange(nx),) * 3, indexing="ij"), -1).reshape(-1, 3)
    # particles whose neighbours' neighbourhoods are whole lattice (2h is about 2.3 spacings)
    interior = np.all((k >= 5) & (k <= nx - 6), axis=1)
    return P, interior


def _lattice_run(v=None, u=None, alpha=None, alpha_u=None, **kw):
    P, inner = _lattice()
    n = len(P)
    h = np.full(n, 1.15 / NX)
    w = _wl(P, np.full(n, 1.0 / n), v=v, u=u, h=h, params=_params(**kw), alpha=alpha, alpha_u=alpha_u)
    return oracle.force_step(w), P, inner, w


# ---- curl and divergence --------------------------------------------------------------------

def test_curl_of_rigid_rotation_on_a_lattice():
    P, _ = _lattice()
    omega = np.array([0.5, -0.25, 1.0])                  # dyadic: w x r is exact in float32
    r, P, inner, _ = _lattice_run(v=np.cross(omega, P))
    assert np.allclose(r["curlv_h"][inner], 2 * np.linalg.norm(omega), rtol=1e-10, atol=0)
    assert np.abs(r["divv_h"][inner]).max() < 1e-10


def test_curl_of_shear_on_a_lattice():
    P, _ = _lattice()
    k = 0.75
    v = np.zeros_like(P)
    v[:, 0] = k * P[:, 1]
    r, P, inner, _ = _lattice_run(v=v)
    assert np.allclose(r["curlv_h"][inner], k, rtol=1e-10, atol=0)
    assert np.abs(r["divv_h"][inner]).max() < 1e-10


def test_curl_of_homologous_flow_vanishes():
    w = W.evrard_sphere(1200, seed=41)
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    k = -0.75
    w.vx[:], w.vy[:], w.vz[:] = (np.asarray(k * P[:, a], np.float32) for a in range(3))
    r = oracle.force_step(w)
    assert np.abs(r["curlv_h"]).max() < 1e-5 * 3 * abs(k)
    assert np.allclose(r["divv_h"], 3 * k, rtol=2e-6)


# ---- Balsara limiter --------------------------------------------------------------------------

def test_balsara_factor_is_one_in_pure_compression():
    w = W.with_dissipation(W.evrard_sphere(1200, seed=42), seed=1, balsara=1, balsara_eta=0.0)
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    w.vx[:], w.vy[:], w.vz[:] = (np.asarray(-1.25 * P[:, a], np.float32) for a in range(3))
    r = oracle.force_step(w)
    assert np.allclose(r["balsara_f"], 1.0, atol=1e-5)
    # and the limited viscosity is then the plain one (f_bar = 1)
    plain = oracle.force_step(W.with_dissipation(w, seed=1, balsara=0, balsara_eta=0.0, u_spread=0.0))
    for k in ("ax", "dudt"):
        assert np.allclose(r[k], plain[k], rtol=1e-4, atol=1e-6 * np.abs(plain[k]).max())
    # with eta_B > 0 the sound-speed term of the denominator: f = 3|k| / (3|k| + eta_B c / h)
    e = oracle.force_step(W.with_dissipation(w, seed=1, balsara=1, balsara_eta=0.5, u_spread=0.0))
    ng = w.n_gas
    expect = 3 * 1.25 / (3 * 1.25 + 0.5 * e["c"][:ng] / e["h"][:ng])
    assert np.allclose(e["balsara_f"][:ng], expect, rtol=1e-5)
    assert expect.min() < 0.9


def test_balsara_switches_viscosity_off_in_shear():
    P, _ = _lattice()
    v = np.zeros_like(P)
    v[:, 0] = 0.75 * P[:, 1]
    on, _, inner, _ = _lattice_run(v=v, balsara=1)
    off, _, _, _ = _lattice_run(v=v, balsara=0)
    assert np.abs(on["balsara_f"][inner]).max() < 1e-9
    # without the limiter the shear heats (viscous heating of approaching pairs; the net viscous
    # force cancels on the lattice either way); with it the interior particles, whose neighbours
    # all have f = 0, are not heated
    assert off["dudt"][inner].min() > 0
    assert np.abs(on["dudt"][inner]).max() < 1e-8 * off["dudt"][inner].min()


# ---- signal-velocity viscosity (Eqs. pvsig, vsig) on a head-on pair --------------------------------

_VR = 0.375


def _pair(s, c=(0.5, 1.5), rho=(1.0, 3.0), m=(0.5, 0.75), h=(0.25, 0.3125), form=1, alpha=1.0, beta=2.0,
          alphas=None, u=(1.0, 1.0), P=(0.0, 0.0), alpha_u=None, conduction=0, cond_vsig=0):
    Ppos = np.array([[0.5 * _VR, 0.0, 0.0], [-0.5 * _VR, 0.0, 0.0]])
    v = np.array([[-0.5 * s, 0.0, 0.0], [0.5 * s, 0.0, 0.0]])
    p = _params(visc_form=form, alpha=alpha, beta=beta, leaf_size=1, variable_alpha=int(alphas is not None),
                conduction=conduction, cond_vsig=cond_vsig)
    w = _wl(Ppos, np.asarray(m, np.float64), v=v, u=np.asarray(u), h=np.asarray(h), params=p, alpha=alphas,
            alpha_u=alpha_u)
    st = dict(h=np.asarray(h, np.float64), rho=np.asarray(rho, np.float64), P=np.asarray(P, np.float64),
              c=np.asarray(c, np.float64), omega=np.ones(2), zeta=np.zeros(2))
    r = oracle.force_step(w, params=p, fixed_lengths=st)
    return r["ax"][0], r["dudt"][0], r


def test_signal_velocity_viscosity_coefficients():
    c = (0.5, 1.5)
    a1, _, _ = _pair(1.0, c=c)
    a2, _, _ = _pair(2.0, c=c)
    B = 0.5 * (a2 - 2.0 * a1)
    A = a1 - B
    # Pi = alpha (c_i + c_j + s) s / rhobar: s^2 / s coefficient ratio 1 / (c_i + c_j); a form with
    # cbar in place of 2 cbar, or without the -w term, gives 2 / (c_i + c_j) or 0
    assert abs(B / A * (c[0] + c[1]) - 1.0) < 1e-12
    assert A > 0 and B > 0            # pushes the approaching particle (at +x) back


def test_signal_velocity_against_the_monaghan_form():
    # linear (alpha) terms of the two forms for the same pair: -2 alpha cbar w / rhobar against
    # -alpha cbar mu / rhobar with mu = hbar w r / (r^2 + 0.01 hbar^2), so their ratio is
    # 2 (r^2 + 0.01 hbar^2) / (hbar r) whatever the kernel gradient and the masses
    h = (0.25, 0.3125)
    hb = 0.5 * (h[0] + h[1])

    def lin(form):
        a1, _, _ = _pair(1.0, form=form, beta=0.0, h=h)
        a2, _, _ = _pair(2.0, form=form, beta=0.0, h=h)
        return a1 - 0.5 * (a2 - 2.0 * a1)

    ratio = lin(1) / lin(0)
    assert abs(ratio / (2 * (_VR ** 2 + 0.01 * hb * hb) / (hb * _VR)) - 1.0) < 1e-12


def test_signal_velocity_viscosity_is_linear_in_alpha_and_free_of_beta():
    a1, _, _ = _pair(1.5, alpha=1.0, beta=2.0)
    a2, _, _ = _pair(1.5, alpha=2.0, beta=0.0)
    a3, _, _ = _pair(1.5, alpha=2.0, beta=7.0)
    assert abs(a2 / a1 - 2.0) < 1e-14
    assert a2 == a3


def test_signal_velocity_heating_is_half_the_pair_work_and_off_when_receding():
    for s in (0.5, 1.0, 3.0):
        a, du, _ = _pair(s)
        assert abs(du - 0.5 * s * a) <= 1e-13 * abs(du) and du > 0
    a, du, _ = _pair(-1.0)
    assert a == 0.0 and du == 0.0


def test_pair_alpha_is_the_arithmetic_mean():
    a1, _, _ = _pair(1.0, alphas=(0.5, 1.5))
    a2, _, _ = _pair(1.0, alphas=(1.0, 1.0))
    a3, _, _ = _pair(1.0, alphas=(2.0, 2.0))
    assert abs(a1 - a2) <= 1e-14 * abs(a2)
    assert abs(a3 / a2 - 2.0) < 1e-14
    # the Monaghan form takes the same mean in its alpha term
    m1, _, _ = _pair(1.0, alphas=(0.5, 1.5), form=0, beta=0.0)
    m2, _, _ = _pair(1.0, alphas=(1.0, 1.0), form=0, beta=0.0)
    assert abs(m1 - m2) <= 1e-14 * abs(m2)


def test_signal_velocity_of_a_pair():
    c = (0.5, 1.5)
    _, _, r = _pair(2.0, c=c)
    assert np.allclose(r["vsig"], c[0] + c[1] + 2.0, rtol=1e-15)
    _, _, r = _pair(-2.0, c=c)                 # receding: c_i + c_j, or the self pair's 2 c_i
    assert np.allclose(r["vsig"], [2.0, 3.0], rtol=1e-15)


# ---- per-particle alpha (Eq. alphaswitch) -----------------------------------------------------------

def test_alpha_decay_of_static_uniform_gas():
    P, _ = _lattice()
    n = len(P)
    rng = np.random.default_rng(43)
    alpha = rng.uniform(0.05, 1.5, n).astype(np.float32)
    u = 0.7
    r, _, inner, w = _lattice_run(u=np.full(n, u), alpha=alpha, variable_alpha=1, alpha_min=0.01, alpha_tau=0.1)
    c = np.sqrt(GAMMA * (GAMMA - 1.0) * np.float64(np.float32(u)))
    h = r["h"][inner]
    assert np.allclose(r["vsig"][inner], 2 * c, rtol=1e-14)
    expect = -(alpha[inner].astype(np.float64) - 0.01) * 2 * c / (0.1 * h)
    assert np.allclose(r["dalpha"][inner], expect, rtol=1e-9)


@pytest.mark.parametrize("k", [-1.25, 0.5])
def test_alpha_source_in_compression_only(k):
    w = W.evrard_sphere(1200, seed=44)
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    w.vx[:], w.vy[:], w.vz[:] = (np.asarray(k * P[:, a], np.float32) for a in range(3))
    w = W.with_dissipation(w, seed=2, alpha=(0.01, 0.01), u_spread=0.0, variable_alpha=1, alpha_min=float(np.float32(0.01)),
                           balsara_eta=0.0)
    r = oracle.force_step(w)
    expect = 0.75 * 3 * abs(k) if k < 0 else 0.0
    assert np.allclose(r["dalpha"], expect, rtol=1e-5, atol=1e-12)


# ---- artificial conductivity ------------------------------------------------------------------------

def _cloud(seed, n=200):
    rng = np.random.default_rng(seed)
    P = rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32).astype(np.float64)
    m = (np.where(np.arange(n) % 3 == 0, 2.5, 1.0) / n).astype(np.float32).astype(np.float64)
    u = rng.uniform(0.5, 1.5, n)
    v = rng.normal(0, 0.3, (n, 3)).astype(np.float32).astype(np.float64)
    alpha = rng.uniform(0.1, 1.5, n)
    alpha_u = rng.uniform(0.0, 1.0, n)
    return P, m, u, v, alpha, alpha_u


@pytest.mark.parametrize("cond_vsig", [0, 1])
def test_conduction_conserves_thermal_energy(cond_vsig):
    P, m, u, _, alpha, alpha_u = _cloud(45)
    p = _params(n_nei_sph=32.0, leaf_size=4, conduction=1, cond_vsig=cond_vsig)
    r = oracle.force_step(_wl(P, m, u=u, params=p, alpha_u=alpha_u))     # at rest: conduction only
    du = m * r["dudt"]
    assert np.abs(du).sum() > 0
    assert abs(du.sum()) < 1e-13 * np.abs(du).sum()


def test_conduction_moves_heat_from_hot_to_cold():
    P, _ = _lattice()
    n = len(P)
    hot = P[:, 0] < 0.5
    u = np.where(hot, 2.0, 1.0)
    r, _, _, _ = _lattice_run(u=u, alpha_u=np.full(n, 0.5), conduction=1)
    du = r["dudt"]
    assert np.all(du[hot] <= 0) and np.all(du[~hot] >= 0)
    assert du[hot].min() < 0 and du[~hot].max() > 0


def test_brookshaw_laplacian_on_a_lattice():
    P, _ = _lattice()
    n = len(P)
    quad, _, inner, _ = _lattice_run(u=1.0 + P[:, 0] ** 2, alpha_u=np.zeros(n), conduction=1, use_tc_gradient=0,
                                     alpha_u_min=0.0)
    assert np.allclose(quad["lapu"][inner], -2.0, rtol=1e-7)
    lin, _, _, _ = _lattice_run(u=1.0 + P[:, 1], alpha_u=np.zeros(n), conduction=1, use_tc_gradient=0)
    assert np.abs(lin["lapu"][inner]).max() < 1e-7
    # the conductivity switch's source with alpha^u at its floor: h |lap u| / sqrt(u), or 0.1 h |lap u|
    u_in = np.float32(1.0) + (P[:, 0] ** 2).astype(np.float32)
    h = quad["h"][inner]
    assert np.allclose(quad["dalpha_u"][inner], 2.0 * h / np.sqrt(u_in[inner].astype(np.float64)), rtol=1e-6)
    q05, _, _, _ = _lattice_run(u=1.0 + P[:, 0] ** 2, alpha_u=np.zeros(n), conduction=1, use_tc_gradient=0,
                                cond_source=1)
    assert np.allclose(q05["dalpha_u"][inner], 0.2 * h, rtol=1e-6)


def test_brookshaw_laplacian_uses_the_neighbour_density():
    # sum_j 2 m_j (u_i - u_j) / rho_j |gradbar W| / r: particle 0's value depends on rho_1 alone,
    # inversely (a pair mean of the densities would depend on rho_0 too)
    kw = dict(u=(2.0, 1.0), alpha_u=(0.5, 0.5), conduction=1)
    _, _, r13 = _pair(0.0, rho=(1.0, 3.0), **kw)
    _, _, r23 = _pair(0.0, rho=(2.0, 3.0), **kw)
    _, _, r115 = _pair(0.0, rho=(1.0, 1.5), **kw)
    assert r13["lapu"][0] == r23["lapu"][0] and r13["lapu"][0] > 0
    assert abs(r115["lapu"][0] / r13["lapu"][0] - 2.0) < 1e-14


@pytest.mark.parametrize("cond_vsig", [0, 1])
def test_conduction_against_the_laplacian(cond_vsig):
    # for a pair at rest with rho_i = rho_j: du_i/dt = -alphabar^u v^u (u_i - u_j)/rho m_j |gradbar W|
    # and lap u_i = 2 m_j (u_i - u_j)/rho |gradbar W| / r, so du_i/dt = -alphabar^u v^u r lap u_i / 2;
    # the Laplacian's scale is fixed by the lattice pin above.  v^u is c_i + c_j at rest (Eq. vsig)
    # or sqrt(|P_i - P_j| / rhobar) = 1 here.
    c = (0.5, 1.5)
    _, du, r = _pair(0.0, c=c, rho=(1.0, 1.0), P=(0.5, 1.5), u=(2.0, 1.0), alpha_u=(0.25, 0.75), conduction=1,
                     cond_vsig=cond_vsig)
    vu = c[0] + c[1] if cond_vsig == 0 else 1.0
    assert abs(du / (-0.5 * vu * _VR * r["lapu"][0] / 2) - 1.0) < 1e-14


def test_pressure_jump_signal_speed():
    kw = dict(u=(2.0, 1.0), alpha_u=(0.5, 0.5), conduction=1, cond_vsig=1, form=1)
    _, du0, _ = _pair(0.0, P=(0.5, 0.5), **kw)
    assert du0 == 0.0                                   # equal pressures: no conduction
    _, du1, _ = _pair(0.0, P=(0.5, 0.75), **kw)
    _, du4, _ = _pair(0.0, P=(0.5, 1.5), **kw)
    _, du4r, _ = _pair(0.0, P=(1.5, 0.5), **kw)
    assert du1 < 0                                      # the hotter particle cools
    assert abs(du4 / du1 - 2.0) < 1e-14                 # sqrt of the pressure jump
    assert du4 == du4r                                  # of its magnitude
    # the mean alpha^u of the pair is arithmetic
    _, dua, _ = _pair(0.0, P=(0.5, 1.5), u=(2.0, 1.0), alpha_u=(0.25, 0.75), conduction=1, cond_vsig=1)
    assert abs(dua - du4) <= 1e-14 * abs(du4)


# ---- all variants at once ---------------------------------------------------------------------------

def test_all_variants_conserve_momentum_and_energy():
    P, m, u, v, alpha, alpha_u = _cloud(46)
    p = _params(n_nei_sph=32.0, leaf_size=4, use_tc_gradient=1, visc_form=1, balsara=1, variable_alpha=1,
                conduction=1)
    r = oracle.force_step(_wl(P, m, v=v, u=u, params=p, alpha=alpha, alpha_u=alpha_u))
    a = np.stack([r["ax"], r["ay"], r["az"]], 1)
    mom = (m[:, None] * a).sum(0)
    assert np.all(np.abs(mom) < 1e-13 * (m[:, None] * np.abs(a)).sum())
    e = m * ((v * a).sum(1) + r["dudt"])
    assert abs(e.sum()) < 1e-13 * np.abs(m * (v * a).sum(1)).sum()
    assert np.all(np.isfinite(r["dalpha"])) and np.all(np.isfinite(r["dalpha_u"]))


def test_switches_integrated_by_the_kicks():
    # static periodic lattice: no forces, du/dt = 0, div v = 0, lap u = 0; each switch decays as
    # d(a - a_min)/dt = -k (a - a_min), k = 2c / (0.1 h).  The kicks use the rate of the last force
    # step, as for u.  With x = k dt/2, the value handed to the first force step is (1 - x) of the
    # start, each later one (1 - 2x) of the one before, and a step ends at (1 - x) of its force
    # step's value: after N steps a - a_min is (1 - x)^2 (1 - 2x)^(N-1) of its start.
    nx = 8
    g = (np.arange(nx) + 0.5) / nx
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    n = len(P)
    rng = np.random.default_rng(47)
    alpha = rng.uniform(0.1, 1.5, n).astype(np.float32)
    alpha_u = rng.uniform(0.0, 1.0, n).astype(np.float32)
    p = _params(n_nei_sph=40.0, periodic_mask=7, periodic_lo=(0, 0, 0), periodic_hi=(1, 1, 1), variable_alpha=1,
                conduction=1, alpha_min=0.0625, alpha_u_min=0.0)
    w = _wl(P, np.full(n, 1.0 / n), u=np.full(n, 0.7), h=np.full(n, 1.2 / nx), params=p, alpha=alpha,
            alpha_u=alpha_u)
    r0 = oracle.force_step(w)
    k = r0["vsig"] / (0.1 * r0["h"])
    assert np.allclose(k, k[0], rtol=1e-12)
    dt = 0.2 / k[0]                        # k dt / 2 = 0.1
    res = oracle.kdk(w, dt, 3)
    f = (1.0 - 0.1) ** 2 * (1.0 - 0.2) ** 2
    assert np.allclose(res["alpha"] - 0.0625, (alpha.astype(np.float64) - 0.0625) * f, rtol=1e-6, atol=0)
    assert np.allclose(res["alpha_u"], alpha_u.astype(np.float64) * f, rtol=1e-6, atol=0)
