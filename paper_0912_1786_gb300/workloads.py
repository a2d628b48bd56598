"""Seeded synthetic particle sets shaped like the paper's test problems.

This module holds only input generation: positions, velocities, masses, internal energies
and starting guesses for the smoothing/softening lengths.  It contains none of the force
step's arithmetic, and it is the one module shared by the CUDA path's tests/benchmark and
the FP64 oracle.  Every array is float32 in the caller's (unsorted) order; gas particles are
the first ``n_gas`` entries.

Shapes (Sect. 5 of the paper):
  * ``evrard_sphere``  -- rho ~ 1/r gas sphere of radius 1, cold (u = 0.05), the adiabatic
    collapse set-up (Sect. 5.8.2, Evrard test).
  * ``plummer``        -- Plummer sphere with isotropic velocities from its distribution function
    (Sect. 5.10, collision of two Plummer spheres).
  * ``hernquist_gas``  -- Hernquist dark-matter halo plus a rho ~ 1/r gas sphere (Sect. 5.11,
    two-component systems).
  * ``shock_tube``     -- 3-D shock tube slab [0,1] x [0,0.1]^2, periodic in y and z
    (Sect. 5.2.2, 3-D tests), on two jittered cubic lattices in place of the relaxed glass.
  * ``ensemble``       -- many independent cold gas spheres with log-uniform N.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

F32 = np.float32


@dataclass
class Params:
    """Run parameters (Sect. 5 defaults where the paper fixes them)."""

    theta: float = 0.5
    n_nei_sph: float = 50.0
    n_nei_grav: float = 50.0
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    beta: float = 2.0
    G: float = 1.0
    gravity: int = 1
    sph: int = 1
    adaptive_softening: int = 1
    periodic_mask: int = 0
    periodic_lo: tuple = (0.0, 0.0, 0.0)
    periodic_hi: tuple = (1.0, 1.0, 1.0)
    leaf_size: int = 8
    group_size: int = 32
    use_tc_gradient: int = 1
    sph_scheme: int = 0            # 0: n-h (Lagrangian) scheme; 1: standard scheme, N_nei inside 2h
    length_group: int = 0          # particles per group walk of the length solves (0: 8)
    # dissipation variants (Sect. 3.3.3); all off is the standard Monaghan viscosity
    visc_form: int = 0             # 0: Monaghan alpha/beta form; 1: signal-velocity form
    balsara: int = 0               # 1: Balsara limiter on the viscosity
    balsara_eta: float = 1e-4
    variable_alpha: int = 0        # 1: per-particle alpha with its time derivative
    alpha_min: float = 0.01
    alpha_tau: float = 0.1
    alpha_source: float = 0.75
    conduction: int = 0            # 1: artificial conductivity with per-particle alpha^u
    cond_vsig: int = 0             # 0: sound-speed signal velocity; 1: pressure-jump signal velocity
    cond_source: int = 0           # 0: h |lap u| / sqrt(u); 1: 0.1 h |lap u|
    alpha_u_min: float = 0.0


@dataclass
class Workload:
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    m: np.ndarray
    u: np.ndarray
    h: np.ndarray
    eps: np.ndarray
    n_gas: int
    params: Params = field(default_factory=Params)
    sys_offsets: np.ndarray | None = None     # batched ensembles: CSR offsets of the systems
    alpha: np.ndarray | None = None           # per-particle viscosity alpha_i (gas), variable alpha
    alpha_u: np.ndarray | None = None         # per-particle conductivity alpha^u_i (gas)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def arrays(self) -> dict:
        return {k: getattr(self, k) for k in ("x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "eps")}


def _isotropic(rng, n):
    cz = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    sz = np.sqrt(1.0 - cz * cz)
    return sz * np.cos(ph), sz * np.sin(ph), cz


def _length_guess(number_density, n_nei):
    # starting guess only: L = eta n^{-1/3} with 4/3 pi (2 eta)^3 = n_nei
    eta = 0.5 * (3.0 * n_nei / (4.0 * np.pi)) ** (1.0 / 3.0)
    return eta * np.maximum(number_density, 1e-30) ** (-1.0 / 3.0)


def _one_over_r_sphere(rng, n, radius=1.0):
    # rho ~ 1/r inside `radius`: M(<r) ~ r^2, so r = radius * sqrt(U)
    r = radius * np.sqrt(rng.uniform(0.0, 1.0, n))
    ux, uy, uz = _isotropic(rng, n)
    return r * ux, r * uy, r * uz, r


def _f32(*arrs):
    return [np.ascontiguousarray(a, dtype=F32) for a in arrs]


def evrard_sphere(n: int = 4096, seed: int = 1, sigma_v: float = 0.0, mass: float = 1.0,
                  u: float = 0.05, params: Params | None = None) -> Workload:
    """rho ~ 1/r gas sphere of radius 1 and total mass `mass`, all gas."""
    rng = np.random.default_rng(seed)
    x, y, z, r = _one_over_r_sphere(rng, n)
    if sigma_v > 0:
        vx, vy, vz = (rng.normal(0.0, sigma_v, n) for _ in range(3))
    else:
        vx = vy = vz = np.zeros(n)
    m = np.full(n, mass / n)
    # rho(r) = M / (2 pi R^2 r)
    nd = (1.0 / (2.0 * np.pi * np.maximum(r, 1e-3))) * n
    p = params or Params(theta=0.5, n_nei_sph=50.0, n_nei_grav=50.0, leaf_size=8)
    hg = _length_guess(nd, p.n_nei_sph)
    x, y, z, vx, vy, vz, m, uu, h, eps = _f32(x, y, z, vx, vy, vz, m, np.full(n, u), hg, hg)
    return Workload("evrard_sphere", x, y, z, vx, vy, vz, m, uu, h, eps, n_gas=n, params=p)


def plummer(n: int = 1 << 20, seed: int = 2, theta: float = 0.6, rmax: float = 20.0,
            params: Params | None = None) -> Workload:
    """Plummer sphere, M = a = G = 1, collisionless (gravity only)."""
    rng = np.random.default_rng(seed)
    rs = np.empty(0)
    while rs.size < n:
        uu = rng.uniform(0.0, 1.0, 2 * n)
        uu = uu[uu > 0]
        r = 1.0 / np.sqrt(uu ** (-2.0 / 3.0) - 1.0)
        rs = np.concatenate([rs, r[r <= rmax]])
    r = rs[:n]
    ux, uy, uz = _isotropic(rng, n)
    # speeds from the distribution function: q^2 (1 - q^2)^{7/2} by rejection
    q = np.empty(0)
    while q.size < n:
        qq = rng.uniform(0.0, 1.0, 2 * n)
        yy = rng.uniform(0.0, 0.1, 2 * n)
        q = np.concatenate([q, qq[yy < qq * qq * (1.0 - qq * qq) ** 3.5]])
    q = q[:n]
    v = q * np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    vx_, vy_, vz_ = _isotropic(rng, n)
    m = np.full(n, 1.0 / n)
    nd = n * (3.0 / (4.0 * np.pi)) * (1.0 + r * r) ** (-2.5)
    p = params or Params(theta=theta, n_nei_grav=32.0, sph=0, leaf_size=8)
    g = _length_guess(nd, p.n_nei_grav)
    zero = np.zeros(n)
    x, y, z, vx, vy, vz, m, uu, h, eps = _f32(r * ux, r * uy, r * uz, v * vx_, v * vy_, v * vz_, m, zero, g, g)
    return Workload("plummer", x, y, z, vx, vy, vz, m, uu, h, eps, n_gas=0, params=p)


def hernquist_gas(n_dm: int = 1 << 21, n_gas: int = 1 << 20, seed: int = 3, gas_fraction: float = 0.1,
                  rmax: float = 50.0, u: float = 0.05, params: Params | None = None) -> Workload:
    """Hernquist dark-matter halo (M = a = 1) plus a rho ~ 1/r gas sphere of radius 1 whose mass
    is `gas_fraction` of the total.  Gas particles come first."""
    rng = np.random.default_rng(seed)
    xg, yg, zg, rg = _one_over_r_sphere(rng, n_gas)
    rd = np.empty(0)
    while rd.size < n_dm:
        s = np.sqrt(rng.uniform(0.0, 1.0, 2 * n_dm))
        s = s[s < 1.0]
        r = s / (1.0 - s)
        rd = np.concatenate([rd, r[r <= rmax]])
    rd = rd[:n_dm]
    ux, uy, uz = _isotropic(rng, n_dm)
    m_gas = gas_fraction / (1.0 - gas_fraction)
    mg = np.full(n_gas, m_gas / n_gas)
    md = np.full(n_dm, 1.0 / n_dm)
    p = params or Params(theta=0.5, n_nei_sph=50.0, n_nei_grav=50.0, leaf_size=8)
    nd_gas = n_gas / (2.0 * np.pi * np.maximum(rg, 1e-3))
    # Hernquist rho = M a / (2 pi r (r + a)^3)
    nd_dm_at = lambda r: n_dm / (2.0 * np.pi * np.maximum(r, 1e-3) * (r + 1.0) ** 3)
    h = _length_guess(nd_gas, p.n_nei_sph)
    eps = np.concatenate([_length_guess(nd_gas + nd_dm_at(rg), p.n_nei_grav),
                          _length_guess(nd_dm_at(rd), p.n_nei_grav)])
    n = n_gas + n_dm
    zero = np.zeros(n)
    uu = np.concatenate([np.full(n_gas, u), np.zeros(n_dm)])
    hh = np.concatenate([h, eps[n_gas:]])
    x, y, z, vx, vy, vz, m, uu, hh, eps = _f32(
        np.concatenate([xg, rd * ux]), np.concatenate([yg, rd * uy]), np.concatenate([zg, rd * uz]),
        zero, zero, zero, np.concatenate([mg, md]), uu, hh, eps)
    return Workload("hernquist_gas", x, y, z, vx, vy, vz, m, uu, hh, eps, n_gas=n_gas, params=p)


def shock_tube(seed: int = 4, left=(275, 55, 55), right=(175, 35, 35), jitter: float = 0.01,
               rho=(1.0, 0.25), pressure=(1.0, 0.1795), gamma: float = 5.0 / 3.0,
               params: Params | None = None) -> Workload:
    """Two cubic lattices in x<0.5 and x>=0.5 of the box [0,1] x [0,0.1]^2 (y, z periodic).
    Each lattice point is jittered by U(-jitter, jitter) lattice spacings per axis."""
    rng = np.random.default_rng(seed)
    xs, ys, zs, ms, us = [], [], [], [], []
    for side, (nx, ny, nz), rho_s, p_s in ((0, left, rho[0], pressure[0]), (1, right, rho[1], pressure[1])):
        dx = 0.5 / nx
        ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        px = 0.5 * side + (ix.ravel() + 0.5) * dx
        py = (iy.ravel() + 0.5) * (0.1 / ny)
        pz = (iz.ravel() + 0.5) * (0.1 / nz)
        k = px.size
        px = px + rng.uniform(-jitter, jitter, k) * dx
        py = py + rng.uniform(-jitter, jitter, k) * (0.1 / ny)
        pz = pz + rng.uniform(-jitter, jitter, k) * (0.1 / nz)
        xs.append(px); ys.append(np.mod(py, 0.1)); zs.append(np.mod(pz, 0.1))
        ms.append(np.full(k, rho_s * 0.5 * 0.1 * 0.1 / k))
        us.append(np.full(k, p_s / ((gamma - 1.0) * rho_s)))
    x, y, z = (np.concatenate(a) for a in (xs, ys, zs))
    m = np.concatenate(ms)
    u = np.concatenate(us)
    n = x.size
    p = params or Params(theta=0.5, n_nei_sph=50.0, gravity=0, adaptive_softening=0, periodic_mask=0b110,
                         periodic_lo=(0.0, 0.0, 0.0), periodic_hi=(1.0, 0.1, 0.1), leaf_size=8, gamma=gamma)
    nd = np.where(x < 0.5, left[0] * left[1] * left[2] / 0.005, right[0] * right[1] * right[2] / 0.005)
    h = _length_guess(nd, p.n_nei_sph)
    zero = np.zeros(n)
    x, y, z, vx, vy, vz, m, u, h, eps = _f32(x, y, z, zero, zero, zero, m, u, h, h)
    return Workload("shock_tube", x, y, z, vx, vy, vz, m, u, h, eps, n_gas=n, params=p)


def ensemble(nsys: int = 64, seed: int = 5, log2_min: float = 10.0, log2_max: float = 17.0,
             params: Params | None = None) -> Workload:
    """`nsys` independent cold rho ~ 1/r gas spheres (M = R = 1 each), N_k = floor(2^(10 + 7U))."""
    rng = np.random.default_rng(seed)
    sizes = np.floor(2.0 ** rng.uniform(log2_min, log2_max, nsys)).astype(np.int64)
    parts = [evrard_sphere(int(k), seed=int(rng.integers(1 << 31)), params=params) for k in sizes]
    cat = {k: np.concatenate([getattr(w, k) for w in parts]) for k in parts[0].arrays()}
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    p = params or parts[0].params
    w = Workload("ensemble", **cat, n_gas=int(offs[-1]), params=p, sys_offsets=offs)
    return w


def periodic_box(n: int = 1 << 20, seed: int = 6, L: float = 1.0, n_gas: int = 0, sigma_v: float = 0.0,
                 params: Params | None = None) -> Workload:
    """Particles in the periodic cube [0, L)^3 (Sect. 4.3): half uniform, half in three Gaussian clumps
    (dispersion 0.05 L, wrapped), equal masses summing to 1, optional gas (the first n_gas) with
    u = 0.5 and isotropic velocities of dispersion sigma_v."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(0.0, L, (n, 3))
    k = n // 2
    centres = rng.uniform(0.1, 0.9, (3, 3)) * L
    P[:k] = np.mod(centres[rng.integers(0, 3, k)] + rng.normal(0, 0.05 * L, (k, 3)), L)
    v = rng.normal(0, sigma_v, (n, 3)) if sigma_v > 0 else np.zeros((n, 3))
    p = params or Params(theta=0.5, gravity=1, sph=1 if n_gas else 0, adaptive_softening=1, n_nei_grav=32.0,
                         n_nei_sph=40.0, leaf_size=8, periodic_mask=7, periodic_lo=(0.0, 0.0, 0.0),
                         periodic_hi=(L, L, L))
    guess = _length_guess(np.full(n, n / L ** 3), 32.0)
    x, y, z, vx, vy, vz, m, uu, h, eps = _f32(P[:, 0], P[:, 1], P[:, 2], v[:, 0], v[:, 1], v[:, 2],
                                              np.full(n, 1.0 / n), np.full(n, 0.5), guess, guess)
    return Workload("periodic_box", x, y, z, vx, vy, vz, m, uu, h, eps, n_gas=n_gas, params=p)


def hot_core(w: Workload, factor: float = 30.0, radius: float = 0.2) -> Workload:
    """A copy of a gas sphere whose internal energy is raised near the centre,
    u (1 + factor exp(-(r/radius)^2)): a wide spread of Courant steps (individual time steps)."""
    import copy
    out = copy.copy(w)
    r = np.sqrt(w.x.astype(np.float64) ** 2 + w.y.astype(np.float64) ** 2 + w.z.astype(np.float64) ** 2)
    out.u = np.ascontiguousarray(w.u * (1.0 + factor * np.exp(-(r / radius) ** 2)), F32)
    return out


def with_dissipation(w: Workload, seed: int = 7, alpha=(0.05, 1.5), alpha_u=(0.0, 1.0), u_spread: float = 0.5,
                     sigma_v: float = 0.0, **params) -> Workload:
    """A copy of `w` with the per-particle inputs of the dissipation variants: alpha_i and alpha^u_i
    uniform in the given ranges, u_i multiplied by a log-uniform factor in [1/(1+s), 1+s] (so that
    neighbouring particles differ in u and the conductivity has work to do), optionally isotropic
    Gaussian velocities of dispersion sigma_v added, and the keyword arguments set on a copy of
    its Params (e.g. visc_form=1, balsara=1, variable_alpha=1, conduction=1)."""
    import copy
    import dataclasses

    rng = np.random.default_rng(seed)
    ng = w.n_gas
    out = copy.copy(w)
    out.params = dataclasses.replace(w.params, **params)
    out.alpha = np.ascontiguousarray(rng.uniform(alpha[0], alpha[1], ng), F32)
    out.alpha_u = np.ascontiguousarray(rng.uniform(alpha_u[0], alpha_u[1], ng), F32)
    if u_spread > 0 and ng:
        k = np.log1p(u_spread)
        uu = w.u.astype(np.float64).copy()
        uu[:ng] *= np.exp(rng.uniform(-k, k, ng))
        out.u = np.ascontiguousarray(uu, F32)
    if sigma_v > 0:
        out.vx, out.vy, out.vz = (np.ascontiguousarray(a + rng.normal(0.0, sigma_v, w.n), F32)
                                  for a in (w.vx, w.vy, w.vz))
    return out


def sample_indices(n: int, k: int, seed: int = 12345) -> np.ndarray:
    """A seeded sample of k distinct particle indices (sorted)."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)
