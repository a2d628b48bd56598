"""ctypes front end of the FP64 C oracle (``evol_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

The oracle is the force step written out plainly in double precision: root cube, Morton keys,
stable sort, recursive pre-order octree, node moments by direct summation, bisection for the
smoothing/softening lengths, and a per-particle tree walk (Sect. 2-3 of the paper).  It shares
no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evol_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build_oracle(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                   "-o", _SO + ".tmp", _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(_SO + ".tmp", _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(_SO)
        d = C.c_double
        for name in ("orc_W", "orc_dWdr", "orc_dWdh", "orc_dWdr_tc", "orc_phi", "orc_dphidr", "orc_dphideps"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d, d]
        L.orc_eta_from_nnei.restype = d
        L.orc_eta_from_nnei.argtypes = [d]
        L.orc_hash_id.restype = C.c_uint64
        L.orc_hash_id.argtypes = [C.c_uint64]
        L.orc_build.restype = C.c_void_p
        L.orc_build.argtypes = [C.c_int64, C.c_int64, _f32p, _f32p, _f32p, _f32p, C.c_int]
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_nnodes.restype = C.c_int64
        L.orc_nnodes.argtypes = [C.c_void_p]
        L.orc_get_cube.argtypes = [C.c_void_p, _f64p, _f64p]
        L.orc_get_keys.argtypes = [C.c_void_p, _u64p]
        L.orc_get_perm.argtypes = [C.c_void_p, _i32p]
        L.orc_get_nodes.argtypes = [C.c_void_p] + [_i32p] * 5
        L.orc_get_moments.argtypes = [C.c_void_p] + [_f64p] * 8
        L.orc_solve_lengths.restype = C.c_int
        L.orc_solve_lengths.argtypes = [C.c_void_p, C.c_int, d, C.c_void_p, C.c_int64, C.c_void_p, C.c_int,
                                        _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, C.c_void_p]
        L.orc_forces.argtypes = ([C.c_void_p, d, d, d, d, d, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                  _f64p, _f64p] + [_f64p] * 3 + [_f64p] * 3 + [_f64p] * 6 +
                                 [C.c_void_p, C.c_int64] + [_f64p] * 5 + [C.c_void_p] * 10 +
                                 [C.c_void_p] * 4)
        L.orc_divv.restype = C.c_int
        L.orc_divv.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, _f64p, _f64p, _f64p, _f64p, C.c_void_p,
                               C.c_int64, C.c_int, _f64p, _f64p, _f64p, C.c_void_p]
        L.orc_eos.argtypes = [C.c_int64, d, _f64p, _f64p, _f64p, _f64p]
        L.orc_ewald_exact.argtypes = [_f64p, d, _f64p, _f64p]
        L.orc_ewald_interp.argtypes = [d, _f64p, _f64p, _f64p]
        L.orc_sph_nbmin.restype = C.c_int
        L.orc_sph_nbmin.argtypes = [C.c_void_p, _f64p, C.c_void_p, C.c_int64, _f64p, C.c_int, _f64p, _f64p, _f64p]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


class _Kernels:
    """The paper's kernel functions, vectorised over numpy arrays (Eqs. spline, softforce,
    softphi, dphidh and the Thomas-Couchman gradient)."""

    def _vec(self, name, r, L):
        f = getattr(lib(), name)
        r, L = np.broadcast_arrays(np.asarray(r, np.float64), np.asarray(L, np.float64))
        out = np.empty(r.shape)
        for idx in np.ndindex(r.shape):
            out[idx] = f(float(r[idx]), float(L[idx]))
        return out if out.shape else float(out)

    def W(self, r, h): return self._vec("orc_W", r, h)
    def dWdr(self, r, h): return self._vec("orc_dWdr", r, h)
    def dWdh(self, r, h): return self._vec("orc_dWdh", r, h)
    def dWdr_tc(self, r, h): return self._vec("orc_dWdr_tc", r, h)
    def phi(self, r, e): return self._vec("orc_phi", r, e)
    def dphidr(self, r, e): return self._vec("orc_dphidr", r, e)
    def dphideps(self, r, e): return self._vec("orc_dphideps", r, e)


kernels = _Kernels()


def ewald(x, L: float = 1.0, exact: bool = True):
    """The Ewald correction (Sect. 4.3) for a unit mass at nearest-image offset x in a periodic
    cube of side L: (f, g), the acceleration (per G m) and potential (per G m) of the replicas beyond
    the nearest image; exact series, or the table interpolation the force pass uses."""
    xv = np.ascontiguousarray(x, np.float64)
    f, g = np.zeros(3), np.zeros(1)
    if exact:
        lib().orc_ewald_exact(xv, float(L), f, g)
    else:
        lib().orc_ewald_interp(float(L), xv, f, g)
    return f, float(g[0])


def eta_from_nnei(n_nei: float) -> float:
    return lib().orc_eta_from_nnei(float(n_nei))


def hash_id(i: int) -> int:
    return int(lib().orc_hash_id(int(i)))


class _Diss(C.Structure):
    # the dissipation-variant block of the force pass (orc_diss in evol_oracle.c)
    _fields_ = [("form", C.c_int), ("balsara", C.c_int), ("var_alpha", C.c_int), ("conduction", C.c_int),
                ("cond_vsig", C.c_int), ("f", C.c_void_p), ("alpha", C.c_void_p), ("alpha_u", C.c_void_p),
                ("u", C.c_void_p)]


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleTree:
    """Oracle tree over one particle set (root cube, keys, permutation, pre-order nodes,
    node moments)."""

    def __init__(self, x, y, z, m, n_gas: int, leaf: int):
        self.n = int(len(x))
        self.n_gas = int(n_gas)
        self._keep = [_c(a, np.float32) for a in (x, y, z, m)]
        self.ptr = lib().orc_build(self.n, self.n_gas, *self._keep, int(leaf))
        if not self.ptr:
            raise ValueError("oracle tree build failed (bad arguments or out of memory)")

    def __del__(self):
        if getattr(self, "ptr", None):
            lib().orc_free(self.ptr)
            self.ptr = None

    @property
    def nnodes(self) -> int:
        return int(lib().orc_nnodes(self.ptr))

    def cube(self):
        c = np.zeros(3)
        s = np.zeros(1)
        lib().orc_get_cube(self.ptr, c, s)
        return c, float(s[0])

    def keys(self):
        k = np.empty(self.n, np.uint64)
        lib().orc_get_keys(self.ptr, k)
        return k

    def perm(self):
        p = np.empty(self.n, np.int32)
        lib().orc_get_perm(self.ptr, p)
        return p

    def nodes(self):
        nn = self.nnodes
        a = [np.empty(nn, np.int32) for _ in range(5)]
        lib().orc_get_nodes(self.ptr, *a)
        return dict(zip(("begin", "end", "level", "next", "nchild"), a))

    def moments(self):
        nn = self.nnodes
        M, com, Q = np.empty(nn), np.empty((nn, 3)), np.empty((nn, 6))
        delta, bmin, bmax, cgeo, l = np.empty(nn), np.empty((nn, 3)), np.empty((nn, 3)), np.empty((nn, 3)), np.empty(nn)
        lib().orc_get_moments(self.ptr, M, com, Q, delta, bmin, bmax, cgeo, l)
        return dict(M=M, com=com, Q=Q, delta=delta, bmin=bmin, bmax=bmax, cgeo=cgeo, l=l)

    def _period(self, params):
        lo = _c(getattr(params, "periodic_lo", (0, 0, 0)), np.float64)
        hi = _c(getattr(params, "periodic_hi", (1, 1, 1)), np.float64)
        return int(getattr(params, "periodic_mask", 0)), lo, hi

    def solve_lengths(self, mode: int, n_nei: float, guess=None, idx=None, params=None):
        """mode 0: gas h -> (h, n, rho, Omega*, zeta); mode 1: eps -> (eps, n, Upsilon, X);
        mode 2: gas h of the standard scheme (N = n_nei neighbours inside 2h) -> (h, n, rho, 1, 0)."""
        n = self.n
        outs = [np.zeros(n) for _ in range(5)]
        pm, lo, hi = self._period(params)
        g = _c(guess, np.float32) if guess is not None else None
        ix = _c(idx, np.int64) if idx is not None else None
        rc = lib().orc_solve_lengths(self.ptr, int(mode), float(n_nei),
                                     ix.ctypes.data if ix is not None else None,
                                     int(len(ix)) if ix is not None else 0,
                                     g.ctypes.data if g is not None else None,
                                     pm, lo, hi, *outs[:4], outs[4].ctypes.data)
        if rc != 0:
            raise RuntimeError(f"oracle length solve failed (code {rc})")
        return outs

    def forces(self, params, state: dict, idx=None, use_tc=None):
        """Force pass.  The dissipation variants of Sect. 3.3.3 are taken from params (visc_form,
        balsara, variable_alpha, conduction, cond_vsig; all 0 by default) with the per-particle
        arrays state["f"] (Balsara factor), state["alpha"], state["alpha_u"] and state["u"]."""
        n = self.n
        z = np.zeros(n)
        g = lambda k: _c(state.get(k, z), np.float64)
        ds = _Diss()
        ds.form = int(getattr(params, "visc_form", 0))
        ds.balsara = int(getattr(params, "balsara", 0))
        ds.var_alpha = int(getattr(params, "variable_alpha", 0))
        ds.conduction = int(getattr(params, "conduction", 0))
        ds.cond_vsig = int(getattr(params, "cond_vsig", 0))
        keep = {k: g(k) for k in ("f", "alpha", "alpha_u", "u")}
        ds.f, ds.alpha, ds.alpha_u, ds.u = (keep[k].ctypes.data for k in ("f", "alpha", "alpha_u", "u"))
        vsig, lapu, lapabs = np.zeros(n), np.zeros(n), np.zeros(n)
        pm, lo, hi = self._period(params)
        ix = _c(idx, np.int64) if idx is not None else None
        out = [np.zeros(n) for _ in range(5)]
        hashes = [np.zeros(n, np.uint64) for _ in range(3)]
        counts = [np.zeros(n, np.int64) for _ in range(3)]
        margin = np.full(n, np.inf)
        aabs, duabs, mumax = np.zeros(n), np.zeros(n), np.zeros(n)
        tc = params.use_tc_gradient if use_tc is None else use_tc
        lib().orc_forces(self.ptr, float(params.theta), float(params.G), float(params.gamma),
                         float(params.alpha), float(params.beta), int(params.gravity), int(params.sph),
                         int(params.adaptive_softening), int(tc), pm, lo, hi,
                         g("vx"), g("vy"), g("vz"), g("eps"), g("ups"), g("X"),
                         g("h"), g("rho"), g("P"), g("c"), g("omega"), g("zeta"),
                         ix.ctypes.data if ix is not None else None, int(len(ix)) if ix is not None else 0,
                         *out, *[a.ctypes.data for a in hashes], *[a.ctypes.data for a in counts],
                         margin.ctypes.data, aabs.ctypes.data, duabs.ctypes.data, mumax.ctypes.data,
                         C.addressof(ds), vsig.ctypes.data, lapu.ctypes.data, lapabs.ctypes.data)
        res = dict(zip(("ax", "ay", "az", "pot", "dudt"), out))
        res.update(zip(("hfar", "hnear", "hsph"), hashes))
        res.update(zip(("nfar", "npp", "nsph"), counts))
        res["margin"] = margin
        res["aabs"] = aabs
        res["duabs"] = duabs
        res["mumax"] = mumax
        res["vsig"] = vsig
        res["lapu"] = lapu
        res["lapabs"] = lapabs
        return res

    def sph_nbmin(self, h, idx, key, params=None):
        """For every gas particle j the smallest key[i] over the gas particles i in idx that are its SPH
        neighbours (r_ij < 2 max(h_i, h_j), i != j); +inf where there is none."""
        out = np.full(self.n, np.inf)
        pm, lo, hi = self._period(params)
        ix = _c(idx, np.int64)
        rc = lib().orc_sph_nbmin(self.ptr, _c(h, np.float64), ix.ctypes.data, int(len(ix)), _c(key, np.float64),
                                 pm, lo, hi, out)
        if rc != 0:
            raise RuntimeError(f"oracle neighbour minimum failed (code {rc})")
        return out

    def divv(self, mode: int, L, nsum, corr, vx, vy, vz, idx=None, params=None, curl=False):
        """Velocity divergence from the discretised continuity equation (Sect. 2.1): mode 1 with the
        softening kernel over all species (corr = Upsilon), mode 0 with the smoothing kernel over
        the gas (corr = Omega*).  Arrays in original order; returns div v (original order), and with
        curl=True also |curl v| from the same neighbour sum."""
        n = self.n
        out = np.zeros(n)
        cv = np.zeros(n) if curl else None
        pm, lo, hi = self._period(params)
        ix = _c(idx, np.int64) if idx is not None else None
        rc = lib().orc_divv(self.ptr, int(mode), _c(L, np.float64), _c(nsum, np.float64), _c(corr, np.float64),
                            _c(vx, np.float64), _c(vy, np.float64), _c(vz, np.float64),
                            ix.ctypes.data if ix is not None else None, int(len(ix)) if ix is not None else 0,
                            pm, lo, hi, out, cv.ctypes.data if curl else None)
        if rc != 0:
            raise RuntimeError(f"oracle divergence failed (code {rc})")
        return (out, cv) if curl else out


def force_step(w, params=None, idx=None, use_tc=None, tree=None, fixed_lengths=None):
    """The whole force step on workload `w` in FP64: tree, eps solve (adaptive softening, all
    particles), h solve (gas), equation of state, and the force pass for the particles in idx
    (all if None).  Returns a dict of original-order float64 arrays."""
    p = params or w.params
    t = tree or OracleTree(w.x, w.y, w.z, w.m, w.n_gas, p.leaf_size)
    n = w.n
    st = {"vx": w.vx.astype(np.float64), "vy": w.vy.astype(np.float64), "vz": w.vz.astype(np.float64)}
    res = {}
    if fixed_lengths is not None:
        st.update(fixed_lengths)
    else:
        if p.gravity:
            if p.adaptive_softening:
                eps, neps, ups, X, _ = t.solve_lengths(1, p.n_nei_grav, guess=w.eps, params=p)
            else:
                eps, neps, ups, X = w.eps.astype(np.float64), np.zeros(n), np.ones(n), np.zeros(n)
            st.update(eps=eps, ups=ups, X=X)
            res.update(eps=eps, n_eps=neps, ups=ups, X=X)
        if p.sph and w.n_gas > 0:
            gidx = np.arange(w.n_gas, dtype=np.int64)
            hmode = 2 if int(getattr(p, "sph_scheme", 0)) == 1 else 0
            h, nh, rho, om, zeta = t.solve_lengths(hmode, p.n_nei_sph, guess=w.h, idx=gidx, params=p)
            P, c = np.zeros(n), np.zeros(n)
            lib().orc_eos(n, float(p.gamma), _c(rho, np.float64), _c(w.u.astype(np.float64), np.float64), P, c)
            P[w.n_gas:] = 0
            c[w.n_gas:] = 0
            st.update(h=h, rho=rho, omega=om, zeta=zeta, P=P, c=c)
            res.update(h=h, n_h=nh, rho=rho, omega=om, zeta=zeta, P=P, c=c)
        # velocity divergence from the discretised continuity equation (Sect. 2.1), with each length
        if p.gravity and p.adaptive_softening:
            res["divv_eps"] = t.divv(1, eps, neps, ups, st["vx"], st["vy"], st["vz"], params=p)
        if p.sph and w.n_gas > 0:
            res["divv_h"], res["curlv_h"] = t.divv(0, h, nh, om, st["vx"], st["vy"], st["vz"], idx=gidx,
                                                   params=p, curl=True)
    diss = p.sph and w.n_gas > 0 and _dissipation_on(p)
    if diss:
        st.update(_dissipation_state(w, p, res, st))
        res["balsara_f"] = st["f"]
    f = t.forces(p, st, idx=idx, use_tc=use_tc)
    res.update(f)
    if diss:
        res.update(_dissipation_rates(w, p, res, st))
    res["tree"] = t
    res["state"] = st
    return res


def _dissipation_on(p) -> bool:
    return bool(getattr(p, "visc_form", 0) or getattr(p, "balsara", 0) or getattr(p, "variable_alpha", 0)
                or getattr(p, "conduction", 0))


def _dissipation_state(w, p, res, st):
    """Per-particle inputs of the dissipation variants (Sect. 3.3.3), original order, gas only.

    Balsara limiter: f_i = |div v_i| / (|div v_i| + |curl v_i| + eta_B c_i / h_i), div v and curl v
    from the smoothing-kernel neighbour sums.  Reading: f_i = 0 where the denominator vanishes (a
    particle at rest relative to its neighbours with u_i = 0).  alpha_i and alpha^u_i come with the
    particles; without them the constant alpha (and alpha^u = 0) is used."""
    n, ng = w.n, w.n_gas
    f = np.zeros(n)
    zero = np.zeros(n)
    dv = np.abs(res.get("divv_h", st.get("divv_h", zero))[:ng])
    cv = res.get("curlv_h", st.get("curlv_h", zero))[:ng]
    den = dv + cv + float(getattr(p, "balsara_eta", 1e-4)) * st["c"][:ng] / st["h"][:ng]
    with np.errstate(invalid="ignore", divide="ignore"):
        f[:ng] = np.where(den > 0, dv / den, 0.0)
    alpha = np.full(n, float(p.alpha))
    a_in = getattr(w, "alpha", None)
    if a_in is not None:
        alpha[:ng] = np.asarray(a_in, np.float64)[:ng]
    alpha_u = np.zeros(n)
    au_in = getattr(w, "alpha_u", None)
    if au_in is not None:
        alpha_u[:ng] = np.asarray(au_in, np.float64)[:ng]
    u = np.zeros(n)
    u[:ng] = np.asarray(w.u, np.float64)[:ng]
    out = {"f": f, "alpha": alpha, "alpha_u": alpha_u, "u": u}
    if "f" in st:                      # a given limiter (fixed-lengths runs) is kept
        out["f"] = np.asarray(st["f"], np.float64)
    return out


def _dissipation_rates(w, p, res, st):
    """Time derivatives of alpha_i (Eq. alphaswitch) and alpha^u_i (Sect. 3.3.3), gas only:

      tau_i        = alpha_tau h_i / v^sig_i,   v^sig_i = max_j v^sig_ij (Eq. vsig; self pair 2 c_i)
      dalpha/dt    = -(alpha_i - alpha_min) / tau_i + alpha_source f_i max(0, -div v_i)
      dalpha^u/dt  = -(alpha^u_i - alpha^u_min) / tau_i + S^u_i,
      S^u_i        = h_i |lap u_i| / sqrt(u_i)      (cond_source 0, Price 2008)
                   = 0.1 h_i |lap u_i|               (cond_source 1, Price 2005)

    Reading: the source term is printed as 0.75 f_i max[0, -|div v_i|], which is zero for every
    flow; the intended switch is on in compression, max(0, -div v_i).  alpha_tau = 0.1 is the
    printed e-folding constant."""
    n, ng = w.n, w.n_gas
    h, vs = st["h"][:ng], res["vsig"][:ng]
    with np.errstate(divide="ignore"):        # particles outside an index sample have v^sig = 0
        tau = float(getattr(p, "alpha_tau", 0.1)) * h / vs
    out = {}
    if getattr(p, "variable_alpha", 0):
        da = np.zeros(n)
        da[:ng] = (-(st["alpha"][:ng] - float(getattr(p, "alpha_min", 0.01))) / tau +
                   float(getattr(p, "alpha_source", 0.75)) * st["f"][:ng] *
                   np.maximum(0.0, -res.get("divv_h", st.get("divv_h", np.zeros(n)))[:ng]))
        out["dalpha"] = da
    if getattr(p, "conduction", 0):
        lap = np.abs(res["lapu"][:ng])
        if int(getattr(p, "cond_source", 0)) == 0:
            S = h * lap / np.sqrt(st["u"][:ng])
        else:
            S = 0.1 * h * lap
        dau = np.zeros(n)
        dau[:ng] = -(st["alpha_u"][:ng] - float(getattr(p, "alpha_u_min", 0.0))) / tau + S
        out["dalpha_u"] = dau
    return out


def kdk(w, dt: float, nsteps: int, params=None):
    """Kick-drift-kick leapfrog with a fixed step (Sect. 4.1) in FP64 on top of force_step.

    The state (x, v, u) is kept in double precision; each force evaluation receives it rounded to
    float32, the oracle's input type.  Periodic axes are wrapped into [lo, hi).  Returns a dict
    with x, y, z, vx, vy, vz, u (float64) and the last force-step result."""
    import copy

    p = params or w.params
    n, ng = w.n, w.n_gas
    X = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    V = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    U = w.u.astype(np.float64).copy()
    cur = copy.copy(w)

    sw = _Switches(w, p, cur)

    def forces():
        cur.x, cur.y, cur.z = (np.ascontiguousarray(X[:, a], np.float32) for a in range(3))
        cur.vx, cur.vy, cur.vz = (np.ascontiguousarray(V[:, a], np.float32) for a in range(3))
        cur.u = np.ascontiguousarray(U, np.float32)
        sw.hand_over()
        r = force_step(cur, params=p)
        A = np.stack([r["ax"], r["ay"], r["az"]], 1)
        return A, r["dudt"], r

    A, DU, r = forces()
    lo = np.asarray(getattr(p, "periodic_lo", (0, 0, 0)), np.float64)
    hi = np.asarray(getattr(p, "periodic_hi", (1, 1, 1)), np.float64)
    for _ in range(nsteps):
        V += 0.5 * dt * A
        U[:ng] += 0.5 * dt * DU[:ng]
        sw.kick(0.5 * dt, r)
        X += dt * V
        for a in range(3):
            if (getattr(p, "periodic_mask", 0) >> a) & 1:
                X[:, a] = lo[a] + np.mod(X[:, a] - lo[a], hi[a] - lo[a])
        A, DU, r = forces()
        V += 0.5 * dt * A
        U[:ng] += 0.5 * dt * DU[:ng]
        sw.kick(0.5 * dt, r)
    return {"x": X[:, 0], "y": X[:, 1], "z": X[:, 2], "vx": V[:, 0], "vy": V[:, 1], "vz": V[:, 2], "u": U,
            **sw.result(), "last": r}


class _Switches:
    """The per-particle dissipation switches alpha_i (variable alpha) and alpha^u_i (conduction) as
    integrator state: kept in FP64, handed to each force step rounded to float32, and advanced by
    the kicks with their time derivatives, as u is (no prediction)."""

    def __init__(self, w, p, cur):
        ng = w.n_gas
        self.cur = cur
        self.al = (np.asarray(w.alpha, np.float64)[:ng].copy()
                   if getattr(p, "variable_alpha", 0) and getattr(w, "alpha", None) is not None else None)
        self.alu = (np.asarray(w.alpha_u, np.float64)[:ng].copy()
                    if getattr(p, "conduction", 0) and getattr(w, "alpha_u", None) is not None else None)

    def hand_over(self):
        if self.al is not None:
            self.cur.alpha = np.ascontiguousarray(self.al, np.float32)
        if self.alu is not None:
            self.cur.alpha_u = np.ascontiguousarray(self.alu, np.float32)

    def kick(self, hdt, r):
        ng = len(self.al) if self.al is not None else (len(self.alu) if self.alu is not None else 0)
        if self.al is not None:
            self.al += hdt * r["dalpha"][:ng]
        if self.alu is not None:
            self.alu += hdt * r["dalpha_u"][:ng]

    def result(self):
        out = {}
        if self.al is not None:
            out["alpha"] = self.al
        if self.alu is not None:
            out["alpha_u"] = self.alu
        return out


@dataclass
class TimeStep:
    """Parameters of the global time step (Sect. 4.2): each eta scales one criterion (0 leaves it
    out); the step is the smallest criterion over all particles, clamped to [dt_min, dt_max]."""
    eta_acc: float = 0.1
    eta_vel: float = 0.0
    eta_av: float = 0.0
    eta_courant: float = 0.1
    eta_u: float = 0.1
    dt_min: float = 0.0
    dt_max: float = 1.0


def timestep_criteria(w, res, vx, vy, vz, u, ts, params=None):
    """Per-particle time-step criteria of Sect. 4.2 from the results of a force step.

    L_i = min(eps_i, h_i) (eps alone for non-gas particles, h alone without gravity).
      dt_acc = eta_acc sqrt(L / |a|)
      dt_vel = eta_vel L / |v|                      (reading: the printed square root is not a time)
      dt_av  = eta_av |v| / |a|                     (reading: the same)
      dt_C   = eta_C h / (h |div v| + c + 1.2 (alpha c + beta max_j |mu_ij|))     (gas; alpha_i
               with variable alpha)
      dt_u   = eta_u |u / (du/dt)|                                                 (gas)
    div v is the smoothing-kernel estimate of the continuity equation.  Returns a dict of arrays
    (inf where a criterion does not apply)."""
    p = params or w.params
    n, ng = w.n, w.n_gas
    inf = np.full(n, np.inf)
    a = np.sqrt(res["ax"] ** 2 + res["ay"] ** 2 + res["az"] ** 2)
    v = np.sqrt(np.asarray(vx, np.float64) ** 2 + np.asarray(vy, np.float64) ** 2 + np.asarray(vz, np.float64) ** 2)
    L = res["eps"].copy() if p.gravity else np.full(n, np.inf)
    if p.sph and ng:
        L[:ng] = np.minimum(L[:ng], res["h"][:ng])
    with np.errstate(divide="ignore", invalid="ignore"):
        out = {"acc": ts.eta_acc * np.sqrt(L / a) if ts.eta_acc > 0 else inf,
               "vel": ts.eta_vel * L / v if ts.eta_vel > 0 else inf,
               "av": ts.eta_av * v / a if ts.eta_av > 0 else inf}
        c_ = inf.copy()
        uu = inf.copy()
        if p.sph and ng:
            h = res["h"][:ng]
            c = res["c"][:ng]
            # alpha_i with variable alpha (the value the force step used)
            al = res["state"]["alpha"][:ng] if getattr(p, "variable_alpha", 0) else p.alpha
            den = h * np.abs(res["divv_h"][:ng]) + c + 1.2 * (al * c + p.beta * res["mumax"][:ng])
            c_[:ng] = ts.eta_courant * h / den if ts.eta_courant > 0 else np.inf
            uu[:ng] = ts.eta_u * np.abs(np.asarray(u[:ng], np.float64) / res["dudt"][:ng]) if ts.eta_u > 0 else np.inf
        out["courant"] = c_
        out["u"] = uu
    for k in out:
        out[k] = np.where(np.isfinite(out[k]) & (out[k] > 0), out[k], np.inf)
    return out


def global_timestep(crit, ts):
    """The smallest criterion over all particles, clamped to [dt_min, dt_max]."""
    dt = min(float(np.min(c)) for c in crit.values())
    return float(min(max(dt, ts.dt_min), ts.dt_max))


def run(w, nsteps: int, ts: TimeStep, params=None, predicted=True):
    """Global-time-step KDK leapfrog (Sect. 4.1-4.2) in FP64 on top of force_step.

    Each step: dt from the criteria of the last force step; v += a dt/2, u += du/dt dt/2;
    x += v dt; a force step at the new positions in which the SPH terms use the predicted
    v_n + a_n dt and the equation of state the predicted u_n + (du/dt)_n dt (Sect. 4.1, when
    `predicted`); v += a dt/2, u += du/dt dt/2.  The state is kept in FP64 and handed to each force
    step rounded to float32.  Returns the final state, the list of time steps and the last
    force-step result."""
    import copy

    p = params or w.params
    n, ng = w.n, w.n_gas
    X = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    V = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    U = w.u.astype(np.float64).copy()
    cur = copy.copy(w)

    sw = _Switches(w, p, cur)

    def forces(vel, uu):
        cur.x, cur.y, cur.z = (np.ascontiguousarray(X[:, a], np.float32) for a in range(3))
        cur.vx, cur.vy, cur.vz = (np.ascontiguousarray(vel[:, a], np.float32) for a in range(3))
        cur.u = np.ascontiguousarray(uu, np.float32)
        sw.hand_over()
        r = force_step(cur, params=p)
        return np.stack([r["ax"], r["ay"], r["az"]], 1), r["dudt"], r

    A, DU, r = forces(V, U)
    lo = np.asarray(getattr(p, "periodic_lo", (0, 0, 0)), np.float64)
    hi = np.asarray(getattr(p, "periodic_hi", (1, 1, 1)), np.float64)
    dts = []
    for _ in range(nsteps):
        crit = timestep_criteria(cur, r, V[:, 0], V[:, 1], V[:, 2], U, ts, params=p)
        dt = global_timestep(crit, ts)
        dts.append(dt)
        V += 0.5 * dt * A
        U[:ng] += 0.5 * dt * DU[:ng]
        sw.kick(0.5 * dt, r)
        X += dt * V
        for a in range(3):
            if (getattr(p, "periodic_mask", 0) >> a) & 1:
                X[:, a] = lo[a] + np.mod(X[:, a] - lo[a], hi[a] - lo[a])
        if predicted:
            Vp = V + 0.5 * dt * A
            Up = U.copy()
            Up[:ng] += 0.5 * dt * DU[:ng]
        else:
            Vp, Up = V, U
        A, DU, r = forces(Vp, Up)
        V += 0.5 * dt * A
        U[:ng] += 0.5 * dt * DU[:ng]
        sw.kick(0.5 * dt, r)
    return {"x": X[:, 0], "y": X[:, 1], "z": X[:, 2], "vx": V[:, 0], "vy": V[:, 1], "vz": V[:, 2], "u": U,
            **sw.result(), "dts": dts, "last": r}


# ---- individual power-of-two time steps (Sect. 4.2.1) -----------------------------------------

_PERSIST = ("eps", "ups", "X", "h", "n_h", "rho", "omega", "zeta", "divv_h", "curlv_h")


def active_force_step(w, active, pers, params=None):
    """Force step in which only the particles in `active` (original indices) are evaluated.

    Their eps (all species, adaptive softening) and h (gas) are solved again from the starting
    guesses w.eps / w.h, and div v, curl v formed for the active gas; every other particle keeps
    what `pers` holds from its last evaluation (eps, Upsilon, X, h, n, rho, Omega*, zeta, div v,
    curl v).  The equation of state takes every gas particle's current u.  `pers` is updated in
    place for the active particles.  Returns a force_step-like dict for all particles, whose
    force results are valid at the active ones."""
    p = params or w.params
    t = OracleTree(w.x, w.y, w.z, w.m, w.n_gas, p.leaf_size)
    n, ng = w.n, w.n_gas
    act = np.asarray(active, np.int64)
    actg = act[act < ng]
    if p.gravity:
        if p.adaptive_softening:
            if len(act):
                eps, _, ups, X, _ = t.solve_lengths(1, p.n_nei_grav, guess=w.eps, idx=act, params=p)
                for k, v in (("eps", eps), ("ups", ups), ("X", X)):
                    pers[k][act] = v[act]
        else:
            pers["eps"][:] = w.eps
            pers["ups"][:] = 1.0
            pers["X"][:] = 0.0
    st = {"vx": w.vx.astype(np.float64), "vy": w.vy.astype(np.float64), "vz": w.vz.astype(np.float64)}
    if p.gravity:
        st.update(eps=pers["eps"].copy(), ups=pers["ups"].copy(), X=pers["X"].copy())
    if p.sph and ng:
        hmode = 2 if int(getattr(p, "sph_scheme", 0)) == 1 else 0
        if len(actg):
            h, nh, rho, om, zeta = t.solve_lengths(hmode, p.n_nei_sph, guess=w.h, idx=actg, params=p)
            for k, v in (("h", h), ("n_h", nh), ("rho", rho), ("omega", om), ("zeta", zeta)):
                pers[k][actg] = v[actg]
            dv, cv = t.divv(0, pers["h"], pers["n_h"], pers["omega"], st["vx"], st["vy"], st["vz"], idx=actg,
                            params=p, curl=True)
            pers["divv_h"][actg] = dv[actg]
            pers["curlv_h"][actg] = cv[actg]
        P, c = np.zeros(n), np.zeros(n)
        lib().orc_eos(n, float(p.gamma), _c(pers["rho"], np.float64), _c(w.u.astype(np.float64), np.float64), P, c)
        P[ng:] = 0
        c[ng:] = 0
        st.update(h=pers["h"].copy(), rho=pers["rho"].copy(), omega=pers["omega"].copy(),
                  zeta=pers["zeta"].copy(), P=P, c=c)
    res = {k: pers[k].copy() for k in _PERSIST}
    if p.sph and ng:
        res.update(P=st["P"], c=st["c"])
    diss = p.sph and ng > 0 and _dissipation_on(p)
    if diss:
        st.update(_dissipation_state(w, p, res, st))
        res["balsara_f"] = st["f"]
    res.update(t.forces(p, st, idx=act))
    if diss:
        res.update(_dissipation_rates(w, p, res, st))
    res["tree"] = t
    res["state"] = st
    return res


@dataclass
class Bins:
    """Individual time steps (Sect. 4.2.1): steps dt_max / 2^k, 0 <= k <= max_bin, on an integer
    timeline of 2^max_bin ticks per largest step; wake_factor > 1 wakes an inactive gas particle
    whose step exceeds wake_factor times the step of an active SPH neighbour (0: off)."""
    max_bin: int = 6
    wake_factor: float = 0.0


def step_ticks(dt, T: int, tick: float):
    """The largest power-of-two step, in ticks, not longer than dt: L = 2^m with L tick <= dt,
    clamped to [1, T] (a criterion shorter than one tick gets the finest step).

    Reading: the printed rule takes the smallest n with dt_max / 2^n >= dt_i, which n = 0 always
    meets; the step is meant not to exceed the criterion, so the largest such step is taken."""
    dt = np.asarray(dt, np.float64)
    L = np.ones(dt.shape, np.int64)
    for _ in range(63):
        grow = (2 * L <= T) & (2 * L * tick <= dt)
        if not grow.any():
            break
        L = np.where(grow, 2 * L, L)
    return L


def _lowbit(t):
    t = np.asarray(t, np.int64)
    return t & -t


def run_bins(w, nlargest: int, ts: TimeStep, bins: Bins, params=None, predicted=True, stop_after=None):
    """Individual power-of-two time steps (Sect. 4.2.1) with KDK kicks, in FP64.

    Integer timeline: T = 2^max_bin ticks per largest step ts.dt_max.  Each particle has a step
    [tb, te] whose length is a power of two that divides tb.  A system step:
      1. t_next = min te; every particle drifts x += v (t_next - t_sys) (v: its half-kicked velocity);
      2. the particles with te = t_next are active: a force step evaluates them only (active_force_step),
         the SPH terms using every particle's velocity and u predicted to t_next,
         v_p = v + a (t_next - (tb + te)/2), u likewise (Sect. 4.1; off with predicted=False);
      3. active particles: second half kick v += a (te - tb)/2, u and the dissipation switches alike;
      4. wake-up: an inactive gas particle j whose step exceeds wake_factor times the step just
         completed by an active SPH neighbour ends its step early, at the first multiple of
         L' > t_next, L' the largest power of two <= wake_factor times that neighbour step; the
         first half kick it received is cut to the shortened step (energy and momentum are then
         not exactly conserved, as the paper says);
      5. active particles, unless t_next ends the run: the criteria of the global step (Sect. 4.2)
         give L = step_ticks(dt_i); a longer step than before only where t_next is a multiple of it:
         L = min(L, largest power of two dividing t_next); tb = t_next, te = t_next + L; first half
         kick v += a L/2.
    Everything starts synchronised at t = 0 with a force step of all particles and ends so at
    nlargest * T (stop_after: end after that many system steps instead, mid-run).  Returns the
    final state, the per-particle steps and counts."""
    import copy

    p = params or w.params
    n, ng = w.n, w.n_gas
    K = int(bins.max_bin)
    T = 1 << K
    tick = ts.dt_max / T
    t_end = int(nlargest) * T
    X = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    V = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    U = w.u.astype(np.float64).copy()
    cur = copy.copy(w)
    sw = _Switches(w, p, cur)
    pers = {k: np.zeros(n) for k in _PERSIST}
    pers["h"][:ng] = w.h[:ng]
    pers["eps"][:] = w.eps
    lo = np.asarray(getattr(p, "periodic_lo", (0, 0, 0)), np.float64)
    hi = np.asarray(getattr(p, "periodic_hi", (1, 1, 1)), np.float64)
    gas = np.arange(n) < ng

    def evaluate(active, vel, uu):
        cur.x, cur.y, cur.z = (np.ascontiguousarray(X[:, a], np.float32) for a in range(3))
        cur.vx, cur.vy, cur.vz = (np.ascontiguousarray(vel[:, a], np.float32) for a in range(3))
        cur.u = np.ascontiguousarray(uu, np.float32)
        cur.h = np.ascontiguousarray(np.where(gas, pers["h"], w.h), np.float32)
        cur.eps = np.ascontiguousarray(pers["eps"], np.float32)
        sw.hand_over()
        return active_force_step(cur, active, pers, p)

    def kick(idx, f_ticks, r_acc, r_du, r_sw):
        hdt = (f_ticks * tick)
        V[idx] += hdt[:, None] * r_acc[idx]
        U[idx] += np.where(gas[idx], hdt * r_du[idx], 0.0)
        for k, arr in (("al", "dalpha"), ("alu", "dalpha_u")):
            a = getattr(sw, k)
            if a is not None:
                g = idx[idx < ng]
                a[g] += (f_ticks[idx < ng] * tick) * r_sw[arr][g]

    allp = np.arange(n, dtype=np.int64)
    A = np.zeros((n, 3))
    DU = np.zeros(n)
    rates = {"dalpha": np.zeros(n), "dalpha_u": np.zeros(n)}
    r = evaluate(allp, V, U)

    def take(r, idx):
        A[idx] = np.stack([r["ax"], r["ay"], r["az"]], 1)[idx]
        DU[idx] = r["dudt"][idx]
        for k in rates:
            if k in r:
                rates[k][idx] = r[k][idx]

    def new_steps(r, idx, tnow):
        crit = timestep_criteria(cur, r, V[:, 0], V[:, 1], V[:, 2], U, ts, params=p)
        dt = np.min(np.stack([c for c in crit.values()]), 0)
        dt = np.where(np.isfinite(dt), dt, ts.dt_max)
        L = step_ticks(dt[idx], T, tick)
        # how close each decision came to a boundary of its power-of-two interval (relative): an
        # FP32 evaluation of the criteria can only decide otherwise below about 1e-6
        q = dt[idx] / (L * tick)
        free = (L < T) & (q >= 1.0)
        if free.any():
            stats["step_margin"] = min(stats["step_margin"], float(np.min(np.minimum(q[free] - 1.0, 2.0 - q[free]) / 2.0)))
        if tnow > 0:
            L = np.minimum(L, int(_lowbit(tnow)))
        tb[idx] = tnow
        te[idx] = tnow + L
        kick(idx, 0.5 * L.astype(np.float64), A, DU, rates)
        return dt

    take(r, allp)
    tb = np.zeros(n, np.int64)
    te = np.zeros(n, np.int64)
    stats = {"system_steps": 0, "active_evaluations": n, "wakeups": 0, "step_margin": np.inf}
    if t_end > 0:
        new_steps(r, allp, 0)
    tsys = 0
    while tsys < t_end:
        tnext = int(te.min())
        X += V * ((tnext - tsys) * tick)
        for a in range(3):
            if (getattr(p, "periodic_mask", 0) >> a) & 1:
                X[:, a] = lo[a] + np.mod(X[:, a] - lo[a], hi[a] - lo[a])
        act = np.flatnonzero(te == tnext).astype(np.int64)
        if predicted:
            tau = (tnext - 0.5 * (tb + te)) * tick
            Vp = V + tau[:, None] * A
            Up = U + np.where(gas, tau * DU, 0.0)
        else:
            Vp, Up = V, U
        r = evaluate(act, Vp, Up)
        take(r, act)
        kick(act, 0.5 * (te[act] - tb[act]).astype(np.float64), A, DU, rates)
        if bins.wake_factor > 0 and ng:
            key = np.full(n, np.inf)
            key[act] = (te[act] - tb[act]).astype(np.float64)
            m = r["tree"].sph_nbmin(pers["h"], act, key, params=p)
            inact = np.flatnonzero(gas & (te != tnext) & np.isfinite(m))
            for j in inact:
                Lj = int(te[j] - tb[j])
                if Lj > bins.wake_factor * m[j]:
                    Lw = int(step_ticks(np.array([bins.wake_factor * m[j] * tick]), T, tick)[0])
                    if Lw < Lj:
                        tn = (tnext // Lw + 1) * Lw
                        if tn < te[j]:
                            cut = 0.5 * (Lj - (tn - tb[j]))
                            kick(np.array([j]), np.array([-cut]), A, DU, rates)
                            te[j] = tn
                            stats["wakeups"] += 1
        if tnext < t_end:
            new_steps(r, act, tnext)
        tsys = tnext
        stats["system_steps"] += 1
        stats["active_evaluations"] += len(act)
        if stop_after is not None and stats["system_steps"] >= stop_after:
            break
    return {"x": X[:, 0], "y": X[:, 1], "z": X[:, 2], "vx": V[:, 0], "vy": V[:, 1], "vz": V[:, 2], "u": U,
            **sw.result(), "tb": tb, "te": te, "stats": stats, "last": r}
