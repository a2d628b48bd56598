"""Thin ctypes binding of the C ABI in include/evol.h (argument marshalling only).

Every computation runs in libevol.so's CUDA kernels; this module only fills the C structs
with the device pointers of torch tensors (or host pointers for ``evol_step_host``) and
checks status codes.  If the library is missing the calls raise: there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libevol.so")

EVOL_OK, EVOL_EINVAL, EVOL_ENOMEM, EVOL_ECUDA = 0, -1, -2, -3
EVOL_EOVERFLOW, EVOL_ENOCONV, EVOL_ETIMEOUT, EVOL_ENAN, EVOL_ESTATE = -4, -5, -6, -7, -8
EVOL_FP32_PLAIN, EVOL_FP32_MIXED = 0, 1
EVOL_DBG_KEYS, EVOL_DBG_PERM, EVOL_DBG_NODES, EVOL_DBG_CUBE = 1, 2, 3, 4
EVOL_DBG_MOMENTS, EVOL_DBG_HASHES, EVOL_DBG_COUNTS, EVOL_DBG_FLOW = 5, 6, 7, 8
EVOL_DBG_DISS, EVOL_DBG_BINS = 9, 10
EVOL_VISC_MONAGHAN, EVOL_VISC_SIGNAL = 0, 1
EVOL_COND_VSIG_SOUND, EVOL_COND_VSIG_PRESSURE = 0, 1
EVOL_COND_SRC_SQRTU, EVOL_COND_SRC_LINEAR = 0, 1
EVOL_SPH_LAGRANGIAN, EVOL_SPH_STANDARD = 0, 1
EVOL_TUNE_LEAF_SIZE, EVOL_TUNE_LENGTH_GROUP = 0, 1

_fp = C.POINTER(C.c_float)


class EvolParticles(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_gas", C.c_int64),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p),
                ("vx", C.c_void_p), ("vy", C.c_void_p), ("vz", C.c_void_p),
                ("m", C.c_void_p), ("u", C.c_void_p), ("h", C.c_void_p), ("eps", C.c_void_p),
                ("alpha", C.c_void_p), ("alpha_u", C.c_void_p)]


class EvolParams(C.Structure):
    _fields_ = [("theta", C.c_float), ("n_nei_sph", C.c_float), ("n_nei_grav", C.c_float),
                ("gamma", C.c_float), ("alpha", C.c_float), ("beta", C.c_float), ("G", C.c_float),
                ("gravity", C.c_int), ("sph", C.c_int), ("adaptive_softening", C.c_int),
                ("use_tc_gradient", C.c_int), ("periodic_mask", C.c_int),
                ("periodic_lo", C.c_float * 3), ("periodic_hi", C.c_float * 3),
                ("precision", C.c_int), ("leaf_size", C.c_int), ("group_size", C.c_int),
                ("visc_form", C.c_int), ("balsara", C.c_int), ("balsara_eta", C.c_float),
                ("variable_alpha", C.c_int), ("alpha_min", C.c_float), ("alpha_tau", C.c_float),
                ("alpha_source", C.c_float), ("conduction", C.c_int), ("cond_vsig", C.c_int),
                ("cond_source", C.c_int), ("alpha_u_min", C.c_float), ("sph_scheme", C.c_int),
                ("length_group", C.c_int)]


class EvolIntegrator(C.Structure):
    _fields_ = [("eta_acc", C.c_float), ("eta_vel", C.c_float), ("eta_av", C.c_float), ("eta_courant", C.c_float),
                ("eta_u", C.c_float), ("dt_min", C.c_float), ("dt_max", C.c_float),
                ("predicted_velocity", C.c_int), ("predict_lengths", C.c_int)]


class EvolBins(C.Structure):
    _fields_ = [("crit", EvolIntegrator), ("max_bin", C.c_int), ("wake_factor", C.c_float)]


class EvolOutputs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("ax", "ay", "az", "pot", "rho", "P", "c", "omega", "zeta",
                                           "dudt", "ups", "X", "dalpha", "dalpha_u")]


OUTPUT_FIELDS = [f[0] for f in EvolOutputs._fields_]
PARTICLE_FIELDS = ["x", "y", "z", "vx", "vy", "vz", "m", "u", "h", "eps", "alpha", "alpha_u"]

_lib = None


def lib():
    """Load libevol.so (raises if it has not been built: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_0912_1786_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, pp = C.c_void_p, C.POINTER
        L.evol_create.argtypes = [pp(vp), C.c_int64, vp]
        L.evol_destroy.argtypes = [vp]
        for name in ("evol_build_tree",):
            getattr(L, name).argtypes = [vp, pp(EvolParticles), pp(EvolParams)]
        for name in ("evol_sph_density", "evol_gravity", "evol_sph_forces", "evol_step", "evol_step_host"):
            getattr(L, name).argtypes = [vp, pp(EvolParticles), pp(EvolParams), pp(EvolOutputs)]
        L.evol_step_batched.argtypes = [vp, C.POINTER(C.c_int64), C.c_int, pp(EvolParticles), pp(EvolParams),
                                         pp(EvolOutputs)]
        for name in ("evol_autotune", "evol_autotune_length_group"):
            getattr(L, name).argtypes = [vp, pp(EvolParticles), pp(EvolParams), pp(EvolOutputs), C.POINTER(C.c_int),
                                         C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_float)]
        L.evol_autotune_batched.argtypes = [vp, C.POINTER(C.c_int64), C.c_int, pp(EvolParticles), pp(EvolParams),
                                            pp(EvolOutputs), C.c_int, C.POINTER(C.c_int), C.c_int, C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_float)]
        L.evol_kdk.argtypes = [vp, pp(EvolParticles), pp(EvolParams), pp(EvolOutputs), C.c_float, C.c_int]
        L.evol_run.argtypes = [vp, pp(EvolParticles), pp(EvolParams), pp(EvolIntegrator), pp(EvolOutputs), C.c_int,
                               pp(C.c_double), pp(C.c_float)]
        L.evol_run_bins.argtypes = [vp, pp(EvolParticles), pp(EvolParams), pp(EvolBins), pp(EvolOutputs), C.c_int,
                                    pp(C.c_double), pp(C.c_int64)]
        L.evol_sync.argtypes = [vp]
        L.evol_get_diagnostics.argtypes = [vp, pp(C.c_double)]
        L.evol_get_timings.argtypes = [vp, pp(C.c_float)]
        L.evol_get_counters.argtypes = [vp, pp(C.c_uint64)]
        L.evol_get_debug.argtypes = [vp, C.c_int, vp, C.c_int64]
        L.evol_get_debug.restype = C.c_int64
        L.evol_set_check_mode.argtypes = [vp, C.c_int]
        L.evol_set_stack_limit.argtypes = [vp, C.c_int64]
        L.evol_sort_keys_noalloc.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp, vp]
        L.evol_fp32_peak.argtypes = [C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_float)]
        L.evol_strerror.argtypes = [C.c_int]
        L.evol_strerror.restype = C.c_char_p
        _lib = L
    return _lib


class EvolError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {lib().evol_strerror(code).decode()} ({code})")
        self.code = code


def _check(code, where):
    if code != EVOL_OK:
        raise EvolError(code, where)
    return code


def _ptr(t):
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):           # numpy (host) arrays for evol_step_host
        return t.ctypes.data
    return int(t)


def make_params(p) -> EvolParams:
    """EvolParams from any object with the fields of workloads.Params."""
    e = EvolParams()
    for k in ("theta", "n_nei_sph", "n_nei_grav", "gamma", "alpha", "beta", "G"):
        setattr(e, k, float(getattr(p, k)))
    e.gravity = int(p.gravity)
    e.sph = int(p.sph)
    e.adaptive_softening = int(p.adaptive_softening)
    e.use_tc_gradient = int(getattr(p, "use_tc_gradient", 1))
    e.periodic_mask = int(getattr(p, "periodic_mask", 0))
    e.periodic_lo = (C.c_float * 3)(*[float(v) for v in getattr(p, "periodic_lo", (0, 0, 0))])
    e.periodic_hi = (C.c_float * 3)(*[float(v) for v in getattr(p, "periodic_hi", (1, 1, 1))])
    e.precision = int(getattr(p, "precision", EVOL_FP32_PLAIN))
    e.leaf_size = int(getattr(p, "leaf_size", 8))
    e.group_size = int(getattr(p, "group_size", 32))
    # dissipation variants (defaults: the paper's constants, every variant off)
    for k, d in (("visc_form", 0), ("balsara", 0), ("variable_alpha", 0), ("conduction", 0), ("cond_vsig", 0),
                 ("cond_source", 0), ("sph_scheme", 0), ("length_group", 0)):
        setattr(e, k, int(getattr(p, k, d)))
    for k, d in (("balsara_eta", 1e-4), ("alpha_min", 0.01), ("alpha_tau", 0.1), ("alpha_source", 0.75),
                 ("alpha_u_min", 0.0)):
        setattr(e, k, float(getattr(p, k, d)))
    return e


def make_particles(n, n_gas, arrays: dict) -> EvolParticles:
    e = EvolParticles()
    e.n, e.n_gas = int(n), int(n_gas)
    for k in PARTICLE_FIELDS:
        setattr(e, k, _ptr(arrays.get(k)))
    return e


def make_outputs(outputs: dict | None) -> EvolOutputs:
    e = EvolOutputs()
    for k in OUTPUT_FIELDS:
        setattr(e, k, _ptr((outputs or {}).get(k)))
    return e


# ---- the C entry points, same names -------------------------------------------------------
def evol_create(max_n: int, stream=None):
    ctx = C.c_void_p()
    s = None if stream is None else _ptr_stream(stream)
    _check(lib().evol_create(C.byref(ctx), int(max_n), s), "evol_create")
    return ctx


def _ptr_stream(stream):
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def evol_destroy(ctx):
    _check(lib().evol_destroy(ctx), "evol_destroy")


def evol_build_tree(ctx, particles: EvolParticles, params: EvolParams):
    return _check(lib().evol_build_tree(ctx, C.byref(particles), C.byref(params)), "evol_build_tree")


def evol_sph_density(ctx, particles, params, outputs):
    return _check(lib().evol_sph_density(ctx, C.byref(particles), C.byref(params), C.byref(outputs)),
                  "evol_sph_density")


def evol_gravity(ctx, particles, params, outputs):
    return _check(lib().evol_gravity(ctx, C.byref(particles), C.byref(params), C.byref(outputs)), "evol_gravity")


def evol_sph_forces(ctx, particles, params, outputs):
    return _check(lib().evol_sph_forces(ctx, C.byref(particles), C.byref(params), C.byref(outputs)),
                  "evol_sph_forces")


def evol_step(ctx, particles, params, outputs):
    return _check(lib().evol_step(ctx, C.byref(particles), C.byref(params), C.byref(outputs)), "evol_step")


def evol_step_host(ctx, particles, params, outputs):
    return _check(lib().evol_step_host(ctx, C.byref(particles), C.byref(params), C.byref(outputs)),
                  "evol_step_host")


def evol_step_batched(ctx, sys_offsets, particles, params, outputs):
    """Independent systems in one step; sys_offsets: host sequence of nsys + 1 particle offsets."""
    offs = (C.c_int64 * len(sys_offsets))(*[int(v) for v in sys_offsets])
    return _check(lib().evol_step_batched(ctx, offs, len(sys_offsets) - 1, C.byref(particles), C.byref(params),
                                          C.byref(outputs)), "evol_step_batched")


def evol_autotune(ctx, particles, params, outputs, candidates=None, reps=3):
    """Fastest leaf size for these particles; returns (best_leaf, {leaf: median ms})."""
    cand = list(candidates) if candidates is not None else [4, 8, 12, 16, 24, 32]
    carr = (C.c_int * len(cand))(*cand)
    ms = (C.c_float * len(cand))()
    best = C.c_int()
    _check(lib().evol_autotune(ctx, C.byref(particles), C.byref(params), C.byref(outputs), carr, len(cand),
                               int(reps), C.byref(best), ms), "evol_autotune")
    return best.value, dict(zip(cand, list(ms)))


def evol_autotune_length_group(ctx, particles, params, outputs, candidates=None, reps=3):
    """Fastest group size of the length solves at these parameters; returns (best, {size: median ms})."""
    cand = list(candidates) if candidates is not None else [4, 8, 16, 32]
    carr = (C.c_int * len(cand))(*cand)
    ms = (C.c_float * len(cand))()
    best = C.c_int()
    _check(lib().evol_autotune_length_group(ctx, C.byref(particles), C.byref(params), C.byref(outputs), carr,
                                            len(cand), int(reps), C.byref(best), ms), "evol_autotune_length_group")
    return best.value, dict(zip(cand, list(ms)))


def evol_autotune_batched(ctx, sys_offsets, particles, params, outputs, which=EVOL_TUNE_LEAF_SIZE, candidates=None,
                          reps=3):
    """Fastest leaf size (which = EVOL_TUNE_LEAF_SIZE) or length-solve group size
    (EVOL_TUNE_LENGTH_GROUP) for a batched step over these systems; returns (best, {value: median ms})."""
    if candidates is None:
        candidates = [4, 8, 12, 16, 24, 32] if which == EVOL_TUNE_LEAF_SIZE else [4, 8, 16, 32]
    cand = list(candidates)
    offs = (C.c_int64 * len(sys_offsets))(*[int(v) for v in sys_offsets])
    carr = (C.c_int * len(cand))(*cand)
    ms = (C.c_float * len(cand))()
    best = C.c_int()
    _check(lib().evol_autotune_batched(ctx, offs, len(sys_offsets) - 1, C.byref(particles), C.byref(params),
                                       C.byref(outputs), int(which), carr, len(cand), int(reps), C.byref(best), ms),
           "evol_autotune_batched")
    return best.value, dict(zip(cand, list(ms)))


def evol_kdk(ctx, particles, params, outputs, dt: float, nsteps: int):
    """Fixed-step kick-drift-kick; updates the particle arrays in place (device tensors)."""
    return _check(lib().evol_kdk(ctx, C.byref(particles), C.byref(params), C.byref(outputs), float(dt), int(nsteps)),
                  "evol_kdk")


def make_integrator(eta_acc=0.1, eta_vel=0.0, eta_av=0.0, eta_courant=0.1, eta_u=0.1, dt_min=0.0, dt_max=1.0,
                    predicted_velocity=1, predict_lengths=1) -> EvolIntegrator:
    e = EvolIntegrator()
    e.eta_acc, e.eta_vel, e.eta_av, e.eta_courant, e.eta_u = (float(eta_acc), float(eta_vel), float(eta_av),
                                                              float(eta_courant), float(eta_u))
    e.dt_min, e.dt_max = float(dt_min), float(dt_max)
    e.predicted_velocity, e.predict_lengths = int(predicted_velocity), int(predict_lengths)
    return e


def evol_run(ctx, particles, params, integrator, outputs, nsteps: int, time: float = 0.0):
    """Global-time-step KDK on the device; updates the particle arrays in place.  Returns
    (time after the steps, last time step)."""
    t = C.c_double(float(time))
    dt = C.c_float()
    _check(lib().evol_run(ctx, C.byref(particles), C.byref(params), C.byref(integrator), C.byref(outputs),
                          int(nsteps), C.byref(t), C.byref(dt)), "evol_run")
    return t.value, dt.value


def make_bins(max_bin=6, wake_factor=0.0, **crit) -> EvolBins:
    """EvolBins: crit takes make_integrator's keywords (dt_max is the largest step)."""
    b = EvolBins()
    b.crit = make_integrator(**crit)
    b.max_bin = int(max_bin)
    b.wake_factor = float(wake_factor)
    return b


def evol_run_bins(ctx, particles, params, bins, outputs, nlargest: int, time: float = 0.0):
    """Individual power-of-two time steps on the device for nlargest largest steps; updates the
    particle arrays in place.  Returns (time, [system steps, evaluations, wake-ups, clamped])."""
    t = C.c_double(float(time))
    st = (C.c_int64 * 4)()
    _check(lib().evol_run_bins(ctx, C.byref(particles), C.byref(params), C.byref(bins), C.byref(outputs),
                               int(nlargest), C.byref(t), st), "evol_run_bins")
    return t.value, list(st)


def evol_sync(ctx, raise_on_error=True):
    rc = lib().evol_sync(ctx)
    if raise_on_error:
        _check(rc, "evol_sync")
    return rc


def evol_get_diagnostics(ctx):
    out = (C.c_double * 16)()
    _check(lib().evol_get_diagnostics(ctx, out), "evol_get_diagnostics")
    return list(out)


def evol_get_timings(ctx):
    out = (C.c_float * 5)()
    _check(lib().evol_get_timings(ctx, out), "evol_get_timings")
    return list(out)


def evol_get_counters(ctx):
    out = (C.c_uint64 * 32)()
    _check(lib().evol_get_counters(ctx, out), "evol_get_counters")
    return list(out)


def evol_set_check_mode(ctx, on: bool):
    _check(lib().evol_set_check_mode(ctx, int(bool(on))), "evol_set_check_mode")


def evol_fp32_peak(iters: int = 20000):
    """Measured FP32 throughput of the current device: (scalar TFLOP/s, packed two-wide TFLOP/s,
    scalar kernel ms)."""
    t, t2, ms = C.c_double(), C.c_double(), C.c_float()
    _check(lib().evol_fp32_peak(int(iters), C.byref(t), C.byref(t2), C.byref(ms)), "evol_fp32_peak")
    return t.value, t2.value, ms.value


def evol_set_stack_limit(ctx, entries: int):
    _check(lib().evol_set_stack_limit(ctx, int(entries)), "evol_set_stack_limit")


EVOL_NOALLOC_MAX_N = 65536


def evol_sort_keys_noalloc(n, x, y, z, keys_sorted, perm, cube=None, stream=None):
    """Allocation-free key + sort stage (device tensors in, device tensors out)."""
    s = None if stream is None else _ptr_stream(stream)
    return _check(lib().evol_sort_keys_noalloc(int(n), _ptr(x), _ptr(y), _ptr(z), _ptr(keys_sorted), _ptr(perm),
                                               _ptr(cube), s), "evol_sort_keys_noalloc")


def evol_get_debug(ctx, what: int, dtype):
    """Copy one debug array; dtype is the numpy element type of `what`."""
    import numpy as np
    cnt = lib().evol_get_debug(ctx, int(what), None, 0)
    if cnt < 0:
        raise EvolError(int(cnt), "evol_get_debug")
    out = np.empty(int(cnt), dtype=dtype)
    rc = lib().evol_get_debug(ctx, int(what), out.ctypes.data, out.nbytes)
    if rc < 0:
        raise EvolError(int(rc), "evol_get_debug")
    return out


@dataclass
class Step:
    """Convenience holder: one context plus the marshalled structs for one particle set."""

    ctx: object
    particles: EvolParticles
    params: EvolParams
    outputs: EvolOutputs
    keep: tuple = ()

    def run(self):
        evol_step(self.ctx, self.particles, self.params, self.outputs)

    def sync(self, raise_on_error=True):
        return evol_sync(self.ctx, raise_on_error)
