#!/usr/bin/env python3
"""Benchmark of the tree + SPH force step on GB300 (one JSON line on stdout).

Default workload: the mixed-species system -- 2^21 Hernquist dark-matter particles plus 2^20
gas particles in a rho ~ 1/r sphere (gas fraction 0.1, u = 0.05, theta = 0.5, 50 neighbours),
one full force step (tree build + eps solve + h solve + gravity/SPH walk) per step, synthetic
seeded data.  `value` = particles per second of the whole step with inputs resident in HBM;
`e2e` = the same through evol_step_host with host buffers (copies inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c1|c2|c3|c4|c5] [--precision plain|mixed]

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own GPU
(the single-system step does not shard); the reported value is the sum over ranks divided by
the slowest rank's time.  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Algorithmic FP32 operations per interaction of the force walk, counted from the source
# (FFMA = 2, FADD/FMUL = 1, MUFU = 1): far node monopole + quadrupole + potential; Newtonian
# particle pair (r >= 2 max(eps_i, eps_j): point-mass force and potential); softened particle pair
# (both softened kernels, potential, adaptive-softening correction); SPH pair (pressure with the
# grad-h factors, Monaghan viscosity, du/dt).
FLOPS_FAR = 53
FLOPS_PP_NEWTON = 19
FLOPS_PP_SOFT = 89
FLOPS_SPH = 85
# Algorithmic DRAM bytes per particle of the tree build (one pass over each kernel's inputs and
# outputs): bbox 12, keys 12 + 12, 8 radix passes x (histogram 8 + scatter 24), permute 40 + 44,
# common prefixes 8 + 5, node counts 5, their scan 16, moments 20; plus per node: fill 16,
# link 80, moments 150.
BUILD_BYTES_PER_PARTICLE = 12 + 24 + 8 * 32 + 84 + 13 + 5 + 16 + 20
BUILD_BYTES_PER_NODE = 16 + 80 + 150


# Measured copy bandwidth of the GB300s (GB/s), the build's HBM roofline denominator.
def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6766.0


HBM_PEAK_GBS = _hbm_peak()
# DRAM bytes per launch of the production walk (dram__bytes_read.sum + dram__bytes_write.sum of a
# one-pass ncu capture of the full-size workload at that leaf size); other workloads and leaf sizes
# report null
WALK_TRAFFIC = {("c3", 16): 497.0e6 + 100.1e6, ("c3", 24): 451.9e6 + 95.1e6, ("c3", 32): 434.1e6 + 93.0e6}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def make_workload(name: str):
    from paper_0912_1786_gb300 import workloads as W
    if name == "c1":
        return W.evrard_sphere(4096, seed=1), "evrard_sphere_4096"
    if name == "c2":
        return W.plummer(1 << 20, seed=2, params=W.Params(theta=0.6, sph=0, n_nei_grav=32.0, leaf_size=8)), \
            "plummer_2^20_theta0.6_gravity_only"
    # the mixed-species workloads default to leaf 24, the size the autotuner picks for them on GB300
    # (the FP64 oracle of the reference arm uses the same value)
    if name == "c3":
        return W.hernquist_gas(n_dm=1 << 21, n_gas=1 << 20, seed=3, params=W.Params(leaf_size=24)), \
            "hernquist_2^21_dm+2^20_gas"
    if name == "c3s":      # one eighth of c3, for profiler captures
        return W.hernquist_gas(n_dm=1 << 18, n_gas=1 << 17, seed=3, params=W.Params(leaf_size=24)), \
            "hernquist_2^18_dm+2^17_gas"
    if name == "c4":
        return W.shock_tube(seed=4), "shock_tube_1046250_periodic_yz"
    if name == "c5":
        return W.ensemble(64, seed=5), "ensemble_64_spheres_N_2^10..2^17"
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd[1:1] = ["-i", self.gpu_id]
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def current_mhz(self):
        """Most recent SM clock sample (MHz), or None."""
        try:
            self.f.flush()
            rows = [ln.split(",") for ln in open(self.path) if ln.count(",") >= 7]
            return float(rows[-1][0]) if rows else None
        except Exception:
            return None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, flags in rows for k, v in enumerate(flags) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def gpu_uuid(torch, dev):
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def oracle_state(w, leaf):
    """The FP64 oracle's tree and lengths of every particle for workload w (eps of all particles,
    h, rho, Omega*, zeta, P, c of the gas), as the force pass needs them."""
    import oracle
    p = w.params
    lib = oracle.lib()
    tree = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, leaf)
    n, ng = w.n, w.n_gas
    st = {}
    if p.gravity and p.adaptive_softening:
        eps, _, ups, X, _ = tree.solve_lengths(1, p.n_nei_grav, guess=w.eps, params=p)
        st.update(eps=eps, ups=ups, X=X)
    elif p.gravity:
        st.update(eps=w.eps.astype(np.float64), ups=np.ones(n), X=np.zeros(n))
    if p.sph and ng:
        h, nh, rho, om, zeta = tree.solve_lengths(0, p.n_nei_sph, guess=w.h, idx=np.arange(ng), params=p)
        P, c = np.zeros(n), np.zeros(n)
        lib.orc_eos(n, float(p.gamma), np.ascontiguousarray(rho), np.ascontiguousarray(w.u, np.float64), P, c)
        P[ng:] = 0
        c[ng:] = 0
        st.update(h=h, rho=rho, omega=om, zeta=zeta, P=P, c=c, n_h=nh)
    st.update(vx=w.vx.astype(np.float64), vy=w.vy.astype(np.float64), vz=w.vz.astype(np.float64))
    return tree, st


def oracle_sample(w, budget_s=25.0, seed=7, leaf=None, state=None):
    """Bounded timing of the FP64 oracle on workload w: a full tree build, the eps and h solves
    on seeded samples of particles and the force walk on a seeded sample, each scaled to its
    per-particle rate.  Returns (particles/s, cores, description)."""
    import oracle
    p = w.params
    leaf = leaf or p.leaf_size
    lib = oracle.lib()
    cores = int(lib.orc_num_threads())
    t0 = time.perf_counter()
    tree = oracle.OracleTree(w.x, w.y, w.z, w.m, w.n_gas, leaf)
    t_build = time.perf_counter() - t0
    n, ng = w.n, w.n_gas
    rng = np.random.default_rng(seed)
    per = 0.0
    desc = [f"leaf {leaf}: tree build of all {n} particles {t_build:.2f}s"]
    s_e = min(n, 60000)
    s_h = min(ng, 30000)
    if p.gravity and p.adaptive_softening:
        idx = np.sort(rng.choice(n, s_e, replace=False))
        t0 = time.perf_counter()
        tree.solve_lengths(1, p.n_nei_grav, guess=w.eps, idx=idx, params=p)
        te = time.perf_counter() - t0
        per += te / s_e * n
        desc.append(f"eps solve {s_e} sampled ({te:.2f}s)")
    if p.sph and ng:
        idx = np.sort(rng.choice(ng, s_h, replace=False))
        t0 = time.perf_counter()
        tree.solve_lengths(0, p.n_nei_sph, guess=w.h, idx=idx, params=p)
        th = time.perf_counter() - t0
        per += th / s_h * ng
        desc.append(f"h solve {s_h} sampled ({th:.2f}s)")
    # neighbour lengths for the force sample come from the oracle's own solve of every particle
    # (set-up, not timed)
    st = (state or oracle_state(w, leaf))[1]
    s_f = min(n, 2000)
    idx = np.sort(rng.choice(n, s_f, replace=False))
    t0 = time.perf_counter()
    tree.forces(p, st, idx=idx)
    tf = time.perf_counter() - t0
    # grow the force sample while the budget allows
    if tf < budget_s / 4 and s_f < n:
        s_f2 = int(min(n, s_f * max(2.0, budget_s / 4 / max(tf, 1e-3))))
        idx = np.sort(rng.choice(n, s_f2, replace=False))
        t0 = time.perf_counter()
        tree.forces(p, st, idx=idx)
        tf = time.perf_counter() - t0
        s_f = s_f2
    per += tf / s_f * n
    desc.append(f"force walk {s_f} sampled ({tf:.2f}s)")
    total = t_build + per
    return n / total, cores, "; ".join(desc) + f"; scaled to {n} particles: {total:.1f}s per step"


# Tolerances the force step is held to against the FP64 oracle (median / 99th percentile of the
# relative error), and the explanation margin of an interaction-set mismatch (relative to the
# threshold plus the particle's coordinate scale).
TOL_MEDIAN, TOL_P99, EXPLAIN_MARGIN, CANCEL_FLOOR = 1e-5, 1e-4, 1e-6, 1e-2


def _rel(got, ref, scale=None):
    """Plain relative error statistics; with `scale`, results below CANCEL_FLOOR of their terms'
    magnitude sum are counted apart and judged by |d| / scale."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    d = np.linalg.norm(got - ref, axis=1) if got.ndim == 2 else np.abs(got - ref)
    r = np.linalg.norm(ref, axis=1) if ref.ndim == 2 else np.abs(ref)
    fl = np.zeros(len(d), bool) if scale is None else r < CANCEL_FLOOR * np.asarray(scale)
    e = d[~fl] / np.maximum(r[~fl], 1e-300)
    out = {"median": float(np.median(e)) if e.size else 0.0, "p99": float(np.percentile(e, 99)) if e.size else 0.0,
           "n": int(len(d))}
    if fl.any():
        fe = d[fl] / np.asarray(scale)[fl]
        out.update(n_floor=int(fl.sum()), floor_p99=float(np.percentile(fe, 99)))
    return out


def form_errors(g, ref, idx, w):
    """Errors of one GPU form (g: caller-order arrays incl. 'hashes') against the oracle on the
    sampled particles idx (ref: the oracle's results)."""
    gi = idx[idx < w.n_gas]
    A = lambda x: np.stack([x["ax"], x["ay"], x["az"]], 1)
    e = {"acc": _rel(A(g)[idx], A(ref)[idx], ref["aabs"][idx])}
    if w.params.gravity:
        e["pot"] = _rel(g["pot"][idx], ref["pot"][idx])
        if w.params.adaptive_softening:
            e["eps"] = _rel(g["eps"][idx], ref["eps"][idx])
    if w.params.sph and len(gi):
        e["h"] = _rel(g["h"][gi], ref["h"][gi])
        e["rho"] = _rel(g["rho"][gi], ref["rho"][gi])
        if np.any(w.vx != 0):
            e["dudt"] = _rel(g["dudt"][gi], ref["dudt"][gi], ref["duabs"][gi])
    if "hashes" in g:
        oh = np.stack([ref["hfar"], ref["hnear"], ref["hsph"]], 1)[idx]
        bad = np.any(g["hashes"][idx] != oh, axis=1)
        mg = ref["margin"][idx][bad]
        e["set_mismatches"] = int(bad.sum())
        e["set_mismatches_explained"] = int((mg < EXPLAIN_MARGIN).sum())
    ok = all(v["median"] <= TOL_MEDIAN and v["p99"] <= TOL_P99 for k, v in e.items() if isinstance(v, dict))
    e["within_tolerance"] = bool(ok and e.get("set_mismatches", 0) == e.get("set_mismatches_explained", 0))
    return e


def plummer_checks(w, g, ostate, dist_seed=12, nsample=1024):
    """Context for the Plummer sphere (G = M = a = 1): shell averages of the radial acceleration
    against the closed form -r (1 + r^2)^(-3/2) with their Poisson noise, and the tree's error
    against the oracle's direct sum (theta = 0) on a seeded sample."""
    import copy
    P = np.stack([w.x, w.y, w.z], 1).astype(np.float64)
    a = np.stack([g["ax"], g["ay"], g["az"]], 1)
    r = np.linalg.norm(P, axis=1)
    ar = (a * P).sum(1) / r
    shells = []
    edges = np.array([0.2, 0.4, 0.7, 1.0, 1.5, 2.5, 4.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        rs = r[sel]
        cf = np.mean(-rs * (1 + rs ** 2) ** -1.5)
        shells.append({"r": [float(lo), float(hi)], "count": int(sel.sum()),
                       "rel_diff": float(abs(ar[sel].mean() - cf) / abs(cf)), "poisson": float(1 / np.sqrt(sel.sum()))})
    p0 = copy.copy(w.params)
    p0.theta = 0.0
    idx = np.sort(np.random.default_rng(dist_seed).choice(w.n, min(w.n, nsample), replace=False))
    ref = ostate[0].forces(p0, ostate[1], idx=idx)
    ad = np.stack([ref["ax"], ref["ay"], ref["az"]], 1)[idx]
    e = np.linalg.norm(a[idx] - ad, axis=1) / np.linalg.norm(ad, axis=1)
    return {"closed_form_shells": shells,
            "tree_vs_direct_sum": {"median": float(np.median(e)), "p99": float(np.percentile(e, 99)),
                                   "n": int(len(idx)), "theta": float(w.params.theta)}}


def gpu_check_step(E, ctx, ds, offsets=None):
    """One more step with interaction-set hashes recorded; caller-order numpy results."""
    E.evol_set_check_mode(ctx, True)
    ds.reset_lengths()
    if offsets is None:
        E.evol_step(ctx, ds.particles, ds.params, ds.outputs)
    else:
        E.evol_step_batched(ctx, offsets, ds.particles, ds.params, ds.outputs)
    E.evol_sync(ctx)
    g = ds.numpy()
    g["hashes"] = E.evol_get_debug(ctx, E.EVOL_DBG_HASHES, np.uint64).reshape(-1, 3)
    E.evol_set_check_mode(ctx, False)
    return g


def run_reference(args):
    """--impl reference: the FP64 CPU oracle, as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, wname = make_workload(args.workload)
    vals = []
    desc = ""
    cores = 1
    for k in range(args.warmup + args.steps):
        v, cores, desc = oracle_sample(w, budget_s=args.ref_budget, seed=100 + k)
        if k >= args.warmup:
            vals.append(v)
    v = statistics.mean(vals)
    line = {"metric": "force-step particles/s (tree gravity+SPH)", "value": v, "unit": "particles/s",
            "impl": "reference", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wname, "n": w.n, "n_gas": w.n_gas, "theta": w.params.theta,
                       "n_nei": w.params.n_nei_sph, "leaf_size": int(w.params.leaf_size)},
            "cpu_baseline": {"value": v, "unit": "particles/s", "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line), flush=True)
    return 0


def time_steps(torch, dev, stream, fn, steps):
    """CUDA-event time of `steps` calls of fn on `stream` (ms)."""
    torch.cuda.synchronize(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fn()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    return t0.elapsed_time(t1)


def other_forms(torch, dev, stream, E, DeviceSet, w, steps, precision_used, leaf, group=0):
    """Throughput of the other precision form (same workload) and, for an ensemble, of one
    launch per system; particles/s each.  Also returns each form's results (caller order, with
    interaction-set hashes for the precision form) for the accuracy comparison."""
    forms, results = {}, {}
    other = E.EVOL_FP32_MIXED if precision_used == E.EVOL_FP32_PLAIN else E.EVOL_FP32_PLAIN
    ds = DeviceSet(w, device=str(dev), precision=other)
    ds.params.leaf_size = leaf
    ds.params.length_group = group
    ctx = E.evol_create(w.n, stream.cuda_stream)
    try:
        if w.sys_offsets is not None:
            offs = [int(v) for v in w.sys_offsets]
            run = lambda: (ds.reset_lengths(), E.evol_step_batched(ctx, offs, ds.particles, ds.params, ds.outputs))
        else:
            run = lambda: (ds.reset_lengths(), E.evol_step(ctx, ds.particles, ds.params, ds.outputs))
        for _ in range(2):
            run()
        E.evol_sync(ctx)
        ms = time_steps(torch, dev, stream, run, steps)
        E.evol_sync(ctx)
        name = "mixed" if other == E.EVOL_FP32_MIXED else "plain"
        forms[name] = w.n * steps / (ms / 1e3)
        results[name] = gpu_check_step(E, ctx, ds, [int(v) for v in w.sys_offsets] if w.sys_offsets is not None else None)
    finally:
        E.evol_destroy(ctx)
    if w.sys_offsets is not None:
        # the same ensemble as one evol_step per system, each on its own slice of the arrays
        from paper_0912_1786_gb300 import evol as E2
        ds = DeviceSet(w, device=str(dev), precision=precision_used)
        ds.params.leaf_size = leaf
        ds.params.length_group = group
        offs = [int(v) for v in w.sys_offsets]
        ctxs, parts = [], []
        try:
            for k in range(len(offs) - 1):
                b, e = offs[k], offs[k + 1]
                arr = {key: (t[b:e] if key not in ("u", "h") or e <= w.n_gas else t[b:min(e, w.n_gas)])
                       for key, t in ds.inp.items()}
                outs = {key: t[b:e] for key, t in ds.out.items()}
                ctxs.append(E2.evol_create(max(e - b, 1), stream.cuda_stream))
                parts.append((E2.make_particles(e - b, e - b, arr), E2.make_outputs(outs)))
            run = lambda: [E2.evol_step(c, pp, ds.params, oo) for c, (pp, oo) in zip(ctxs, parts)]
            for _ in range(2):
                ds.reset_lengths()
                run()
            torch.cuda.synchronize(dev)
            ms = time_steps(torch, dev, stream, lambda: (ds.reset_lengths(), run()), steps)
            forms["per_system_launches"] = w.n * steps / (ms / 1e3)
            ds.reset_lengths()
            run()
            torch.cuda.synchronize(dev)
            results["per_system_launches"] = ds.numpy()
        finally:
            for c in ctxs:
                E2.evol_destroy(c)
    return forms, results


DISSIPATION_ALL = dict(visc_form=1, balsara=1, variable_alpha=1, conduction=1)


def ewald_block(torch, dev, stream, E, DeviceSet, n, steps):
    """Periodic gravity (Sect. 4.3): the same particles (a clustered periodic box, gravity only,
    adaptive softening) once with the Ewald correction and once without periodicity; particles/s,
    walk time and far-node interactions of each, and their ratio (the paper: the interpolation
    almost doubles the tree time)."""
    import dataclasses
    from paper_0912_1786_gb300 import workloads as W
    wp = W.periodic_box(n, seed=6)
    wo = W.Workload(wp.name, wp.x, wp.y, wp.z, wp.vx, wp.vy, wp.vz, wp.m, wp.u, wp.h, wp.eps, n_gas=0,
                    params=dataclasses.replace(wp.params, periodic_mask=0))
    out = {"input": f"periodic_box n={n} (half uniform, half three clumps), gravity only, adaptive eps (32)"}
    for name, ww in (("ewald", wp), ("open", wo)):
        ds = DeviceSet(ww, device=str(dev))
        ctx = E.evol_create(ww.n, stream.cuda_stream)
        try:
            run = lambda: (ds.reset_lengths(), E.evol_step(ctx, ds.particles, ds.params, ds.outputs))
            for _ in range(2):
                run()
            E.evol_sync(ctx)
            ms, walks = 0.0, []
            for _ in range(steps):
                ms += time_steps(torch, dev, stream, run, 1)
                walks.append(E.evol_get_timings(ctx)[3])
            E.evol_sync(ctx)
            cnt = E.evol_get_counters(ctx)
            out[name] = {"particles_per_s": ww.n * steps / (ms / 1e3), "ms_per_step": ms / steps,
                         "walk_ms": statistics.mean(walks), "far_interactions": int(cnt[0]),
                         "pair_interactions": int(cnt[1])}
        finally:
            E.evol_destroy(ctx)
    out["walk_time_ratio"] = out["ewald"]["walk_ms"] / out["open"]["walk_ms"]
    return out


def bins_block(torch, dev, stream, E, DeviceSet, n):
    """Individual power-of-two time steps (Sect. 4.2.1) on an Evrard sphere with a hot core (a wide
    spread of Courant steps): one largest step of evol_run_bins against the same span taken by the
    global step at the finest step in use, estimated as (system steps + 1) force steps of all
    particles."""
    from paper_0912_1786_gb300 import workloads as W
    w = W.hot_core(W.evrard_sphere(n, seed=21, sigma_v=0.05))
    ds = DeviceSet(w, device=str(dev))
    ctx = E.evol_create(w.n, stream.cuda_stream)
    K, dt_max = 10, 0.0625
    try:
        b = E.make_bins(K, 4.0, eta_acc=0.1, eta_courant=0.2, eta_u=0.2, dt_max=dt_max, predicted_velocity=1,
                        predict_lengths=0)
        E.evol_run_bins(ctx, ds.particles, ds.params, b, ds.outputs, 1)           # graph recording
        E.evol_sync(ctx)
        # the same arrays (the recorded graph holds their addresses) back at the start
        for k, a in w.arrays().items():
            t = ds.inp[k]
            t.copy_(torch.from_numpy(np.ascontiguousarray(a[: t.numel()], np.float32)).to(t.device))
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, st = E.evol_run_bins(ctx, ds.particles, ds.params, b, ds.outputs, 1)
        torch.cuda.synchronize(dev)
        t_bins = time.perf_counter() - t0
        E.evol_sync(ctx)
        # one force step of every particle, the unit of the global-step estimate
        ds3 = DeviceSet(w, device=str(dev))
        run = lambda: (ds3.reset_lengths(), E.evol_step(ctx, ds3.particles, ds3.params, ds3.outputs))
        run()
        E.evol_sync(ctx)
        ms_step = time_steps(torch, dev, stream, run, 3) / 3
    finally:
        E.evol_destroy(ctx)
    glob = (st[0] + 1) * ms_step / 1e3
    return {"input": f"evrard_sphere n={n} with a hot core (u x (1 + 30 exp(-(r/0.2)^2))), sigma_v 0.05",
            "max_bin": K, "dt_max": dt_max, "wake_factor": 4.0,
            "system_steps": st[0], "particle_evaluations": st[1], "wakeups": st[2], "criteria_below_tick": st[3],
            "wall_s": t_bins, "evaluations_per_s": st[1] / t_bins,
            "global_step_estimate_s": glob, "speedup_vs_global_step": glob / t_bins,
            "note": "wall time includes one host synchronisation per system step"}


def dissipation_form(torch, dev, stream, E, DeviceSet, w, steps, leaf, ostate, sample=2000):
    """The dissipation variants (signal-velocity viscosity, Balsara limiter, variable alpha,
    conductivity) on the same particles with seeded velocities (sigma 0.1, so that the viscosity
    acts), per-particle alpha, alpha^u and u spread: throughput of the standard form and of all
    variants on that input, their walk times, and the variants' errors against the oracle on a
    seeded sample (the oracle reuses the main form's lengths: the positions are the same)."""
    import oracle
    from paper_0912_1786_gb300 import workloads as W
    wd = W.with_dissipation(w, seed=13, sigma_v=0.1, **DISSIPATION_ALL)
    ws = W.with_dissipation(w, seed=13, sigma_v=0.1)           # same input, standard viscosity
    out = {"input": "main workload + isotropic velocities sigma 0.1 (seed 13), alpha in [0.05, 1.5], "
                    "alpha^u in [0, 1], u spread x[1/1.5, 1.5]"}
    rates = {}
    res = None
    for name, ww in (("standard", ws), ("all_variants", wd)):
        ds = DeviceSet(ww, device=str(dev))
        ds.params.leaf_size = leaf
        ctx = E.evol_create(ww.n, stream.cuda_stream)
        try:
            run = lambda: (ds.reset_lengths(), E.evol_step(ctx, ds.particles, ds.params, ds.outputs))
            for _ in range(2):
                run()
            E.evol_sync(ctx)
            walks = []
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            ms = 0.0
            for _ in range(steps):
                ms += time_steps(torch, dev, stream, run, 1)
                walks.append(E.evol_get_timings(ctx)[3])
            E.evol_sync(ctx)
            rates[name] = {"particles_per_s": ww.n * steps / (ms / 1e3), "ms_per_step": ms / steps,
                           "walk_ms": statistics.mean(walks)}
            if name == "all_variants":
                res = gpu_check_step(E, ctx, ds)
        finally:
            E.evol_destroy(ctx)
    out["rates"] = rates
    if ostate is None:
        return out
    # the oracle on the sample: lengths from the main form's solve, flow quantities with the new
    # velocities, equation of state with the new u
    tree, st0 = ostate
    ng = wd.n_gas
    gas = np.arange(ng, dtype=np.int64)
    vx, vy, vz = (getattr(wd, k).astype(np.float64) for k in ("vx", "vy", "vz"))
    divv, curl = tree.divv(0, st0["h"], st0["n_h"], st0["omega"], vx, vy, vz, idx=gas, params=wd.params, curl=True)
    P, c = np.zeros(wd.n), np.zeros(wd.n)
    oracle.lib().orc_eos(wd.n, float(wd.params.gamma), np.ascontiguousarray(st0["rho"]),
                         np.ascontiguousarray(wd.u, np.float64), P, c)
    P[ng:] = 0
    c[ng:] = 0
    fixed = {k: v for k, v in st0.items() if k not in ("vx", "vy", "vz", "n_h")}
    fixed.update(P=P, c=c, divv_h=divv, curlv_h=curl)
    sidx = np.sort(np.random.default_rng(17).choice(wd.n, min(wd.n, sample), replace=False))
    ref = oracle.force_step(wd, idx=sidx, tree=tree, fixed_lengths=fixed)
    gi = sidx[sidx < ng]
    A = lambda x: np.stack([x["ax"], x["ay"], x["az"]], 1)
    e = {"acc": _rel(A(res)[sidx], A(ref)[sidx], ref["aabs"][sidx]),
         "dudt": _rel(res["dudt"][gi], ref["dudt"][gi], ref["duabs"][gi])}
    tau = wd.params.alpha_tau * ref["state"]["h"][gi] / ref["vsig"][gi]
    rs = ref["state"]
    sc_a = np.abs(rs["alpha"][gi] - wd.params.alpha_min) / tau + wd.params.alpha_source * rs["f"][gi] * np.abs(divv[gi])
    e["dalpha"] = _rel(res["dalpha"][gi], ref["dalpha"][gi], sc_a)
    sc_u = (np.abs(rs["alpha_u"][gi] - wd.params.alpha_u_min) / tau +
            ref["state"]["h"][gi] * ref["lapabs"][gi] / np.sqrt(rs["u"][gi]))
    e["dalpha_u"] = _rel(res["dalpha_u"][gi], ref["dalpha_u"][gi], sc_u)
    oh = np.stack([ref["hfar"], ref["hnear"], ref["hsph"]], 1)[sidx]
    bad = np.any(res["hashes"][sidx] != oh, axis=1)
    e["set_mismatches"] = int(bad.sum())
    e["set_mismatches_explained"] = int((ref["margin"][sidx][bad] < EXPLAIN_MARGIN).sum())
    ok = all(v["median"] <= TOL_MEDIAN and v["p99"] <= TOL_P99 for v in e.values() if isinstance(v, dict))
    e["within_tolerance"] = bool(ok and e["set_mismatches"] == e["set_mismatches_explained"])
    e["sample"] = f"{len(sidx)} particles (seed 17), {len(gi)} gas"
    out["accuracy"] = e
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c3s", "c4", "c5"])
    ap.add_argument("--precision", default="plain", choices=["plain", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the periodic-gravity and individual-step blocks")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--leaf", type=int, default=0, help="fixed leaf size (skips the autotune)")
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--theta", type=float, default=None, help="opening angle (overrides the workload's)")
    ap.add_argument("--kdk-steps", type=int, default=0,
                    help="time this many fixed-step KDK steps (one captured graph) per bench step")
    ap.add_argument("--kdk-dt", type=float, default=1e-4)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_0912_1786_gb300 import build, evol as E
    from paper_0912_1786_gb300.device import DeviceSet

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    build.build()

    w, wname = make_workload(args.workload)
    if args.theta is not None:
        w.params.theta = float(args.theta)
        wname = f"{wname.split('_theta')[0]}_theta{args.theta:g}" if "theta" in wname else f"{wname}_theta{args.theta:g}"
    prec = E.EVOL_FP32_MIXED if args.precision == "mixed" else E.EVOL_FP32_PLAIN
    ds = DeviceSet(w, device=str(dev), precision=prec)
    stream = torch.cuda.current_stream(dev)
    ctx = E.evol_create(w.n, stream.cuda_stream)
    autotune = None
    offsets = [int(v) for v in w.sys_offsets] if w.sys_offsets is not None else None
    if args.leaf > 0:
        ds.params.leaf_size = args.leaf
    elif not args.no_autotune and offsets is None:
        best, ms = E.evol_autotune(ctx, ds.particles, ds.params, ds.outputs, candidates=[12, 16, 24, 32, 48], reps=3)
        ds.params.leaf_size = best
        # then the length solves' group size at that leaf size
        bg, msg = E.evol_autotune_length_group(ctx, ds.particles, ds.params, ds.outputs, candidates=[8, 16, 32],
                                               reps=3)
        ds.params.length_group = bg
        autotune = {"leaf_size": best, "median_ms_by_leaf": ms, "length_group": bg,
                    "median_ms_by_length_group": msg}
    elif not args.no_autotune:
        # the batched step: the same two tuners, timing the batched step over all systems
        best, ms = E.evol_autotune_batched(ctx, offsets, ds.particles, ds.params, ds.outputs,
                                           which=E.EVOL_TUNE_LEAF_SIZE, candidates=[8, 12, 16, 24], reps=3)
        ds.params.leaf_size = best
        bg, msg = E.evol_autotune_batched(ctx, offsets, ds.particles, ds.params, ds.outputs,
                                          which=E.EVOL_TUNE_LENGTH_GROUP, candidates=[8, 16, 32], reps=3)
        ds.params.length_group = bg
        autotune = {"leaf_size": best, "median_ms_by_leaf": ms, "length_group": bg,
                    "median_ms_by_length_group": msg}

    kdk_initial = {k: t.clone() for k, t in ds.inp.items()} if args.kdk_steps > 0 else None

    def one_step():
        if args.kdk_steps > 0:
            # a leapfrog run of kdk_steps steps from the initial state (restored on the device: the
            # state evolves in place and lengths carry over from step to step within the run)
            for k, t in kdk_initial.items():
                ds.inp[k].copy_(t, non_blocking=True)
            E.evol_kdk(ctx, ds.particles, ds.params, ds.outputs, args.kdk_dt, args.kdk_steps)
            return
        ds.reset_lengths()
        if offsets is not None:
            E.evol_step_batched(ctx, offsets, ds.particles, ds.params, ds.outputs)
        else:
            E.evol_step(ctx, ds.particles, ds.params, ds.outputs)

    for _ in range(args.warmup):
        one_step()
    E.evol_sync(ctx)

    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    time.sleep(0.5)
    # the FP32 roofline's denominator, measured on this GPU now (one ~80 ms FMA-chain kernel)
    peak_scalar, peak_packed, _ = E.evol_fp32_peak(20000)
    peak_tflops = max(peak_scalar, peak_packed)
    peak_clock = sampler.current_mhz()
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    walk_ms, phase = [], []
    t_start.record(stream)
    for _ in range(args.steps):
        one_step()
        rc = E.evol_sync(ctx)                     # per-step status; also lets the phase events be read
        tm = E.evol_get_timings(ctx)
        walk_ms.append(tm[3])
        phase.append(tm)
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = t_start.elapsed_time(t_end)
    clocks = sampler.stop()
    units = w.n * max(args.kdk_steps, 1)          # particles (x KDK steps) per bench step
    value, ms_max = replica_rate(dist, dev, ms, units, args.steps, world)
    diag = E.evol_get_diagnostics(ctx)
    cnt = E.evol_get_counters(ctx)               # work counters of the last timed step
    n_total = w.n * world

    # ---- e2e through the host-buffer entry point (pinned host memory) ----
    e2e = None
    if not args.no_e2e and args.kdk_steps == 0:
        host_in = {}
        for k, a in w.arrays().items():
            t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
            host_in[k] = t
        host_out = {k: torch.zeros(w.n_gas if k in ("rho", "P", "c", "omega", "zeta", "dudt") else w.n,
                                   dtype=torch.float32).pin_memory()
                    for k in ("ax", "ay", "az", "pot", "rho", "P", "c", "omega", "zeta", "dudt")}
        hp = E.make_particles(w.n, w.n_gas, host_in)
        ho = E.make_outputs(host_out)
        h2d = sum(w.n_gas * 4 if k in ("u", "h") else w.n * 4 for k in host_in)
        d2h = sum(int(t.numel()) * 4 for t in host_out.values()) + (w.n_gas + w.n) * 4
        ke = max(1, min(args.steps, 5))
        h0, e0 = host_in["h"].clone(), host_in["eps"].clone()

        def host_step():
            if offsets is None:
                E.evol_step_host(ctx, hp, ds.params, ho)
                return
            # independent systems: no host-buffer entry point takes offsets, so the inputs are
            # copied to the device set, the batched step runs, and the outputs come back
            for k, t in host_in.items():
                ds.inp[k].copy_(t[: ds.inp[k].numel()], non_blocking=True)
            E.evol_step_batched(ctx, offsets, ds.particles, ds.params, ds.outputs)
            for k, t in host_out.items():
                t.copy_(ds.out[k][: t.numel()], non_blocking=True)
            for k in ("h", "eps"):
                host_in[k][: ds.inp[k].numel()].copy_(ds.inp[k], non_blocking=True)
            E.evol_sync(ctx)

        host_step()                                        # warm (captures the host-path graph)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(ke):
            host_in["h"].copy_(h0)
            host_in["eps"].copy_(e0)
            host_step()
        te = time.perf_counter() - t0
        if dist:
            t = torch.tensor([te], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        e2e = {"value": n_total * ke / te, "unit": "particles/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": ke}

    main_form = args.precision if offsets is None else f"batched_{args.precision}"
    forms = {main_form: value}
    accuracy = None
    ostate = None
    diss_block = None
    extras = None
    if not args.no_forms:
        g_main = gpu_check_step(E, ctx, ds, offsets)
        rates, results = other_forms(torch, dev, stream, E, DeviceSet, w, max(2, min(args.steps, 5)), prec,
                                     int(ds.params.leaf_size), int(ds.params.length_group))
        forms.update(rates)
        results[main_form] = g_main
        accuracy = {}
        if rank == 0 and world == 1 and offsets is None:
            # every form against the FP64 oracle on a seeded sample of particles
            ostate = oracle_state(w, int(ds.params.leaf_size))
            sidx = np.sort(np.random.default_rng(11).choice(w.n, min(w.n, 2000), replace=False))
            ref = ostate[0].forces(w.params, ostate[1], idx=sidx)
            for k in ("eps", "h", "rho"):
                if k in ostate[1]:
                    ref[k] = ostate[1][k]
            for name, g in results.items():
                accuracy[name] = form_errors(g, ref, sidx, w)
            accuracy["sample"] = f"{len(sidx)} particles (seed 11), oracle leaf {int(ds.params.leaf_size)}"
            if args.workload == "c2":
                accuracy["plummer"] = plummer_checks(w, g_main, ostate, dist_seed=12)
        # the forms against each other
        A = lambda x: np.stack([x["ax"], x["ay"], x["az"]], 1)
        for name, g in results.items():
            if name != main_form:
                accuracy[f"{name}_vs_{main_form}"] = _rel(A(g), A(g_main))
        # the dissipation variants (Sect. 3.3.3) on the gas of a single system
        if w.params.sph and w.n_gas > 0 and offsets is None and rank == 0 and world == 1:
            diss_block = dissipation_form(torch, dev, stream, E, DeviceSet, w, max(2, min(args.steps, 5)),
                                          int(ds.params.leaf_size), ostate)
    if not args.no_extras and rank == 0 and world == 1 and offsets is None and args.kdk_steps == 0:
        # periodic gravity (Sect. 4.3) and individual time steps (Sect. 4.2.1) at 2^20 particles
        extras = {"ewald": ewald_block(torch, dev, stream, E, DeviceSet, 1 << 20, 3),
                  "individual_steps": bins_block(torch, dev, stream, E, DeviceSet, 1 << 20)}

    # ---- roofline of the dominant kernel (the force walk) ----
    far, pp, sph, soft = float(cnt[0]), float(cnt[1]), float(cnt[2]), float(cnt[8])
    flops = far * FLOPS_FAR + (pp - soft) * FLOPS_PP_NEWTON + soft * FLOPS_PP_SOFT + sph * FLOPS_SPH
    walk_s = statistics.mean(walk_ms) / 1e3
    achieved = flops / walk_s / 1e12
    clk = clocks["sm_mhz"] if clocks else None
    roofline = {"bound": "alu", "kernel": "k_walk (gravity + SPH force walk)", "achieved": achieved,
                "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                "traffic": WALK_TRAFFIC.get((args.workload, int(ds.params.leaf_size))) if prec == E.EVOL_FP32_PLAIN else None,
                "peak_basis": f"measured in this run at {peak_clock} MHz: FMA-chain kernels (evol_fp32_peak), "
                              f"scalar {peak_scalar:.1f}, packed f32x2 {peak_packed:.1f} TFLOP/s; the larger",
                "walk_ms": walk_s * 1e3,
                "flops_per_step": flops,
                "interactions_per_step": {"far": far, "pp_newtonian": pp - soft, "pp_softened": soft, "sph": sph},
                "flops_per_interaction": {"far": FLOPS_FAR, "pp_newtonian": FLOPS_PP_NEWTON,
                                          "pp_softened": FLOPS_PP_SOFT, "sph": FLOPS_SPH},
                "lane_fill": {"far": far / max(cnt[9], 1), "pair_pass1": pp / max(cnt[10], 1),
                              "pair_pass2": (soft + sph) / max(cnt[11], 1)}}
    ph = np.mean(np.array(phase), axis=0).tolist()
    build_bytes = float(w.n * BUILD_BYTES_PER_PARTICLE + diag[11] * BUILD_BYTES_PER_NODE)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            v, cores, desc = oracle_sample(w, leaf=int(ds.params.leaf_size), state=ostate)
            cpu = {"value": v, "unit": "particles/s", "cores": cores, "kind": "oracle", "sample": desc}
        except Exception as ex:     # the baseline is reported, never required
            cpu = {"value": None, "unit": "particles/s", "cores": None, "kind": "oracle", "sample": f"failed: {ex}"}

    E.evol_destroy(ctx)
    if rank == 0:
        metric = ("KDK particle-steps/s (fixed step, one captured graph)" if args.kdk_steps > 0
                  else "force-step particles/s (tree gravity+SPH)")
        line = {"metric": metric, "value": value, "unit": "particle-steps/s" if args.kdk_steps > 0 else "particles/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "precision": args.precision, "data": "synthetic",
                "config": {"workload": wname, "n": w.n, "n_gas": w.n_gas, "theta": w.params.theta,
                           "n_nei": w.params.n_nei_sph, "leaf_size": int(ds.params.leaf_size),
                           "length_group": int(ds.params.length_group) or 8,
                           "kdk_steps_per_bench_step": args.kdk_steps or None,
                           "autotune": autotune,
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "working set > L2 (inputs 40 B/particle x 3.1M + tree), no flush"},
                "phase_ms": {"build": ph[0], "eps_solve": ph[1], "h_solve": ph[2], "walk": ph[3], "total": ph[4]},
                "build_roofline": {"bound": "hbm", "achieved": build_bytes / (ph[0] * 1e-3) / 1e9,
                                   "peak": HBM_PEAK_GBS, "unit": "GB/s",
                                   "frac": build_bytes / (ph[0] * 1e-3) / 1e9 / HBM_PEAK_GBS,
                                   "algorithmic_bytes": build_bytes},
                "interactions_per_s": {"far": far / walk_s, "pp": pp / walk_s, "sph": sph / walk_s},
                "length_iterations_per_particle": diag[15] / max(1, w.n + w.n_gas),
                "status_last_step": rc,
                "counters": cnt,
                "forms_particles_per_s": forms,
                "forms_accuracy": accuracy,
                "dissipation_variants": diss_block,
                "periodic_and_individual_steps": extras,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": None}
        lps = launches_per_step(w)
        line["gpu_launches"] = (lps + args.kdk_steps * (lps + 3)) * args.steps if args.kdk_steps else lps * args.steps
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def launches_per_step(w):
    """Kernels of ours per evol_step: bbox 2, keys 1, 8 radix passes x (hist + 3 scan + scatter),
    permute, lcp, count, 3 scan, fill, link, moments, eps solve, h solve, pack, node-lengths 2,
    walk, unpermute, diagnostics 2."""
    p = w.params
    k = 2 + 1 + 8 * 5 + 1 + 1 + 1 + 3 + 1 + 1 + 1
    k += 1 if (p.gravity and p.adaptive_softening) else 0
    k += 1 if (p.sph and w.n_gas) else 0
    k += 1 + 2 + 1 + 1 + 2
    return k


def replica_rate(dist, device, ms_local, units_per_rank, steps, world):
    """Whole-job rate of `world` independent replicas (one system does not shard on this path):
    the units all ranks processed over the slowest rank's time (max over ranks).  Returns the rate
    in units/s and that time in ms."""
    ms_max = ms_local
    if dist is not None:
        import torch
        t = torch.tensor([float(ms_local)], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return units_per_rank * world * steps / (ms_max / 1e3), ms_max


if __name__ == "__main__":
    sys.exit(main())
