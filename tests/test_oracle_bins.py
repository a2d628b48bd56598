"""Pins of the oracle's individual power-of-two time steps (Sect. 4.2.1).

* With one bin (max_bin = 0), or when no criterion asks for less than the largest step, the scheme
  is the global-step KDK of Sect. 4.1-4.2 with that fixed step.
* The timeline: every step is a power of two of ticks that divides its start, every particle is
  synchronised at the end of a largest step, a particle moves to a longer step only where the
  current time is a multiple of it, and the count of force evaluations is the sum over particles
  of their steps taken.
* Step selection: the largest power of two not longer than the criterion (brute force).
* Wake-up: a particle woken by a neighbour with a much shorter step ends its step at the first
  boundary of the shorter step and has received exactly half that shortened step of kick.
"""
import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W


def _ts(**kw):
    base = dict(eta_acc=0.1, eta_courant=0.2, eta_u=0.2, dt_max=0.05)
    base.update(kw)
    return oracle.TimeStep(**base)


def test_step_ticks_brute_force():
    rng = np.random.default_rng(71)
    T, tick = 64, 0.05 / 64
    dt = np.exp(rng.uniform(np.log(tick / 4), np.log(0.2), 2000))
    L = oracle.step_ticks(dt, T, tick)
    for d, l in zip(dt, L):
        cand = [2 ** k for k in range(7) if 2 ** k * tick <= d]
        assert l == (max(cand) if cand else 1)


def test_single_bin_is_the_fixed_step_kdk():
    w = W.evrard_sphere(500, seed=72, sigma_v=0.1)
    ts = _ts(dt_max=2e-3)
    b = oracle.run_bins(w, 3, ts, oracle.Bins(max_bin=0))
    g = oracle.run(w, 3, _ts(dt_min=2e-3, dt_max=2e-3))
    for k in ("x", "vx", "u"):
        assert np.allclose(b[k], g[k], rtol=1e-12, atol=1e-15), k
    assert b["stats"]["system_steps"] == 3 and b["stats"]["active_evaluations"] == 4 * w.n


def test_bins_unused_when_every_criterion_allows_the_largest_step():
    w = W.evrard_sphere(500, seed=73, sigma_v=0.1)
    ts = _ts(dt_max=2e-3)
    crit = oracle.timestep_criteria(w, oracle.force_step(w), w.vx, w.vy, w.vz, w.u, ts)
    assert min(float(np.min(c)) for c in crit.values()) > 2e-3 * 1.01
    b = oracle.run_bins(w, 2, ts, oracle.Bins(max_bin=4))
    g = oracle.run(w, 2, _ts(dt_min=2e-3, dt_max=2e-3))
    for k in ("x", "vx", "u"):
        assert np.allclose(b[k], g[k], rtol=1e-12, atol=1e-15), k


def test_timeline_invariants_and_evaluation_count():
    w = W.evrard_sphere(800, seed=74, sigma_v=0.2)
    ts = _ts(dt_max=0.08)
    K = 5
    T = 1 << K
    seen = []
    for stop in range(1, 40):
        b = oracle.run_bins(w, 1, ts, oracle.Bins(max_bin=K), stop_after=stop)
        tb, te = b["tb"], b["te"]
        L = te - tb
        assert np.all(L > 0) and np.all((L & (L - 1)) == 0)          # powers of two
        assert np.all(tb % L == 0)                                     # a step starts on its own boundary
        seen.append(len(np.unique(L)))
        if b["stats"]["system_steps"] < stop:
            break
    assert max(seen) >= 3                                              # several bins in use
    end = oracle.run_bins(w, 1, ts, oracle.Bins(max_bin=K))
    assert np.all(end["te"] == T)                                      # synchronised at the end
    # force evaluations: more than one step per particle (several bins), fewer than the finest bin's
    assert end["stats"]["active_evaluations"] > 2 * w.n and end["stats"]["active_evaluations"] < (T + 1) * w.n


def test_longer_step_only_on_its_own_boundary():
    # step_ticks decides the wish; the rule caps it by the largest power of two dividing t
    for t in (1, 2, 3, 4, 6, 8, 12, 16, 24):
        for want in (1, 2, 4, 8, 16, 32):
            got = min(want, t & -t)
            assert t % got == 0 and (got == want or t % (2 * got) != 0)


def test_wake_up_shortens_the_step_and_its_kick():
    # a hot particle at the centre of a cold sphere takes a much shorter Courant step than its
    # neighbours; with wake-up on they end their steps at its next boundary
    w = W.evrard_sphere(600, seed=75, sigma_v=0.05)
    r = np.sqrt(w.x.astype(np.float64) ** 2 + w.y ** 2 + w.z ** 2)
    hot = int(np.argmin(r))
    w.u[hot] = np.float32(w.u[hot] * 400.0)
    ts = _ts(dt_max=0.05)
    K = 6
    base = oracle.run_bins(w, 1, ts, oracle.Bins(max_bin=K, wake_factor=0.0), stop_after=1)
    woke = oracle.run_bins(w, 1, ts, oracle.Bins(max_bin=K, wake_factor=4.0), stop_after=1)
    assert woke["stats"]["wakeups"] > 0
    L0 = base["te"] - base["tb"]
    L1 = woke["te"] - woke["tb"]
    changed = np.flatnonzero(L1 != L0)
    assert len(changed) == woke["stats"]["wakeups"]
    assert np.all(L1[changed] < L0[changed])
    # every particle active in that first system step had the finest step L_hot; a woken one ends at
    # the first multiple of L' = 4 L_hot (the largest power of two <= 4 L_hot) after t = L_hot
    L_hot = int(L0.min())
    assert L0[hot] == L_hot
    assert np.all(woke["te"][changed] == 4 * L_hot)
    # the woken particles are still inactive after this first system step: their velocity change
    # since the start is the (cut) first half kick, a0 (te' - tb)/2 with a0 the starting acceleration
    r0 = oracle.force_step(w)
    a0 = np.stack([r0["ax"], r0["ay"], r0["az"]], 1)
    tick = ts.dt_max / (1 << K)
    v0 = np.stack([w.vx, w.vy, w.vz], 1).astype(np.float64)
    dv = np.stack([woke["vx"], woke["vy"], woke["vz"]], 1) - v0
    exp = a0 * (0.5 * L1 * tick)[:, None]
    assert np.allclose(dv[changed], exp[changed], rtol=1e-9, atol=1e-14)
