"""Pins of the oracle's tree: root cube, Morton keys, sort permutation, node ranges and moments.

Each check uses an independent route: exact rational arithmetic for the keys, numpy's lexsort
for the permutation, a brute-force enumeration of all occupied cells for the node set, and the
multipole error law for the quadrupole.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_0912_1786_gb300 import workloads as W


def _cloud(n, seed, clustered=False):
    rng = np.random.default_rng(seed)
    if clustered:
        c = rng.normal(0, 1, (n, 3)) * rng.choice([1e-3, 1e-1, 1.0], size=(n, 1))
    else:
        c = rng.uniform(-1, 1, (n, 3))
    x, y, z = (np.ascontiguousarray(c[:, a], np.float32) for a in range(3))
    m = rng.uniform(0.5, 2.0, n).astype(np.float32)
    return x, y, z, m


def _deinterleave(k):
    q = [0, 0, 0]
    for b in range(21):
        for a in range(3):
            q[a] |= ((int(k) >> (3 * b + (2 - a))) & 1) << b
    return q


@pytest.mark.parametrize("n,seed,clustered", [(1, 0, False), (7, 1, False), (300, 2, False), (513, 3, True)])
def test_root_cube_and_keys_exact(n, seed, clustered):
    x, y, z, m = _cloud(n, seed, clustered)
    t = oracle.OracleTree(x, y, z, m, 0, 1)
    corner, side = t.cube()
    P = np.stack([x, y, z], 1).astype(np.float64)
    assert np.array_equal(corner, P.min(0))
    ext = (P.max(0) - P.min(0)).max()
    # side: a power of two, the smallest one >= ext (1 + 2^-20)
    mant, ex = np.frexp(side)
    assert mant == 0.5
    if ext > 0:
        assert side >= ext * (1 + 2.0 ** -20) and side / 2 < ext * (1 + 2.0 ** -20)
    keys = t.keys()
    for i in range(n):
        q = _deinterleave(keys[i])
        for a in range(3):
            exact = (Fraction(float(P[i, a])) - Fraction(float(corner[a]))) * (2 ** 21) / Fraction(side)
            qa = min(max(int(exact // 1), 0), 2 ** 21 - 1)
            assert q[a] == qa


@pytest.mark.parametrize("n,seed,clustered", [(300, 2, False), (2000, 4, True)])
def test_sort_is_stable_by_key(n, seed, clustered):
    x, y, z, m = _cloud(n, seed, clustered)
    # duplicate some particles so that equal keys occur
    x[: n // 10] = x[n // 2: n // 2 + n // 10]
    y[: n // 10] = y[n // 2: n // 2 + n // 10]
    z[: n // 10] = z[n // 2: n // 2 + n // 10]
    t = oracle.OracleTree(x, y, z, m, 0, 1)
    keys = t.keys()
    ref = np.lexsort((np.arange(n), keys))
    assert np.array_equal(t.perm(), ref.astype(np.int32))


def _brute_nodes(keys_sorted, leaf):
    """All occupied cells, keep those whose parent holds more than `leaf` particles."""
    n = len(keys_sorted)
    cells = {(0, 0): (0, n)}
    for lev in range(1, 22):
        pre = (keys_sorted >> np.uint64(3 * (21 - lev))).astype(np.uint64)
        starts = np.flatnonzero(np.concatenate([[True], pre[1:] != pre[:-1]]))
        ends = np.concatenate([starts[1:], [n]])
        for b, e in zip(starts, ends):
            cells[(lev, int(b))] = (int(b), int(e))
    out = set()
    for (lev, b), (bb, e) in cells.items():
        if lev == 0:
            out.add((0, bb, e))
            continue
        pb = None
        # parent: the level-(lev-1) cell containing position b
        for (pl, pbeg), (s, t) in ((k, v) for k, v in cells.items() if k[0] == lev - 1):
            if s <= b < t:
                pb = (s, t)
                break
        if pb[1] - pb[0] > leaf:
            out.add((lev, bb, e))
    return out


@pytest.mark.parametrize("n,seed,clustered,leaf", [(1, 0, False, 1), (64, 5, False, 1), (200, 6, True, 1),
                                                   (333, 7, False, 4), (257, 8, True, 8)])
def test_nodes_match_brute_force_cells(n, seed, clustered, leaf):
    x, y, z, m = _cloud(n, seed, clustered)
    t = oracle.OracleTree(x, y, z, m, 0, leaf)
    ks = t.keys()[t.perm()]
    nd = t.nodes()
    got = set(zip(nd["level"].tolist(), nd["begin"].tolist(), nd["end"].tolist()))
    assert got == _brute_nodes(ks, leaf)
    nn = t.nnodes
    # pre-order: sorted by (begin, level); subtree skip pointers; children counts
    order = np.lexsort((nd["level"], nd["begin"]))
    assert np.array_equal(order, np.arange(nn))
    for i in range(nn):
        sub = [j for j in range(i + 1, nn) if nd["begin"][j] < nd["end"][i] and nd["level"][j] > nd["level"][i]]
        assert nd["next"][i] == i + 1 + len(sub)
        cnt = nd["end"][i] - nd["begin"][i]
        internal = cnt > leaf and nd["level"][i] < 21
        kids = [j for j in sub if nd["level"][j] == nd["level"][i] + 1]
        assert nd["nchild"][i] == (len(kids) if internal else 0)
        if internal:
            assert sum(nd["end"][j] - nd["begin"][j] for j in kids) == cnt


def test_identical_particles_make_one_deep_leaf():
    n = 9
    x = np.full(n, 0.25, np.float32)
    t = oracle.OracleTree(x, x.copy(), x.copy(), np.ones(n, np.float32), 0, 1)
    nd = t.nodes()
    # extent 0 -> side 1; all keys equal -> a chain down to a level-21 leaf holding all 9
    assert t.cube()[1] == 1.0
    assert t.nnodes == 22 and nd["level"][-1] == 21 and nd["end"][-1] - nd["begin"][-1] == n


def test_moments_by_definition_and_geometry():
    x, y, z, m = _cloud(400, 9, True)
    t = oracle.OracleTree(x, y, z, m, 0, 4)
    nd, mo = t.nodes(), t.moments()
    perm = t.perm()
    P = np.stack([x, y, z], 1).astype(np.float64)
    corner, side = t.cube()
    for i in range(0, t.nnodes, 7):
        j = perm[nd["begin"][i]:nd["end"][i]]
        mm = m[j].astype(np.float64)
        assert np.isclose(mo["M"][i], mm.sum(), rtol=1e-14)
        com = (mm[:, None] * P[j]).sum(0) / mm.sum()
        assert np.allclose(mo["com"][i], com, rtol=1e-13, atol=1e-15)
        # quadrupole is traceless and symmetric by construction (xx + yy + zz = 0)
        assert abs(mo["Q"][i][:3].sum()) < 1e-12 * max(1e-30, np.abs(mo["Q"][i]).max())
        # particles lie in the node's cube and its bounding box
        l = mo["l"][i]
        assert np.isclose(l, side / 2 ** nd["level"][i])
        lo = mo["cgeo"][i] - l / 2
        assert np.all(P[j] >= lo - 1e-12) and np.all(P[j] < lo + l + 1e-12)
        assert np.allclose(mo["bmin"][i], P[j].min(0)) and np.allclose(mo["bmax"][i], P[j].max(0))
        assert np.isclose(mo["delta"][i], np.linalg.norm(mo["com"][i] - mo["cgeo"][i]))


def test_quadrupole_far_field_error_law():
    # A far node's monopole+quadrupole field differs from the exact sum at octupole order: the
    # error falls as d^-5 in the acceleration (d^-3 relative to the monopole term) and as d^-4 in
    # the potential.  A sign or
    # transposition mistake in the quadrupole leaves a d^-4 error instead.
    rng = np.random.default_rng(11)
    k = 64
    cl = rng.normal(0, 0.05, (k, 3)) + np.array([0.013, -0.021, 0.007])
    errs, perrs = [], []
    for dist in (1.0, 2.0, 4.0):
        probe = np.array([[dist, 0.37 * dist, -0.21 * dist]])
        P = np.concatenate([cl, probe]).astype(np.float32)
        m = np.concatenate([rng.uniform(0.5, 1.5, k), [1e-6]]).astype(np.float32)
        w = W.Workload("q", P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy(), *(np.zeros(k + 1, np.float32),) * 3,
                       m, np.zeros(k + 1, np.float32), np.full(k + 1, 1e-4, np.float32),
                       np.full(k + 1, 1e-4, np.float32), n_gas=0,
                       params=W.Params(theta=1.0, sph=0, adaptive_softening=0, leaf_size=4))
        far = oracle.force_step(w, idx=np.array([k]))
        ex = oracle.force_step(w, params=W.Params(theta=0.0, sph=0, adaptive_softening=0, leaf_size=4), idx=np.array([k]))
        assert far["nfar"][k] >= 1       # the cluster was taken as a far node
        a_far = np.array([far["ax"][k], far["ay"][k], far["az"][k]])
        a_ex = np.array([ex["ax"][k], ex["ay"][k], ex["az"][k]])
        errs.append(np.linalg.norm(a_far - a_ex))
        perrs.append(abs(far["pot"][k] - ex["pot"][k]))
    # d^-5 law: x32 per doubling (allow 20 .. 50); a d^-4 law would give x16
    for e1, e2 in zip(errs, errs[1:]):
        assert 20.0 < e1 / e2 < 50.0, errs
    # the potential's error is of octupole order too, d^-4: x16 per doubling (a wrong quadrupole
    # potential term -(1/2) d.Q.d / d^5 would leave a d^-3 error, x8)
    for e1, e2 in zip(perrs, perrs[1:]):
        assert 11.0 < e1 / e2 < 24.0, perrs
