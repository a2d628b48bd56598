"""The allocation-free key + sort entry point (for callers that may not allocate device memory
where they call the library) returns exactly what the allocating tree build computes.

Collected last on purpose: if it fails, a run that stops at the first failure has already run
every other test.  It also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_0912_1786_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference(ctx, E, w):
    from paper_0912_1786_gb300.device import DeviceSet
    ds = DeviceSet(w)
    E.evol_build_tree(ctx, ds.particles, ds.params)
    E.evol_sync(ctx)
    keys = E.evol_get_debug(ctx, E.EVOL_DBG_KEYS, np.uint64)
    perm = E.evol_get_debug(ctx, E.EVOL_DBG_PERM, np.int32)
    cube = E.evol_get_debug(ctx, E.EVOL_DBG_CUBE, np.float64)
    return keys, perm, cube


def _noalloc(E, torch, w, stream):
    dev = torch.device("cuda:0")
    x, y, z = (torch.from_numpy(getattr(w, k)).to(dev) for k in ("x", "y", "z"))
    keys = torch.empty(w.n, dtype=torch.int64, device=dev)
    perm = torch.empty(w.n, dtype=torch.int32, device=dev)
    cube = torch.empty(4, dtype=torch.float64, device=dev)
    E.evol_sort_keys_noalloc(w.n, x, y, z, keys, perm, cube, stream)
    torch.cuda.synchronize()
    return keys.cpu().numpy().view(np.uint64), perm.cpu().numpy(), cube.cpu().numpy()


def test_noalloc_sort_matches_tree_build_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_0912_1786_gb300 import build, evol as E
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    # the set-up call a caller that may not allocate later makes at start-up: n = 0, no pointers
    E.evol_sort_keys_noalloc(0, None, None, None, None, None, None, stream)
    ctx = E.evol_create(E.EVOL_NOALLOC_MAX_N, stream)
    try:
        # two different particle sets back to back: the second call must not see the first's leftovers
        cases = [W.hernquist_gas(n_dm=40000, n_gas=5003, seed=31), W.evrard_sphere(E.EVOL_NOALLOC_MAX_N, seed=32)]
        for w in cases:
            rk, rp, rc = _reference(ctx, E, w)
            k, p, c = _noalloc(E, torch, w, stream)
            assert np.array_equal(c, rc)
            assert np.array_equal(k, rk)
            assert np.array_equal(p, rp)
    finally:
        E.evol_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_its_static_scratch():
    torch = pytest.importorskip("torch")
    from paper_0912_1786_gb300 import build, evol as E
    build.build()
    n = E.EVOL_NOALLOC_MAX_N + 1
    dev = torch.device("cuda:0")
    x = torch.zeros(n, device=dev)
    keys = torch.empty(n, dtype=torch.int64, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    with pytest.raises(E.EvolError) as ei:
        E.evol_sort_keys_noalloc(n, x, x, x, keys, perm)
    assert ei.value.code == E.EVOL_EINVAL
