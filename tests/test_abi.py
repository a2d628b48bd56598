"""The C-ABI library builds, loads and exports every entry point that include/evol.h declares.
No compute call is made here (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(evol_\w+)\s*\(", src))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_0912_1786_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"evol_build_tree", "evol_gravity", "evol_sph_density", "evol_sph_forces", "evol_step"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_is_host_only():
    from paper_0912_1786_gb300 import evol as E
    assert E.lib().evol_strerror(E.EVOL_ENOCONV).decode().startswith("smoothing")


def test_no_cpu_fallback_without_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_0912_1786_gb300 import evol as E
    with pytest.raises(E.EvolError) as ei:
        E.evol_create(16)
    assert ei.value.code == E.EVOL_ECUDA


def test_binding_struct_layouts_match_header():
    # sizes of the C structs as laid out by the compiler (x86-64 / aarch64 LP64 ABI)
    from paper_0912_1786_gb300 import evol as E
    assert ctypes.sizeof(E.EvolParticles) == 16 + 10 * 8
    assert ctypes.sizeof(E.EvolOutputs) == 12 * 8
    assert ctypes.sizeof(E.EvolParams) == 7 * 4 + 5 * 4 + 6 * 4 + 3 * 4
