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


def test_binding_struct_layouts_match_header(tmp_path):
    # every field of the ctypes mirrors sits at the offset the C compiler gives it in include/evol.h,
    # and the structs have the same size (a C program built against the header prints both)
    import shutil
    import subprocess
    from paper_0912_1786_gb300 import evol as E
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    structs = {"evol_particles": E.EvolParticles, "evol_params": E.EvolParams, "evol_outputs": E.EvolOutputs,
               "evol_integrator": E.EvolIntegrator, "evol_bins": E.EvolBins}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "evol.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln.strip())}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert got[(cname, f[0])] == getattr(py, f[0]).offset, (cname, f[0])
