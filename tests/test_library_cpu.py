"""Host-side checks of the C ABI: the library builds for sm_103a, loads
without a GPU, and exports every entry point that include/*.h declares."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(nbp_[A-Za-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1911_10814_gb300 import build, nbp
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"
    # the binding covers the whole ABI under the same names
    assert names == set(nbp.SIGNATURES), sorted(names ^ set(nbp.SIGNATURES))


def test_default_options_match_paper_settings():
    from paper_1911_10814_gb300 import nbp
    o = nbp.default_options()
    assert o.rtol == 1e-8 and o.atol == 1e-50
    assert o.m == o.m_A == o.m_S == o.nmax == o.nmax_A == o.nmax_S == 200
    assert (o.rtol_A, o.rtol_S, o.rtol_I) == (1e-3, 1e-2, 1e-2)


def test_no_cpu_fallback_without_gpu():
    import pytest
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import synth
    from paper_1911_10814_gb300 import Solver
    with pytest.raises(RuntimeError):
        Solver(synth.generate(synth.tiny()))


def test_ctypes_mirrors_match_the_header_layout(tmp_path):
    """Every structure the binding passes through the C ABI has the size and
    field offsets the header gives it (a C program built against
    include/nbp.h prints them)."""
    import subprocess
    from paper_1911_10814_gb300 import nbp
    mirrors = [nbp.nbp_system, nbp.nbp_options, nbp.nbp_info, nbp.nbp_profile_info, nbp.nbp_rcr, nbp.nbp_mesh,
               nbp.nbp_vms_params, nbp.nbp_newton_opts, nbp.nbp_newton_info]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nbp.h"', "int main(void) {"]
    for cls in mirrors:
        name = cls.__name__
        lines.append(f'    printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.rsplit(" ", 1) for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cls in mirrors:
        name = cls.__name__
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, f"{name}.{f}"
