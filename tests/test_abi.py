"""The C ABI library builds for sm_103a, loads, and exports every entry point
that ``include/*.h`` declares; the ctypes mirrors match the C struct layouts.
(No compute calls: this runs without a GPU.)"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cp(?:2d)?_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_function():
    from paper_2603_24010_gb300 import native
    lib = native.lib()
    names = declared_functions()
    assert names, "no declarations found"
    assert set(native.EXPORTS) == names
    for n in sorted(names):
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", native.library_path()],
                         capture_output=True, text=True, check=True).stdout
    for n in names:
        assert re.search(r"\bT %s$" % n, out, flags=re.M), n


def test_library_targets_sm_103a():
    from paper_2603_24010_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_status_strings_without_gpu():
    from paper_2603_24010_gb300 import native
    assert native.cp_status_str(0) == "ok"
    assert "residual" in native.cp_status_str(native.ERR_RESIDUAL)


def test_struct_layouts_match_c(tmp_path):
    from paper_2603_24010_gb300 import native
    src = tmp_path / "sizes.c"
    fields = {
        "cp_gap": ["d", "weight", "sigma0", "n_cells"],
        "cp_circuit": ["R", "polarity", "kind"],
        "cp_see_beam": ["gamma_coef", "beam_Emax_eV", "beam_per_step", "beam_mode"],
        "cp_run": ["dt", "seed", "capacity", "max_steps", "precision", "compact_every"],
        "cp_diag": ["step", "V_gap", "max_cfl", "J_hat", "absorbed", "emitted", "injected",
                    "n_live", "conv_count"],
        "cp_predictor": ["in_scale", "out_scale", "bound"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cp.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", INCLUDE, "-o", str(exe), str(src)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for s, fs in fields.items():
        cls = getattr(native, s)
        assert int(got[s]) == C.sizeof(cls), s
        for f in fs:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)
