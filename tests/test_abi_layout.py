"""The ctypes structures of the binding mirror the C header: gcc compiles a
probe that prints sizeof and every field's offsetof from include/vtsplat.h,
and each must equal the ctypes layout (a field added to one side only, or
reordered, fails here before it can reach a kernel)."""

import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2506_02741_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "vt_intrinsics": L.Intrinsics,
    "vt_section": L.SectionC,
    "vt_grads": L.GradsC,
    "vt_view": L.ViewC,
    "vt_l1_weights": L.L1WeightsC,
    "vt_adam_params": L.AdamParamsC,
}


def _c_layout(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vtsplat.h"', 'int main(void) {']
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ['return 0;', '}']
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_ctypes_structs_match_header(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    got = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for f in cls._fields_:
            assert got[(name, f[0])] == getattr(cls, f[0]).offset, (name, f[0])
