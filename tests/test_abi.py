"""CPU checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/vtsplat.h declares (no GPU calls)."""

import ctypes
import os
import re


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(vt_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2506_02741_gb300 import _lib as L
    from paper_2506_02741_gb300 import build
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"vt_render", "vt_render_backward", "vt_backproject"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(L.EXPORTS)
    assert L.lib().vt_version().decode().startswith("vtsplat")


def test_workspace_size_is_host_only():
    from paper_2506_02741_gb300 import _lib as L
    lib = L.lib()
    b1 = lib.vt_workspace_bytes(1000, 64, 48, 0)
    b2 = lib.vt_workspace_bytes(2000, 64, 48, 0)
    assert b2 > b1 > 0
    assert lib.vt_workspace_bytes(-1, 64, 48, 0) == 0


def test_oracle_and_library_share_nothing():
    """The oracle sources neither include the library headers nor name its
    symbols, and the CUDA sources never include the oracle."""
    orc = open(os.path.join(ROOT, "oracle", "vt_oracle.c")).read()
    assert "vtsplat.h" not in orc and "vt_render" not in orc
    csrc = os.path.join(ROOT, "paper_2506_02741_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read(), f
    for f in ("api.py", "_lib.py", "build.py", "__init__.py"):
        src = open(os.path.join(ROOT, "paper_2506_02741_gb300", f)).read()
        assert "import oracle" not in src and "from oracle" not in src, f
