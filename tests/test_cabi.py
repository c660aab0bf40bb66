"""The C-ABI library builds, loads and exports every function declared in include/*.h (no GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(", text,
                             flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof"):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("mgr_create", "mgr_setup", "mgr_apply", "fgmres_solve", "mgr_destroy", "mgr_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1801_08464_gb300 import _build
    path = _build.build()
    so = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(so, n)]
    assert not missing, missing


def test_no_cpu_fallback_without_library(monkeypatch, tmp_path):
    import paper_1801_08464_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg, "LIBPATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        pkg.lib()


def test_options_defaults_match_header():
    import paper_1801_08464_gb300 as pkg
    from paper_1801_08464_gb300 import _build
    _build.build()
    o = pkg.options()
    assert o.precision == 0 and o.global_relax == 1
    assert list(o.frelax_sweeps)[:3] == [1, 2, 2] and list(o.restrict_type)[:3] == [1, 0, 0]
    assert o.amg_max_coarse == 256 and abs(o.amg_theta - 0.25) < 1e-15
    assert ctypes.sizeof(pkg.Options) == 256  # layout of mgr_options_t (x86-64 and aarch64 alike)
