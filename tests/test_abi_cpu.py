"""The C-ABI library builds, loads and exports every symbol include/fsi.h declares.

Runs without a GPU: no compute call is made.
"""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fsi_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_function():
    from paper_1810_04289_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    from paper_1810_04289_gb300 import fsi
    assert sorted(fsi.EXPORTS) == names


def test_default_options_and_argument_errors():
    from paper_1810_04289_gb300 import fsi
    o = fsi.fsi_default_options()
    assert o.dt == 1e-3 and o.newton_rtol == 1e-6 and o.gmres_rtol == 1e-3
    assert o.gmres_restart == 30 and o.n_subdomains == 64 and o.overlap == 1 and o.precision == 0
    L = fsi.lib()
    # null arguments are rejected before any device work
    assert L.fsi_create(None, None, None, 1, None, None, None) == 1
    assert L.fsi_residual(None, None, None) == 1
    assert L.fsi_step(None, None) == 1
    assert L.fsi_destroy(None) == 0
    assert L.fsi_last_error(None) == b"no context"
