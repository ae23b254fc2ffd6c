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
    # the fields after them line up with the C struct (a shifted layout would misread these)
    assert (o.ilu_level, o.threads_per_row, o.ordering, o.factor_mode, o.verbose, o.fault_test) == (1, 32, 1, 0, 0, 0)
    L = fsi.lib()
    # null arguments are rejected before any device work
    assert L.fsi_create(None, None, None, 1, None, None, None) == 1
    assert L.fsi_residual(None, None, None) == 1
    assert L.fsi_step(None, None) == 1
    assert L.fsi_destroy(None) == 0
    assert L.fsi_last_error(None) == b"no context"


def _mesh_struct(X, T, D, G):
    import numpy as np
    from paper_1810_04289_gb300 import fsi
    keep = [np.ascontiguousarray(a) for a in (X, T, D, G)]
    m = fsi.FsiMesh(X.shape[0], T.shape[0], keep[0].ctypes.data, keep[1].ctypes.data, keep[2].ctypes.data,
                    keep[3].ctypes.data, None)
    return m, keep


def _create(m, opts):
    import ctypes
    from paper_1810_04289_gb300 import fsi
    mat = fsi.FsiMaterial(1.05, 0.035, 1.2, 3e6, 0.45, 0.0)
    bc = fsi.FsiBc()
    bc.normal[:] = [0.0, 0.0, 1.0]
    bc.radius = 1.0
    ctx = ctypes.c_void_p()
    st = fsi.lib().fsi_create(ctypes.byref(m), ctypes.byref(mat), ctypes.byref(bc), 1, ctypes.byref(opts), None,
                              ctypes.byref(ctx))
    return st, ctx


def test_create_rejects_bad_meshes_and_options_on_the_host():
    # validation runs before any device call, so these need no GPU
    import numpy as np
    import vesselmesh as vm
    from paper_1810_04289_gb300 import fsi
    box = vm.box_mesh(1, 1.0, domain=0)
    X = box.X.astype(np.float64)
    T = box.tets.astype(np.int32)
    D = box.tet_domain.astype(np.uint8)
    G = box.node_tag.astype(np.uint32)
    bad = T.copy()
    bad[0, 0] = 99                                  # vertex out of range
    m, keep = _mesh_struct(X, bad, D, G)
    st, ctx = _create(m, fsi.fsi_default_options())
    assert st == 2 and not ctx.value
    flipped = T.copy()
    flipped[0, [2, 3]] = flipped[0, [3, 2]]        # negatively oriented tet
    m, keep = _mesh_struct(X, flipped, D, G)
    st, ctx = _create(m, fsi.fsi_default_options())
    assert st == 2 and not ctx.value
    m, keep = _mesh_struct(X, T, D, G)
    st, ctx = _create(m, fsi.fsi_default_options(precision=5))
    assert st == 1 and not ctx.value
    # empty inputs and out-of-range options are refused before any device work
    m, keep = _mesh_struct(X, T[:0], D[:0], G)
    assert _create(m, fsi.fsi_default_options())[0] == 1            # no tets
    m, keep = _mesh_struct(X[:0], T[:0], D[:0], G[:0])
    assert _create(m, fsi.fsi_default_options())[0] == 1            # no nodes
    bad_d = D.copy()
    bad_d[0] = 3
    m, keep = _mesh_struct(X, T, bad_d, G)
    assert _create(m, fsi.fsi_default_options())[0] == 2            # domain not 0/1
    m, keep = _mesh_struct(X, T, D, G)
    assert _create(m, fsi.fsi_default_options(gmres_restart=65))[0] == 1
    assert _create(m, fsi.fsi_default_options(ilu_level=4))[0] == 1


def test_autotune_default_grid():
    """Subdomain counts are powers of two giving 40..1000 nodes per subdomain; both
    ILU levels, the three orderings that reorder (RCM, lumen-first RCM, nested
    dissection), overlap 1 and 2 and both SpMV row mappings are searched."""
    from paper_1810_04289_gb300.autotune import default_grid, KNOBS
    g = default_grid(46657)
    assert g["n_subdomains"] == (64, 128, 256, 512, 1024)
    assert all(40 <= 46657 / k <= 1000 for k in g["n_subdomains"])
    assert g["ilu_level"] == (1, 2) and g["ordering"] == (1, 2, 3)
    assert g["overlap"] == (1, 2) and g["threads_per_row"] == (32, 16)
    assert set(KNOBS) == set(g)
    assert default_grid(30)["n_subdomains"] == (1,)


def test_autotune_coordinate_search_logic(monkeypatch):
    """The coordinate search visits every value of every knob with the others at
    their best so far, never times a candidate twice and returns the fastest
    converged one (the timing is replaced by a fake cost on the CPU)."""
    from paper_1810_04289_gb300 import autotune as A
    from paper_1810_04289_gb300 import fsi

    class FakeMesh:
        n_nodes = 46657

    calls = []

    def fake(mesh, material, y0, opt, t0, torch):
        key = (opt.n_subdomains, opt.ilu_level, opt.ordering, opt.overlap, opt.threads_per_row)
        calls.append(key)
        # converges except for ordering 3; cheapest at 512 subdomains, ILU(2), overlap 1, 16 per row
        if opt.ordering == 3:
            return dict(seconds=9.0, iterations=1000, converged=False)
        t = abs(opt.n_subdomains - 512) / 512 + (0 if opt.ilu_level == 2 else 0.3) + 0.2 * (opt.overlap - 1)
        t += 0.0 if opt.threads_per_row == 16 else 0.05
        return dict(seconds=1.0 + t, iterations=100, converged=True)

    monkeypatch.setattr(A, "_candidate", fake)
    import sys
    import types
    monkeypatch.setitem(sys.modules, "torch", types.ModuleType("torch"))
    best, table = A.autotune(FakeMesh(), {}, None, base=fsi.FsiOptions())
    assert (best.n_subdomains, best.ilu_level, best.ordering, best.overlap, best.threads_per_row) == (512, 2, 1, 1, 16)
    assert len(calls) == len(set(calls)) == len(table)
    g = A.default_grid(46657)
    assert len(calls) <= sum(len(v) for v in g.values()) * 2
