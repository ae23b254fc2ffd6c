"""The solver's host-side Schwarz plan (csrc/setup.cpp: partition, overlap,
subdomain orderings of Sec. 4.5 including nested dissection, ILU(k) fill of
Sec. 4.3) against the oracle's plain statement of the same steps
(oracle/ras_oracle.py), on the CPU.

The setup code is compiled here with the host compiler (no GPU involved) and
driven through a small test harness (tests/native/plan_export.cpp). For every
subdomain the owned set, the local row order (global node of every row), the
nested-dissection items and the kept ILU(k) pattern must be identical.
"""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import vesselmesh as vm
from oracle import ras_oracle as RO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1810_04289_gb300", "csrc")
HARNESS = os.path.join(ROOT, "tests", "native", "plan_export.cpp")


@pytest.fixture(scope="module")
def planlib():
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tempfile.mkdtemp(prefix="fsi_plan_")
    so = os.path.join(d, "libplan.so")
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-fopenmp", "-shared", "-fPIC", "-I", CSRC, HARNESS,
                        os.path.join(CSRC, "setup.cpp"), "-o", so], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(so)
    L.plan_new.restype = ctypes.c_void_p
    L.plan_new.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                           ctypes.c_void_p]
    L.plan_free.argtypes = [ctypes.c_void_p]
    L.plan_array.restype = ctypes.c_void_p
    L.plan_array.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]
    yield L
    shutil.rmtree(d, ignore_errors=True)


def node_rank(m):
    tag = m.node_tag
    return np.where((tag & vm.INTERFACE) != 0, 1, np.where((tag & vm.FLUID) != 0, 0, 2)).astype(np.uint8)


def host_plan(L, m, nsub, overlap, fill, ordering):
    X = np.ascontiguousarray(m.X, dtype=np.float64)
    T = np.ascontiguousarray(m.tets, dtype=np.int32)
    NP = np.ascontiguousarray(m.node_problem, dtype=np.int32)
    rk = np.ascontiguousarray(node_rank(m))
    h = L.plan_new(m.n_nodes, X.ctypes.data, m.n_tets, T.ctypes.data, NP.ctypes.data, m.n_problems, nsub,
                   overlap, fill, ordering, rk.ctypes.data)
    out = {}
    types = {"gnode": np.int32, "col": np.int32, "sd_depth": np.int32, "owned": np.uint8}
    for name in ("sd_row", "gnode", "owned", "row_ptr", "col", "diag", "sd_depth", "sd_item", "item_row"):
        n = ctypes.c_int64()
        ptr = L.plan_array(h, name.encode(), ctypes.byref(n))
        dt = types.get(name, np.int64)
        out[name] = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                          shape=(n.value,)).copy() if n.value > 0 else np.zeros(0, dt)
    L.plan_free(h)
    return out


MESHES = {
    "tube": lambda: vm.tube_config("tube-12x8x4"),
    "tree": lambda: vm.tree_mesh(generations=3, r0=0.2, h=0.08, seed=7),
    "batch": lambda: vm.concat_meshes([vm.tube_mesh(4, 8, 2, 1, seed=1),
                                       vm.tube_mesh(6, 6, 2, 1, radius=0.4, length=3.0, seed=2)]),
}


@pytest.mark.parametrize("mesh", ["tube", "tree", "batch"])
@pytest.mark.parametrize("ordering", [0, 1, 2, 3])
def test_host_plan_matches_oracle(planlib, mesh, ordering):
    m = MESHES[mesh]()
    adj = RO.node_graph(m.n_nodes, m.tets)
    rank = node_rank(m)
    owner = RO.partition_rcb(m.X, m.node_problem, m.n_problems, 4 if mesh != "tree" else 8)
    cases = [(4 if mesh != "tree" else 8, 1, 1), (1, 1, 2), (16, 2, 0)] if mesh != "tree" else [(8, 1, 2), (64, 1, 1)]
    for nsub, overlap, fill in cases:
        H = host_plan(planlib, m, nsub, overlap, fill, ordering)
        owner = RO.partition_rcb(m.X, m.node_problem, m.n_problems, nsub)
        n_sd = len(H["sd_row"]) - 1
        assert n_sd == owner.max() + 1
        for s in range(n_sd):
            a, b = H["sd_row"][s], H["sd_row"][s + 1]
            own = np.nonzero(owner == s)[0]
            nodes = RO.overlap(own, adj, overlap)
            order = RO.subdomain_order(nodes, adj, ordering, rank, m.X)
            assert np.array_equal(H["gnode"][a:b], order), (nsub, s)
            assert np.array_equal(H["owned"][a:b].astype(bool), owner[order] == s)
            if ordering == 3:
                items, D = RO.nested_dissection(nodes, adj, m.X)
                assert H["sd_depth"][s] == D
                ends = np.cumsum([len(it) for it in items])
                assert np.array_equal(H["item_row"][H["sd_item"][s]:H["sd_item"][s + 1]], ends)
            keep = RO.ilu_levels(order, adj, fill) <= fill
            rows = [H["col"][H["row_ptr"][q]:H["row_ptr"][q + 1]] - a for q in range(a, b)]
            mine = np.zeros_like(keep)
            for i, cs in enumerate(rows):
                mine[i, cs] = True
            assert np.array_equal(mine, keep), (nsub, s, fill)
