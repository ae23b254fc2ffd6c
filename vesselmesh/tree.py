"""Kuhn-voxel meshes: a plain box (test meshes) and the bifurcating tree."""
import numpy as np
from .mesh import Mesh, FLUID, WALL, INLET, OUTLET, WALL_END, OUTER, orient_positive, tag_nodes

_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def kuhn_grid(nx, ny, nz, h, origin=(0.0, 0.0, 0.0)):
    """Nodes and Kuhn tets of an nx x ny x nz grid of cubes of side h (6 tets per cube)."""
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    X = np.stack([ii, jj, kk], axis=-1).reshape(-1, 3) * h + np.asarray(origin, dtype=np.float64)

    def nid(i, j, k):
        return (i * (ny + 1) + j) * (nz + 1) + k

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.reshape(-1), cj.reshape(-1), ck.reshape(-1)
    tets = []
    for p in _PERMS:
        c = np.zeros((3, ci.size), dtype=np.int64)
        vs = [nid(ci, cj, ck)]
        for ax in p:
            c[ax] += 1
            vs.append(nid(ci + c[0], cj + c[1], ck + c[2]))
        tets.append(np.stack(vs, axis=1))
    # cell-major order: the 6 tets of one cube are adjacent
    tets = np.stack(tets, axis=1).reshape(-1, 4)
    return X, tets


def box_mesh(n=3, h=1.0 / 3.0, domain=0, jitter=0.0, seed=0):
    """Unit-ish box of n^3 Kuhn cubes, every tet in one domain (0 fluid, 1 wall).

    Interior nodes may be jittered by +-jitter*h per coordinate. Test meshes only:
    no caps, so no INLET/OUTLET/WALL_END tags.
    """
    X, tets = kuhn_grid(n, n, n, h)
    if jitter:
        rng = np.random.default_rng(seed)
        idx = np.round(X / h).astype(np.int64)
        interior = np.all((idx > 0) & (idx < n), axis=1)
        X[interior] += jitter * h * rng.uniform(-1, 1, size=(interior.sum(), 3))
    tets = orient_positive(X, tets).astype(np.int32)
    dom = np.full(len(tets), domain, dtype=np.uint8)
    tag = tag_nodes(len(X), tets, dom)
    return Mesh(X, tets, dom, tag, np.zeros(len(X), dtype=np.int32),
                [{"center": np.zeros(3), "normal": np.array([0.0, 0.0, 1.0]), "radius": 1.0,
                  "peak": 0.0, "amp": 0.0, "freq": 0.0, "phase": 0.0}],
                {"kind": "box", "n": n, "h": h})


def tree_mesh(*a, **k):
    raise NotImplementedError


def tree_config(*a, **k):
    raise NotImplementedError
