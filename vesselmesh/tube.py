"""Straight compliant tube: polar index grid split into Kuhn tetrahedra.

Index space (theta, r, z). Cell (j, k, i) has corners (j+dj, k+dk, i+di). Every
cell is cut into the 6 Kuhn tetrahedra along its index diagonal (one per order of
the three unit steps). The innermost ring (k = 0) touches the axis, where all
theta corners coincide; only the 3 Kuhn paths that take the r step before the
theta step stay non-degenerate there, so those cells get 3 tets. The Kuhn split is
translation invariant in index space, so the periodic theta seam is conforming.
Cells with k < n_radial_fluid are lumen (fluid), the rest are wall.
"""
import numpy as np
from .mesh import (Mesh, FLUID, WALL, INTERFACE, INLET, OUTLET, WALL_END, OUTER,
                   orient_positive, tag_nodes)

_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
_AXIS_PERMS = [p for p in _PERMS if p.index(1) < p.index(0)]   # r step before theta step

SEED_BASE = 1810042890


def tube_mesh(n_axial, n_theta, n_radial_fluid, n_radial_wall, radius=0.5, length=4.0,
              wall=0.1, jitter=0.05, seed=0, origin=(0.0, 0.0, 0.0),
              peak=30.0, amp=0.5, freq=1.0, phase=0.0):
    nz, nt, nrf, nrw = int(n_axial), int(n_theta), int(n_radial_fluid), int(n_radial_wall)
    nr = nrf + nrw
    per_plane = 1 + nt * nr

    def nid(k, j, i):
        if k == 0:
            return i * per_plane
        return i * per_plane + 1 + (k - 1) * nt + (j % nt)

    N = (nz + 1) * per_plane
    # reference coordinates
    rk = np.array([radius * k / nrf if k <= nrf else radius + wall * (k - nrf) / nrw
                   for k in range(nr + 1)])
    drk = np.array([radius / nrf if k <= nrf else wall / nrw for k in range(nr + 1)])
    th = 2.0 * np.pi * np.arange(nt) / nt
    zz = length * np.arange(nz + 1) / nz
    rng = np.random.default_rng(seed)
    X = np.zeros((N, 3))
    kk = np.zeros(N, dtype=np.int64)
    ii = np.zeros(N, dtype=np.int64)
    for i in range(nz + 1):
        b = i * per_plane
        X[b] = (0.0, 0.0, zz[i])
        kk[b], ii[b] = 0, i
        for k in range(1, nr + 1):
            s = b + 1 + (k - 1) * nt
            X[s:s + nt, 0] = rk[k] * np.cos(th)
            X[s:s + nt, 1] = rk[k] * np.sin(th)
            X[s:s + nt, 2] = zz[i]
            kk[s:s + nt], ii[s:s + nt] = k, i
    # jitter interior nodes (not on a cap, the interface or the outer surface)
    interior = (ii > 0) & (ii < nz) & (kk != nrf) & (kk != nr)
    u = rng.uniform(-1.0, 1.0, size=(N, 3))
    dz = length / nz
    dth = 2.0 * np.pi / nt
    for n in np.nonzero(interior)[0]:
        k = kk[n]
        if k == 0:
            X[n, 0] += jitter * drk[0] * u[n, 0]
            X[n, 1] += jitter * drk[0] * u[n, 1]
        else:
            r = rk[k] + jitter * drk[k] * u[n, 0]
            t = np.arctan2(X[n, 1], X[n, 0]) + jitter * dth * u[n, 1]
            X[n, 0], X[n, 1] = r * np.cos(t), r * np.sin(t)
        X[n, 2] += jitter * dz * u[n, 2]
    # Kuhn tets
    tets, dom = [], []
    for i in range(nz):
        for k in range(nr):
            perms = _AXIS_PERMS if k == 0 else _PERMS
            d = 0 if k < nrf else 1
            for j in range(nt):
                for p in perms:
                    c = [0, 0, 0]
                    vs = [nid(k, j, i)]
                    for ax in p:
                        c[ax] += 1
                        vs.append(nid(k + c[1], j + c[0], i + c[2]))
                    tets.append(vs)
                    dom.append(d)
    tets = np.array(tets, dtype=np.int64)
    X = X + np.asarray(origin, dtype=np.float64)
    tets = orient_positive(X, tets).astype(np.int32)
    dom = np.array(dom, dtype=np.uint8)
    tag = tag_nodes(N, tets, dom)
    fl = (tag & FLUID) != 0
    wl = (tag & WALL) != 0
    tag[fl & (ii == 0)] |= INLET
    tag[fl & (ii == nz)] |= OUTLET
    tag[wl & ((ii == 0) | (ii == nz))] |= WALL_END
    tag[kk == nr] |= OUTER
    inlet = {"center": np.asarray(origin, dtype=np.float64), "normal": np.array([0.0, 0.0, 1.0]),
             "radius": float(radius), "peak": float(peak), "amp": float(amp),
             "freq": float(freq), "phase": float(phase)}
    info = {"kind": "tube", "n_axial": nz, "n_theta": nt, "n_radial_fluid": nrf,
            "n_radial_wall": nrw, "radius": radius, "length": length, "wall": wall,
            "seed": seed, "jitter": jitter, "origin": list(map(float, origin))}
    return Mesh(X, tets, dom, tag, np.zeros(N, dtype=np.int32), [inlet], info)


TUBE_CONFIGS = {
    # straight tube of the FP64 parity case: 12 axial x 8 around x (3 fluid + 1 wall) radial
    "tube-12x8x4": dict(n_axial=12, n_theta=8, n_radial_fluid=3, n_radial_wall=1, seed=SEED_BASE + 0),
    # refined tube: 96 x 32 x (12 + 3)
    "tube-96x32x15": dict(n_axial=96, n_theta=32, n_radial_fluid=12, n_radial_wall=3, seed=SEED_BASE + 1),
    # further refined tube near 1.07M unknowns: 160 x 48 x (18 + 4)
    "tube-160x48x22": dict(n_axial=160, n_theta=48, n_radial_fluid=18, n_radial_wall=4, seed=SEED_BASE + 1),
}


def tube_config(name, **over):
    kw = dict(TUBE_CONFIGS[name])
    kw.update(over)
    return tube_mesh(**kw)


def batch_tubes(n_tubes=64, seed=SEED_BASE + 3, unk_lo=5e3, unk_hi=2e5, wall=0.1):
    """Independent tubes of random radius, length, size and inflow phase.

    radius ~ U(0.2, 1.0) cm, length ~ U(2, 8) cm, target unknowns log-uniform in
    [unk_lo, unk_hi], phase ~ U(0, 2 pi). The cells are chosen near-isotropic to hit
    the target size; the wall gets max(1, round(wall / h)) radial cells.
    """
    from .mesh import concat_meshes
    rng = np.random.default_rng(seed)
    meshes = []
    for p in range(n_tubes):
        R = rng.uniform(0.2, 1.0)
        L = rng.uniform(2.0, 8.0)
        target = np.exp(rng.uniform(np.log(unk_lo), np.log(unk_hi)))
        ph = rng.uniform(0.0, 2.0 * np.pi)
        # nodes ~ target / 6.5; nodes ~ nz * nt * nr with nt ~ 2 pi nrf, dz ~ R / nrf
        best = None
        for nrf in range(2, 60):
            h = R / nrf
            nt = max(8, int(round(2 * np.pi * R / h / 2)) * 2)
            nz = max(2, int(round(L / h)))
            nrw = max(1, int(round(wall / h)))
            nodes = (nz + 1) * (1 + nt * (nrf + nrw))
            err = abs(np.log(nodes * 6.5 / target))
            if best is None or err < best[0]:
                best = (err, nz, nt, nrf, nrw)
        _, nz, nt, nrf, nrw = best
        m = tube_mesh(nz, nt, nrf, nrw, radius=R, length=L, wall=wall,
                      seed=int(rng.integers(1 << 31)), origin=(0.0, 0.0, 0.0), phase=ph)
        meshes.append(m)
    return concat_meshes(meshes)
