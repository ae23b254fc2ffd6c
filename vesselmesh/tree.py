"""Kuhn-voxel meshes: a plain box (test meshes) and the bifurcating tree."""
import numpy as np
from .mesh import (Mesh, FLUID, WALL, INTERFACE, INLET, OUTLET, WALL_END, OUTER, orient_positive, tag_nodes,
                   match_faces)

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


def _rotate(v, axis, ang):
    """Rotate vector v about the unit axis by ang (Rodrigues)."""
    axis = axis / np.linalg.norm(axis)
    return (v * np.cos(ang) + np.cross(axis, v) * np.sin(ang) + axis * np.dot(axis, v) * (1 - np.cos(ang)))


def tree_branches(generations, r0, ratio, ratio_noise=0.0, angle=(35.0, 60.0), length_factor=8.0,
                  plane_jitter=20.0, seed=0):
    """Seeded bifurcating tree of straight branches.

    The root starts at the origin along +z with radius r0. Every branch ends in
    a Y-bifurcation into two daughters of radius r * ratio * (1 +- ratio_noise),
    each leaving the parent axis at an angle drawn from U(angle), on opposite
    sides, in a plane rotated 90 deg +- U(plane_jitter) about the parent axis
    from the parent's own branching plane. Branch length = length_factor * r.
    Returns a list of dicts: p0, p1, radius, parent, leaf.
    """
    rng = np.random.default_rng(seed)
    br = [dict(p0=np.zeros(3), p1=np.array([0.0, 0.0, length_factor * r0]), radius=r0, parent=-1,
               plane=np.array([1.0, 0.0, 0.0]), gen=0)]
    frontier = [0]
    for g in range(1, generations):
        nxt = []
        for b in frontier:
            P = br[b]
            axis = (P["p1"] - P["p0"]) / np.linalg.norm(P["p1"] - P["p0"])
            plane = _rotate(P["plane"], axis, np.deg2rad(90.0 + rng.uniform(-plane_jitter, plane_jitter)))
            plane -= axis * np.dot(plane, axis)
            plane /= np.linalg.norm(plane)
            for side in (-1.0, 1.0):
                th = np.deg2rad(rng.uniform(*angle))
                d = np.cos(th) * axis + side * np.sin(th) * plane
                r = P["radius"] * ratio * (1.0 + ratio_noise * rng.uniform(-1.0, 1.0))
                br.append(dict(p0=P["p1"].copy(), p1=P["p1"] + length_factor * r * d, radius=r, parent=b,
                               plane=plane, gen=g))
                nxt.append(len(br) - 1)
        frontier = nxt
    children = {i: [] for i in range(len(br))}
    for i, b in enumerate(br):
        if b["parent"] >= 0:
            children[b["parent"]].append(i)
    for i, b in enumerate(br):
        b["leaf"] = len(children[i]) == 0
    return br


def _branch_distance(pts, b, flat_start, flat_end):
    """Distance from pts to the branch axis segment; inf where a flat cap cuts it off."""
    d = b["p1"] - b["p0"]
    L = np.linalg.norm(d)
    d = d / L
    rel = pts - b["p0"]
    t = rel @ d
    tc = np.clip(t, 0.0, L)
    v = rel - tc[:, None] * d[None, :]
    dist = np.sqrt(np.add.reduce(v * v, axis=1))
    if flat_start:
        dist = np.where(t < 0.0, np.inf, dist)
    if flat_end:
        dist = np.where(t > L, np.inf, dist)
    return dist


def tree_mesh(generations=3, r0=1.2, ratio=0.79, ratio_noise=0.0, angle=(35.0, 60.0), length_factor=8.0,
              wall=0.1, h=0.04, seed=0, peak=30.0, amp=0.5, freq=1.0 / 0.8, phase=0.0):
    """Kuhn-voxel FSI mesh of a bifurcating tree (lumen + wall of fixed thickness).

    Background grid of cubes of side h (z-planes through the inlet), 6 Kuhn
    tets per cube; a tet is lumen if its centroid lies inside the union of the
    branch capsules (flat cut at the root inlet and at every leaf outlet), wall
    if it lies within `wall` outside that union, else dropped. The wet interface
    comes from the face walk of Algorithm 1 (Sec. 4.8). Caps: fluid boundary
    faces that are not interface faces lie on the inlet plane (INLET) or at a
    leaf outlet (OUTLET); wall nodes within h/2 of a cap plane are WALL_END.
    """
    br = tree_branches(generations, r0, ratio, ratio_noise, angle, length_factor, seed=seed)
    rmax_all = max(b["radius"] for b in br) + wall
    pts_all = np.array([b["p0"] for b in br] + [b["p1"] for b in br])
    lo = pts_all.min(axis=0) - rmax_all - 2 * h
    hi = pts_all.max(axis=0) + rmax_all + 2 * h
    lo[2] = 0.0                                   # the inlet plane z = 0 is a grid plane
    n = np.ceil((hi - lo) / h).astype(np.int64)
    # candidate cubes per branch (bounding box of the dilated capsule)
    cubes = []
    boxes = []
    for i, b in enumerate(br):
        R = b["radius"] + wall + h
        bl = np.minimum(b["p0"], b["p1"]) - R
        bh = np.maximum(b["p0"], b["p1"]) + R
        i0 = np.maximum(np.floor((bl - lo) / h).astype(np.int64), 0)
        i1 = np.minimum(np.ceil((bh - lo) / h).astype(np.int64), n)
        boxes.append((i0, i1))
        gx, gy, gz = np.meshgrid(np.arange(i0[0], i1[0]), np.arange(i0[1], i1[1]), np.arange(i0[2], i1[2]),
                                 indexing="ij")
        c = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
        ctr = lo + (c + 0.5) * h
        dist = _branch_distance(ctr, b, b["parent"] < 0, b["leaf"])
        keep = dist < b["radius"] + wall + 0.9 * h
        cubes.append(c[keep])
    cubes = np.concatenate(cubes)
    # distinct cubes in lexicographic (x, y, z) order, through one integer key
    ckey = np.unique(cubes[:, 2] + n[2] * (cubes[:, 1] + n[1] * cubes[:, 0]))
    cubes = np.stack([ckey // (n[1] * n[2]), (ckey // n[2]) % n[1], ckey % n[2]], axis=1)
    # Kuhn tets of the candidate cubes, vertex ids on the global grid
    def gid(ix, iy, iz):
        return (iz * (n[1] + 1) + iy) * (n[0] + 1) + ix
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    tv = []
    for p in perms:
        cc = np.zeros_like(cubes)
        vs = [gid(cubes[:, 0], cubes[:, 1], cubes[:, 2])]
        for ax in p:
            cc[:, ax] += 1
            vs.append(gid(cubes[:, 0] + cc[:, 0], cubes[:, 1] + cc[:, 1], cubes[:, 2] + cc[:, 2]))
        tv.append(np.stack(vs, axis=1))
    tv = np.concatenate(tv, axis=0)
    # classify tets by centroid: min over branches of (distance - radius)
    def coords(g):
        ix = g % (n[0] + 1)
        iy = (g // (n[0] + 1)) % (n[1] + 1)
        iz = g // ((n[0] + 1) * (n[1] + 1))
        return lo + np.stack([ix, iy, iz], axis=1) * h
    ctr = sum(coords(tv[:, a]) for a in range(4)) / 4.0
    # a centroid outside a branch's box of cubes is farther than radius + wall + h
    # from that branch, so each branch is measured only on the tets of its box
    # (tet p * nc + c lies in cube c; the cubes are sorted by x first)
    nc = len(cubes)
    gap = np.full(len(tv), np.inf)
    for b, (i0, i1) in zip(br, boxes):
        a0, a1 = np.searchsorted(cubes[:, 0], [i0[0], i1[0]])
        cs = np.arange(a0, a1)
        cs = cs[(cubes[cs, 1] >= i0[1]) & (cubes[cs, 1] < i1[1]) & (cubes[cs, 2] >= i0[2]) & (cubes[cs, 2] < i1[2])]
        sel = (np.arange(6)[:, None] * nc + cs[None, :]).ravel()
        gap[sel] = np.minimum(gap[sel], _branch_distance(ctr[sel], b, b["parent"] < 0, b["leaf"]) - b["radius"])
    fluid = gap < 0.0
    wallm = (~fluid) & (gap < wall)
    keep = fluid | wallm
    tv = tv[keep]
    dom = np.where(fluid[keep], 0, 1).astype(np.uint8)
    # compact node numbering in grid order (z-planes from the inlet)
    ids, inv = np.unique(tv.ravel(), return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int64)
    X = coords(ids)
    tets = orient_positive(X, tets).astype(np.int32)
    N = len(ids)
    matched = match_faces(tets)
    tag = tag_nodes(N, tets, dom, matched)
    # caps: fluid boundary faces that are not interface faces
    faces, partner = matched
    owner = np.arange(len(faces)) // 4
    bnd = partner < 0
    fl = (tag & FLUID) != 0
    wl = (tag & WALL) != 0
    fb = faces[bnd & (dom[owner] == 0)]
    cap_nodes = np.unique(fb)
    inlet = cap_nodes[np.abs(X[cap_nodes, 2]) < 1e-9]
    tag[inlet] |= INLET
    tag[np.setdiff1d(cap_nodes, inlet)] |= OUTLET
    # wall ends: wall nodes within h/2 of the inlet plane or of a leaf's end plane
    wend = wl & (np.abs(X[:, 2]) < 0.5 * h)
    for b in br:
        if b["leaf"]:
            d = (b["p1"] - b["p0"]) / np.linalg.norm(b["p1"] - b["p0"])
            t = (X - b["p1"]) @ d
            near = np.linalg.norm((X - b["p1"]) - t[:, None] * d[None, :], axis=1) < b["radius"] + wall + h
            wend |= wl & near & (np.abs(t) < 0.5 * h + 1e-12)
    tag[wend] |= WALL_END
    wb = faces[bnd & (dom[owner] == 1)]
    outer = np.zeros(N, dtype=bool)
    outer[np.unique(wb)] = True
    tag[outer & wl & ~((tag & INTERFACE) != 0)] |= OUTER
    inl = {"center": np.zeros(3), "normal": np.array([0.0, 0.0, 1.0]), "radius": float(r0), "peak": float(peak),
           "amp": float(amp), "freq": float(freq), "phase": float(phase)}
    info = {"kind": "tree", "generations": generations, "branches": len(br), "r0": r0, "ratio": ratio,
            "ratio_noise": ratio_noise, "h": h, "wall": wall, "seed": seed, "length": float(hi[2] - lo[2]),
            "leaves": int(sum(b["leaf"] for b in br))}
    return Mesh(X, tets, dom, tag, np.zeros(N, dtype=np.int32), [inl], info)


TREE_CONFIGS = {
    # 3 generations of Y-bifurcations (7 branches), daughter ratio 0.79, root radius 1.2 cm
    "tree-3gen": dict(generations=3, r0=1.2, ratio=0.79, h=0.04, seed=1810042890 + 2),
    # 7 generations (127 branches), Murray ratio 2^(-1/3) with +-10% noise, root radius 1.4 cm
    "tree-7gen": dict(generations=7, r0=1.4, ratio=2.0 ** (-1.0 / 3.0), ratio_noise=0.1, h=0.045,
                      seed=1810042890 + 4),
}


def tree_config(name, **over):
    kw = dict(TREE_CONFIGS[name])
    kw.update(over)
    return tree_mesh(**kw)
