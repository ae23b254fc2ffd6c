"""Mesh container, node tags and the interface-face search.

Node tags are bit flags. A node is FLUID if it belongs to a fluid tetrahedron and
WALL if it belongs to a wall tetrahedron; INTERFACE nodes are the vertices of the
wet interface, found by the face walk of Algorithm 1 (Sec. 4.8): every face of a
fluid tetrahedron whose neighbour across that face is a wall tetrahedron is an
interface triangle.
"""
from dataclasses import dataclass, field
import numpy as np

FLUID = 1
WALL = 2
INTERFACE = 4
INLET = 8       # fluid node on an inflow cap
OUTLET = 16     # fluid node on an outflow cap
WALL_END = 32   # wall node on a cap (clamped wall end)
OUTER = 64      # wall node on the outer wall surface

# local vertex triples of the four faces of a tetrahedron (face f omits vertex f)
TET_FACES = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]], dtype=np.int64)


@dataclass
class Mesh:
    """A conforming tetrahedral FSI mesh (fluid lumen + wall) with node tags.

    X           (N,3) float64   reference (t=0) node coordinates, cm
    tets        (T,4) int32     vertex ids, positively oriented
    tet_domain  (T,)  uint8     0 = fluid, 1 = wall
    node_tag    (N,)  uint32    bit flags FLUID|WALL|INTERFACE|INLET|OUTLET|WALL_END|OUTER
    node_problem(N,)  int32     problem id of each node (batched meshes), all 0 otherwise
    inlets      list of dicts, one per problem: center (3,), normal (3,) pointing into
                the lumen, radius, and the waveform (peak, amp, freq, phase)
    """
    X: np.ndarray
    tets: np.ndarray
    tet_domain: np.ndarray
    node_tag: np.ndarray
    node_problem: np.ndarray
    inlets: list
    info: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return int(self.X.shape[0])

    @property
    def n_tets(self):
        return int(self.tets.shape[0])

    @property
    def n_problems(self):
        return len(self.inlets)


def match_faces(tets):
    """Pair up the faces of a conforming tet mesh.

    Returns (faces, partner): faces (4T,3) int64 vertex triples oriented as in
    their tetrahedron (face f of tet t is row 4t+f and omits vertex f), and
    partner (4T,) the row of the same triangle in the neighbouring tet, or -1
    on the boundary. Faces are matched by their sorted vertex triple, sorted on
    two integer keys (first two vertices combined, then the third).
    """
    tets = np.asarray(tets, dtype=np.int64)
    faces = tets[:, TET_FACES].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    n = int(key.max()) + 1 if key.size else 1
    k01 = key[:, 0] * n + key[:, 1]
    order = np.lexsort((key[:, 2], k01))
    same = (k01[order[1:]] == k01[order[:-1]]) & (key[order[1:], 2] == key[order[:-1], 2])
    partner = -np.ones(len(faces), dtype=np.int64)
    i0 = order[:-1][same]
    i1 = order[1:][same]
    partner[i0] = i1
    partner[i1] = i0
    return faces, partner


def interface_faces(tets, tet_domain, matched=None):
    """Algorithm 1 (Sec. 4.8): faces of fluid tets shared with a wall tet.

    Returns an (F,3) int64 array of vertex ids, oriented as in the fluid
    tetrahedron, in increasing order of (fluid tet, face). matched: the output
    of match_faces(tets), if already at hand.
    """
    faces, partner = match_faces(tets) if matched is None else matched
    dom = np.asarray(tet_domain)
    own = np.arange(len(faces)) // 4
    sel = (partner >= 0) & (dom[own] == 0)
    sel[sel] = dom[partner[sel] // 4] == 1
    return faces[sel]


def tag_nodes(n_nodes, tets, tet_domain, matched=None):
    """FLUID / WALL / INTERFACE flags from the tet domains and Algorithm 1."""
    tag = np.zeros(n_nodes, dtype=np.uint32)
    tets = np.asarray(tets, dtype=np.int64)
    dom = np.asarray(tet_domain)
    for d, bit in ((0, FLUID), (1, WALL)):
        mark = np.zeros(n_nodes, dtype=bool)
        mark[tets[dom == d].ravel()] = True
        tag[mark] |= bit
    f = interface_faces(tets, tet_domain, matched)
    if f.size:
        mark = np.zeros(n_nodes, dtype=bool)
        mark[f.ravel()] = True
        tag[mark] |= INTERFACE
    return tag


def orient_positive(X, tets):
    """Swap two vertices of every negatively oriented tet."""
    e1 = X[tets[:, 1]] - X[tets[:, 0]]
    e2 = X[tets[:, 2]] - X[tets[:, 0]]
    e3 = X[tets[:, 3]] - X[tets[:, 0]]
    det = np.einsum("ij,ij->i", e1, np.cross(e2, e3))
    neg = det < 0
    t = tets.copy()
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def count_unknowns(mesh):
    """Unknowns as the paper counts them: 7 per fluid node (u, p, d), 3 per wall-only node."""
    fl = (mesh.node_tag & FLUID) != 0
    return int(7 * fl.sum() + 3 * (~fl).sum())


def concat_meshes(meshes):
    """Stack independent problems into one node/tet numbering (batched workload)."""
    Xs, Ts, Ds, Gs, Ps, inl = [], [], [], [], [], []
    off = 0
    for p, m in enumerate(meshes):
        Xs.append(m.X)
        Ts.append(m.tets + off)
        Ds.append(m.tet_domain)
        Gs.append(m.node_tag)
        Ps.append(np.full(m.n_nodes, p, dtype=np.int32))
        inl.extend(m.inlets)
        off += m.n_nodes
    return Mesh(np.concatenate(Xs), np.concatenate(Ts).astype(np.int32), np.concatenate(Ds),
                np.concatenate(Gs), np.concatenate(Ps), inl,
                {"problems": [m.info for m in meshes]})
