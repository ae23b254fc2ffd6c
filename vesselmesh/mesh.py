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


def interface_faces(tets, tet_domain):
    """Algorithm 1 (Sec. 4.8): faces of fluid tets shared with a wall tet.

    Faces are matched by their sorted vertex triple. Returns an (F,3) int64 array
    of vertex ids, oriented as in the fluid tetrahedron.
    """
    tets = np.asarray(tets, dtype=np.int64)
    T = tets.shape[0]
    faces = tets[:, TET_FACES]                      # (T,4,3)
    key = np.sort(faces, axis=2).reshape(-1, 3)
    owner = np.repeat(np.arange(T), 4)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0]))
    ks = key[order]
    same = np.all(ks[1:] == ks[:-1], axis=1)
    i0 = order[:-1][same]
    i1 = order[1:][same]
    d0 = tet_domain[owner[i0]]
    d1 = tet_domain[owner[i1]]
    out = []
    m = (d0 == 0) & (d1 == 1)
    out.append(faces.reshape(-1, 3)[i0[m]])
    m = (d0 == 1) & (d1 == 0)
    out.append(faces.reshape(-1, 3)[i1[m]])
    return np.concatenate(out, axis=0)


def tag_nodes(n_nodes, tets, tet_domain):
    """FLUID / WALL / INTERFACE flags from the tet domains and Algorithm 1."""
    tag = np.zeros(n_nodes, dtype=np.uint32)
    tets = np.asarray(tets, dtype=np.int64)
    tag[np.unique(tets[tet_domain == 0])] |= FLUID
    tag[np.unique(tets[tet_domain == 1])] |= WALL
    f = interface_faces(tets, tet_domain)
    if f.size:
        tag[np.unique(f)] |= INTERFACE
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
