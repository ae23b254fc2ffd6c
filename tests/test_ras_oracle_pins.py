"""Pins of the oracle's restricted additive Schwarz / block ILU(k) preconditioner
(Sec. 3, Eq. 14-16; Sec. 4.3 fill levels; Sec. 4.5 orderings) against facts of
linear algebra: exact factorisations where ILU drops nothing, the Schwarz sum
with exact subdomain solves, known ILU(1) fill of the 5-point grid, and the
partition and ordering invariants. None of them runs the CUDA solver.
"""
import numpy as np
import scipy.sparse as sp
import pytest

import vesselmesh as vm
from oracle import ras_oracle as RO
from oracle import fsi_oracle as O


def block_matrix_on_graph(adj, seed, diag_shift=20.0):
    """A random 7x7-block matrix whose block graph is adj (plus the diagonal),
    made diagonally dominant so that every factorisation exists."""
    rng = np.random.default_rng(seed)
    n = len(adj)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in list(adj[i]) + [i]:
            B = rng.normal(size=(7, 7))
            if j == i:
                B += diag_shift * np.eye(7) * (1 + len(adj[i]))
            for a in range(7):
                rows.extend([7 * i + a] * 7)
                cols.extend(7 * j + np.arange(7))
                vals.extend(B[a])
    return sp.csr_matrix((vals, (rows, cols)), shape=(7 * n, 7 * n))


def path_graph(n, perm):
    """Path v_0 - v_1 - ... with the node numbers permuted by perm."""
    adj = [set() for _ in range(n)]
    for k in range(n - 1):
        a, b = perm[k], perm[k + 1]
        adj[a].add(b)
        adj[b].add(a)
    return [np.array(sorted(s), dtype=np.int64) for s in adj]


def tree_graph(n, seed):
    rng = np.random.default_rng(seed)
    adj = [set() for _ in range(n)]
    for v in range(1, n):
        p = int(rng.integers(0, v))
        adj[v].add(p)
        adj[p].add(v)
    return [np.array(sorted(s), dtype=np.int64) for s in adj]


def grid_graph(n):
    adj = [set() for _ in range(n * n)]
    for y in range(n):
        for x in range(n):
            i = y * n + x
            if x + 1 < n:
                adj[i].add(i + 1); adj[i + 1].add(i)
            if y + 1 < n:
                adj[i].add(i + n); adj[i + n].add(i)
    return [np.array(sorted(s), dtype=np.int64) for s in adj]


def exact(J, r):
    import scipy.sparse.linalg as spla
    return spla.spsolve(J.tocsc(), r.reshape(-1)).reshape(-1, 7)


@pytest.mark.parametrize("graph", ["path", "tree"])
def test_bilu0_is_exact_lu_on_trees(graph):
    """On a tree graph, reverse Cuthill-McKee numbers every node after all of its
    children, so elimination creates no fill: block ILU(0) is the exact block LU and
    one-subdomain RAS is J^{-1}."""
    n = 40
    rng = np.random.default_rng(3)
    adj = path_graph(n, rng.permutation(n)) if graph == "path" else tree_graph(n, 4)
    J = block_matrix_on_graph(adj, 5)
    X = rng.normal(size=(n, 3))
    r = rng.normal(size=(n, 7))
    ras = RO.RAS(J, X, None, None, 1, 1, 0, 0, 1, adj=adj)
    z = ras.apply(r)
    ze = exact(J, r)
    assert np.abs(z - ze).max() < 1e-12 * np.abs(ze).max()


def test_bilu0_is_not_exact_on_a_grid():
    """The same ILU(0) on a graph with cycles drops fill: the apply is no longer
    J^{-1} (guards the exact-LU pins against a degenerate test)."""
    adj = grid_graph(6)
    J = block_matrix_on_graph(adj, 6, diag_shift=0.5)
    r = np.random.default_rng(7).normal(size=(36, 7))
    z = RO.RAS(J, np.random.default_rng(8).normal(size=(36, 3)), None, None, 1, 1, 0, 0, 1, adj=adj).apply(r)
    ze = exact(J, r)
    assert np.abs(z - ze).max() > 1e-6 * np.abs(ze).max()


@pytest.mark.parametrize("ordering", [0, 1])
def test_full_fill_ilu_is_exact_lu(ordering):
    """ILU(k) with k at least the matrix size keeps every fill entry: it is the exact
    LU, in any order."""
    m = vm.tube_mesh(2, 4, 1, 1, seed=1)
    n = m.n_nodes
    adj = RO.node_graph(n, m.tets)
    J = block_matrix_on_graph(adj, 9, diag_shift=2.0)
    r = np.random.default_rng(10).normal(size=(n, 7))
    z = RO.RAS(J, m.X, m.tets, None, 1, 1, 0, n, ordering).apply(r)
    ze = exact(J, r)
    assert np.abs(z - ze).max() < 1e-11 * np.abs(ze).max()


def test_ras_with_exact_subdomain_solves_is_the_schwarz_sum():
    """With every fill entry kept, the subdomain solves are exact and the apply is
    sum_i (R_i^0)^T (R_i^delta J (R_i^delta)^T)^{-1} R_i^delta r (Eq. 16), formed here
    from dense inverses of the extracted blocks; with overlap covering the whole
    mesh it is J^{-1} r."""
    m = vm.tube_mesh(3, 6, 1, 1, seed=2)
    n = m.n_nodes
    adj = RO.node_graph(n, m.tets)
    J = block_matrix_on_graph(adj, 11, diag_shift=2.0)
    r = np.random.default_rng(12).normal(size=(n, 7))
    owner = RO.partition_rcb(m.X, None, 1, 4)
    z_ref = np.zeros((n, 7))
    Jd = J.toarray()
    for s in range(4):
        own = np.nonzero(owner == s)[0]
        nodes = RO.overlap(own, adj, 1)
        dofs = (7 * nodes[:, None] + np.arange(7)).reshape(-1)
        zi = np.linalg.solve(Jd[np.ix_(dofs, dofs)], r[nodes].reshape(-1)).reshape(-1, 7)
        mine = np.isin(nodes, own)
        z_ref[nodes[mine]] = zi[mine]
    z = RO.RAS(J, m.X, m.tets, None, 1, 4, 1, n, 1).apply(r)
    assert np.abs(z - z_ref).max() < 1e-11 * np.abs(z_ref).max()
    z_all = RO.RAS(J, m.X, m.tets, None, 1, 4, n, n, 1).apply(r)
    ze = exact(J, r)
    assert np.abs(z_all - ze).max() < 1e-11 * np.abs(ze).max()


def test_ilu1_fill_of_the_five_point_grid():
    """ILU(1) of the 5-point matrix in natural order adds exactly the fill of level
    1: entries between (x, y) and (x - 1, y + 1), i.e. 2 (n - 1)^2 off-pattern
    entries, all at offset +-(n - 1); ILU(0) adds none and ILU(2) adds more."""
    n = 7
    adj = grid_graph(n)
    order = np.arange(n * n)
    lev0 = RO.ilu_levels(order, adj, 0)
    lev1 = RO.ilu_levels(order, adj, 1)
    lev2 = RO.ilu_levels(order, adj, 2)
    base = (lev0 == 0)
    assert base.sum() == n * n + 4 * n * (n - 1)
    fill1 = np.argwhere((lev1 <= 1) & ~base)
    assert len(fill1) == 2 * (n - 1) ** 2
    assert set(np.abs(fill1[:, 0] - fill1[:, 1])) == {n - 1}
    assert ((lev2 <= 2) & ~(lev1 <= 1)).sum() > 0


def test_partition_and_overlap_invariants():
    """Every node is owned by exactly one subdomain; bisection keeps the parts'
    sizes within one of each other when the count is a power of two; the overlap
    of delta layers holds every node within graph distance delta."""
    m = vm.tube_mesh(6, 8, 2, 1, seed=3)
    n = m.n_nodes
    adj = RO.node_graph(n, m.tets)
    owner = RO.partition_rcb(m.X, None, 1, 8)
    sizes = np.bincount(owner)
    assert owner.min() == 0 and len(sizes) == 8 and sizes.max() - sizes.min() <= 1
    own = np.nonzero(owner == 3)[0]
    ov = RO.overlap(own, adj, 2)
    # graph distance by BFS
    dist = np.full(n, -1)
    dist[own] = 0
    front = list(own)
    for d in (1, 2):
        nxt = []
        for v in front:
            for w in adj[v]:
                if dist[w] < 0:
                    dist[w] = d
                    nxt.append(w)
        front = nxt
    assert set(ov.tolist()) == set(np.nonzero(dist >= 0)[0].tolist())


def test_partition_of_a_line_is_contiguous():
    """Points on a line are cut into contiguous runs of equal size, ties broken by
    node number."""
    X = np.zeros((16, 3))
    X[:, 0] = np.array([3, 1, 4, 1, 5, 9, 2, 6, 5, 3, 5, 8, 9, 7, 9, 3], dtype=float)
    owner = RO.partition_rcb(X, None, 1, 4)
    order = np.lexsort((np.arange(16), X[:, 0]))
    assert list(owner[order]) == [0] * 4 + [1] * 4 + [2] * 4 + [3] * 4


def test_rcm_bandwidth_on_a_shuffled_path_and_grid():
    """Reverse Cuthill-McKee recovers bandwidth 1 on a path whatever the node
    numbering, and bandwidth n on an n x n grid."""
    rng = np.random.default_rng(13)
    n = 30
    adj = path_graph(n, rng.permutation(n))
    order = RO.rcm(np.arange(n), adj)
    pos = np.empty(n, dtype=int)
    pos[order] = np.arange(n)
    bw = max(abs(pos[a] - pos[b]) for a in range(n) for b in adj[a])
    assert sorted(order.tolist()) == list(range(n)) and bw == 1
    g = 6
    adj = grid_graph(g)
    perm = rng.permutation(g * g)
    inv = np.argsort(perm)
    adjp = [np.array(sorted(perm[w] for w in adj[inv[v]]), dtype=np.int64) for v in range(g * g)]
    order = RO.rcm(np.arange(g * g), adjp)
    pos = np.empty(g * g, dtype=int)
    pos[order] = np.arange(g * g)
    bw = max(abs(pos[a] - pos[b]) for a in range(g * g) for b in adjp[a])
    assert bw <= g


def test_full_fill_on_the_fsi_jacobian_is_exact():
    """On the FSI Jacobian of the parity tube (constraint rows, interface rows,
    7x7 blocks with entries from 1 to 1e7), one subdomain with every fill level kept
    solves J z = r to rounding: the extraction of J_i^delta and the block
    elimination handle the real block structure."""
    m = vm.tube_config("tube-12x8x4")
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets)
    y = vm.poiseuille_state(m)
    J = P.jacobian(y, y, y, 1e-3)
    r = np.random.default_rng(14).normal(size=(m.n_nodes, 7))
    z = RO.RAS(J, m.X, m.tets, None, 1, 1, 1, 20, 1).apply(r)
    res = r.reshape(-1) - J @ z.reshape(-1)
    assert np.linalg.norm(res) < 1e-8 * np.linalg.norm(r)


def test_nested_dissection_items_are_independent():
    """Nested dissection (Sec. 4.5): the items cover the subdomain once, and no
    edge and no fill entry of any level (even full fill) joins two items of the
    same phase, so their triangular solves can run side by side; D follows the
    leaf-size rule."""
    m = vm.tube_mesh(8, 12, 3, 1, seed=4)
    n = m.n_nodes
    adj = RO.node_graph(n, m.tets)
    nodes = np.arange(n)
    items, D = RO.nested_dissection(nodes, adj, m.X)
    assert D == 3 and len(items) == 2 ** (D + 1) - 1
    assert sorted(v for it in items for v in it) == list(range(n))
    order = RO.subdomain_order(nodes, adj, 3, X=m.X)
    pos = np.empty(n, dtype=int)
    pos[order] = np.arange(n)
    lev = RO.ilu_levels(order, adj, n)                  # every fill entry kept
    phases, k = [], 0
    for p in range(D + 1):
        cnt = 2 ** (D - p)
        phases.append(items[k:k + cnt])
        k += cnt
    for ph in phases:
        for a in range(len(ph)):
            for b in range(len(ph)):
                if a == b or not ph[a] or not ph[b]:
                    continue
                ia, ib = pos[np.array(ph[a])], pos[np.array(ph[b])]
                assert (lev[np.ix_(ia, ib)] <= n).sum() == 0
    # a small subdomain is not dissected
    assert RO.nested_dissection(nodes[:95], adj, m.X)[1] == 0
    assert RO.nested_dissection(nodes[:96], adj, m.X)[1] == 1


def test_nested_dissection_full_fill_is_exact():
    m = vm.tube_mesh(3, 8, 2, 1, seed=5)
    n = m.n_nodes
    adj = RO.node_graph(n, m.tets)
    J = block_matrix_on_graph(adj, 15, diag_shift=2.0)
    r = np.random.default_rng(16).normal(size=(n, 7))
    z = RO.RAS(J, m.X, m.tets, None, 1, 1, 0, n, 3).apply(r)
    ze = exact(J, r)
    assert np.abs(z - ze).max() < 1e-11 * np.abs(ze).max()
