"""Plain reference of the restricted additive Schwarz preconditioner with block
ILU(k) subdomain solves (Sec. 3, Eq. 14-16; ILU fill levels of Sec. 4.3; subdomain
orderings of Sec. 4.5).

TEST INFRASTRUCTURE ONLY. The tests compare the CUDA preconditioner apply with
this module; the solver library never calls it, and it imports nothing but numpy.

What it computes, step by step, for a Jacobian J (7x7 blocks, one block row per
mesh node) and a vector r:

1. Partition (one GPU has no processor grid; the partition is a property of the
   preconditioner): the subdomain count is shared out over the independent
   problems in proportion to their node counts (rounded half up, at least 1),
   then each problem's nodes are split by recursive coordinate bisection: the
   set is cut across the axis of its largest bounding-box extent (ties: the
   lower axis), the lower part taking floor(n * p_low / p) nodes in the order of
   (coordinate, node number), with p_low = floor(p / 2) of the p parts.
2. Overlap (Omega_i^delta, Sec. 3): delta layers of graph neighbours, the graph
   being "two nodes share a tetrahedron".
3. Order of each overlapped subdomain (Sec. 4.5): natural (node number), reverse
   Cuthill-McKee, reverse Cuthill-McKee stably sorted by a node rank (lumen,
   interface, wall), or nested dissection (see nested_dissection) with reverse
   Cuthill-McKee inside every part. Cuthill-McKee here: start at the unvisited node of least
   degree (ties: lowest node number), move the start to the last node reached by
   a breadth-first search that visits neighbours in increasing node number, then
   number breadth first, each node's unnumbered neighbours by increasing
   (degree, node number); the whole order is reversed at the end.
4. J_i^delta = R_i^delta J (R_i^delta)^T (Eq. 15, read with the transposes in
   the standard places): the blocks of J between nodes of the subdomain.
5. Block ILU(k): the level of fill of entry (q, j) is 0 on the graph of
   J_i^delta (and the diagonal) and min over k < q of lev(q,k) + lev(k,j) + 1
   along the elimination; entries of level <= k are kept. Elimination by rows:
   for each kept k < q in increasing order, L_qk = A_qk A_kk^{-1}, then
   A_qj -= L_qk A_kj for every kept j > k of row q.
6. Apply (Eq. 16): z = sum_i (R_i^0)^T U_i^{-1} L_i^{-1} R_i^delta r, with
   R_i^0 the restriction to the nodes the subdomain owns (restricted additive
   Schwarz): forward substitution with the unit lower factor, back substitution
   with the upper factor, and only the owned rows written.

Every step is written plainly (dense per-subdomain arrays, Python loops over
rows); it is meant for meshes of a few hundred to a few thousand nodes.
"""
import numpy as np

INF = np.iinfo(np.int64).max // 4


def node_graph(n_nodes, tets):
    """Neighbours of every node (nodes sharing a tetrahedron), self excluded:
    a list of sorted int64 arrays."""
    tets = np.asarray(tets, dtype=np.int64)
    nb = [set() for _ in range(n_nodes)]
    for t in tets:
        for a in t:
            nb[int(a)].update(int(b) for b in t if b != a)
    return [np.array(sorted(s), dtype=np.int64) for s in nb]


def partition_rcb(X, node_problem, n_problems, n_sub):
    """Owner subdomain of every node (step 1); returns an int array."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    node_problem = np.zeros(n, dtype=np.int64) if node_problem is None else np.asarray(node_problem)
    owner = -np.ones(n, dtype=np.int64)
    nxt = 0

    def split(idx, parts, first):
        if parts <= 1 or len(idx) <= 1:
            owner[idx] = first
            return
        ext = X[idx].max(axis=0) - X[idx].min(axis=0)
        ax = int(np.argmax(ext))
        order = np.lexsort((idx, X[idx, ax]))          # by coordinate, then node number
        srt = idx[order]
        pl = parts // 2
        cut = len(idx) * pl // parts
        split(srt[:cut], pl, first)
        split(srt[cut:], parts - pl, first + pl)

    for p in range(n_problems):
        idx = np.nonzero(node_problem == p)[0]
        if len(idx) == 0:
            continue
        k = int(np.floor(n_sub * len(idx) / n + 0.5))
        k = max(1, min(k, len(idx)))
        split(idx, k, nxt)
        nxt += k
    return owner


def overlap(own, adj, delta):
    """Owned nodes plus delta layers of neighbours (step 2), sorted."""
    S = set(int(v) for v in own)
    front = list(S)
    for _ in range(delta):
        new = set()
        for v in front:
            for w in adj[v]:
                if int(w) not in S:
                    new.add(int(w))
        S |= new
        front = list(new)
    return np.array(sorted(S), dtype=np.int64)


def rcm(nodes, adj):
    """Reverse Cuthill-McKee order of the node set (step 3)."""
    S = set(int(v) for v in nodes)
    nbs = {int(v): [int(w) for w in adj[v] if int(w) in S] for v in nodes}
    deg = {v: len(nbs[v]) for v in nbs}
    seen = set()
    order = []
    while len(order) < len(S):
        start = min((v for v in S if v not in seen), key=lambda v: (deg[v], v))
        bfs, reached = [start], {start}
        h = 0
        while h < len(bfs):
            for w in nbs[bfs[h]]:                       # increasing node number
                if w not in reached and w not in seen:
                    reached.add(w)
                    bfs.append(w)
            h += 1
        start = bfs[-1]
        seen.add(start)
        head = len(order)
        order.append(start)
        while head < len(order):
            v = order[head]
            head += 1
            new = [w for w in nbs[v] if w not in seen]
            for w in new:
                seen.add(w)
            order.extend(sorted(new, key=lambda w: (deg[w], w)))
    return np.array(order[::-1], dtype=np.int64)


ND_MIN_LEAF = 48


def nested_dissection(nodes, adj, X):
    """Nested-dissection items of an overlapped subdomain (Sec. 4.5's ND).

    Depth D: the largest D <= 3 with |nodes| >= 48 * 2^D. Each piece is cut at
    the median of its longest coordinate axis: ordered by (coordinate, node
    number), the lower floor(n/2) nodes form the lower half; the separator is the
    set of lower-half nodes with a graph neighbour in the upper half, the rest of
    the lower half and the upper half are the two children. Returns the items in
    phase-major order (the 2^D leaves left to right, then the separators from the
    deepest level up to the root's), each a list of node numbers, and D. No edge
    joins two items of the same phase.
    """
    X = np.asarray(X)
    m = len(nodes)
    D = 0
    while D < 3 and m >= ND_MIN_LEAF * 2 ** (D + 1):
        D += 1
    cur = [[int(v) for v in nodes]]
    seps = []
    for _ in range(D):
        nxt, lvl = [], []
        for S in cur:
            if S:
                ext = X[S].max(axis=0) - X[S].min(axis=0)
                ax = int(np.argmax(ext))
            else:
                ax = 0
            S = sorted(S, key=lambda v: (X[v, ax], v))
            half = len(S) // 2
            upper = set(S[half:])
            sep = [v for v in S[:half] if any(int(w) in upper for w in adj[v])]
            sset = set(sep)
            nxt += [[v for v in S[:half] if v not in sset], S[half:]]
            lvl.append(sep)
        cur = nxt
        seps.append(lvl)
    items = list(cur)
    for lvl in reversed(seps):
        items += lvl
    return items, D


def subdomain_order(nodes, adj, ordering, node_rank=None, X=None):
    """Local order of an overlapped subdomain: 0 natural, 1 RCM, 2 RCM stably
    sorted by node_rank, 3 nested dissection with RCM inside every item."""
    if ordering == 0:
        return np.array(sorted(int(v) for v in nodes), dtype=np.int64)
    if ordering == 3:
        items, _ = nested_dissection(nodes, adj, X)
        parts = [rcm(np.array(it, dtype=np.int64), adj) for it in items]
        return np.concatenate(parts) if parts else np.zeros(0, dtype=np.int64)
    order = rcm(nodes, adj)
    if ordering == 2:
        order = order[np.argsort(np.asarray(node_rank)[order], kind="stable")]
    return order


def ilu_levels(order, adj, fill):
    """Level-of-fill matrix (m x m, INF = dropped) of the subdomain in `order` (step 5)."""
    m = len(order)
    pos = {int(v): i for i, v in enumerate(order)}
    lev = np.full((m, m), INF, dtype=np.int64)
    for i, v in enumerate(order):
        lev[i, i] = 0
        for w in adj[v]:
            j = pos.get(int(w))
            if j is not None:
                lev[i, j] = 0
    for q in range(m):
        for k in range(q):
            if lev[q, k] > fill:
                continue
            cand = lev[q, k] + lev[k, k + 1:] + 1
            cand = np.where(lev[k, k + 1:] <= fill, cand, INF)
            cand = np.where(cand <= fill, cand, INF)
            lev[q, k + 1:] = np.minimum(lev[q, k + 1:], cand)
    return lev


def block_ilu(A, keep):
    """Block ILU on the kept pattern (step 5). A: (m, m, 7, 7) blocks of J_i^delta,
    keep: (m, m) bool. Returns (A, Dinv): the strictly lower blocks of A hold L
    (unit diagonal implied), the upper blocks U, Dinv the inverted pivots. The
    arithmetic is in A's dtype."""
    A = A.copy()
    m = A.shape[0]
    Dinv = np.zeros((m, 7, 7), dtype=A.dtype)
    for q in range(m):
        for k in range(q):
            if not keep[q, k]:
                continue
            A[q, k] = A[q, k] @ Dinv[k]
            js = np.nonzero(keep[q, k + 1:] & keep[k, k + 1:])[0] + k + 1
            if len(js):
                A[q, js] -= np.einsum("ab,jbc->jac", A[q, k], A[k, js])
        Dinv[q] = np.linalg.inv(A[q, q])
    return A, Dinv


class RAS:
    """The preconditioner of Eq. 16 for a block Jacobian on a mesh.

    J: scipy sparse (7N x 7N) Jacobian; X (N,3) reference coordinates; tets
    (T,4); node_problem (N,) or None; node_rank (N,) for ordering 2; adj: the
    node graph as a list of sorted neighbour arrays, in place of the one the
    tetrahedra give (tests on plain graphs). dtype: the arithmetic of the
    factorisation and the solves (FP64, or FP32 as in the mixed-precision form,
    where the subdomain factors and solves are FP32 and the vectors FP64 outside).
    """

    def __init__(self, J, X, tets, node_problem, n_problems, n_sub, delta, fill, ordering, node_rank=None,
                 adj=None, dtype=np.float64):
        import scipy.sparse as sp
        N = np.asarray(X).shape[0]
        self.N = N
        adj = node_graph(N, tets) if adj is None else adj
        owner = partition_rcb(X, node_problem, n_problems, n_sub)
        Jc = sp.csr_matrix(J)
        self.subs = []
        for s in range(int(owner.max()) + 1):
            own = np.nonzero(owner == s)[0]
            if len(own) == 0:
                continue
            nodes = overlap(own, adj, delta)
            order = subdomain_order(nodes, adj, ordering, node_rank, X)
            keep = ilu_levels(order, adj, fill) <= fill
            m = len(order)
            dofs = (7 * order[:, None] + np.arange(7)[None, :]).reshape(-1)
            Jd = Jc[dofs][:, dofs].toarray().reshape(m, 7, m, 7).transpose(0, 2, 1, 3)
            A = np.where(keep[:, :, None, None], Jd, 0.0).astype(dtype)
            LU, Dinv = block_ilu(A, keep)
            self.subs.append(dict(order=order, owned=(owner[order] == s), keep=keep, LU=LU, Dinv=Dinv))

    def apply(self, r):
        """z = B^{-1} r for r of shape (N, 7)."""
        r = np.asarray(r, dtype=np.float64).reshape(self.N, 7)
        z = np.zeros_like(r)
        for sd in self.subs:
            order, keep, LU, Dinv = sd["order"], sd["keep"], sd["LU"], sd["Dinv"]
            m = len(order)
            w = r[order].astype(LU.dtype)
            for q in range(m):
                for k in np.nonzero(keep[q, :q])[0]:
                    w[q] -= LU[q, k] @ w[k]
            for q in range(m - 1, -1, -1):
                t = w[q].copy()
                for j in np.nonzero(keep[q, q + 1:])[0] + q + 1:
                    t -= LU[q, j] @ w[j]
                w[q] = Dinv[q] @ t
            z[order[sd["owned"]]] = w[sd["owned"]]
        return z
