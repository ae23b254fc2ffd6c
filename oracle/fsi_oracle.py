"""CPU FP64 oracle for one backward-Euler step of the monolithic FSI system.

TEST INFRASTRUCTURE ONLY. This module is the slow, plain reference that the CUDA
solver is checked against. Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import it; the solver library never calls it.

It follows Kong, Kheyfets, Finol & Cai, "Simulation of unsteady blood flows in a
patient-specific compliant pulmonary artery with a highly parallel monolithically
coupled fluid-structure interaction algorithm" (arXiv 1810.04289), Sec. 2-3:

* ALE map x = X + d_m (Sec. 2.1), harmonic mesh motion (Eq. 1);
* St. Venant-Kirchhoff wall in total Lagrangian form (Eq. 2 and the stress
  definitions after it);
* ALE incompressible Navier-Stokes with sigma_f = -p I + 2 mu eps(u) (Eq. 3);
* P1-P1 stabilised fluid, P1 wall and mesh motion, strong interface coupling with
  one set of unknowns per interface node (Sec. 2.2, Eq. 6-7);
* backward Euler in time with the mass matrix on the current geometry (Eq. 9),
  giving F(y) = 0 per step (Eq. 10);
* Newton with backtracking (Eq. 11-12).

Where the method's result has a plain definition (the solution y_n of F(y) = 0),
the oracle computes that definition directly: exact Newton with a sparse direct
linear solve (scipy SuperLU, a library primitive) to a tight tolerance, instead of
the preconditioned GMRES of Eq. 13-16. The Jacobian is obtained by the
complex-step method (Squire & Trapp, SIAM Rev. 1998): every residual routine
below is written with analytic operations only, so evaluating it at y + i h e_k
gives dF/dy_k = Im F / h exactly up to rounding. This is independent of the
hand-derived Jacobian of the CUDA path.

Readings of points the paper leaves open (stabilisation form and constants,
interface rows, boundary rows, line search) are listed in the module's design
notes and restated next to the code that uses them.

Parity unpinned: the values of the stabilisation parameters tau_M and tau_C. The
paper defers the stabilisation to its references and fixes no constant; the pins
check what the stabilised method must do with any admissible tau (patch tests,
Poiseuille convergence, discrete mass conservation, dissipativity of the
stabilisation terms, the complex-step Jacobian against finite differences), not
the constants themselves. The interface rows are pinned (a pressurised coupled
tube against the plane-strain Lame solution; wrong routings fail it).

Node block layout (7 dofs): [u_x, u_y, u_z, p, d_x, d_y, d_z].
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# node tags (same bit values as the mesh generator's; restated here so that the
# oracle imports nothing but numpy/scipy)
FLUID, WALL, INTERFACE, INLET, OUTLET, WALL_END, OUTER = 1, 2, 4, 8, 16, 32, 64

# 4-point degree-2 tetrahedral rule: barycentric (alpha, beta, beta, beta), weight 1/4
_QA = 0.5854101966249685
_QB = 0.1381966011250105
QP_N = np.array([[_QA, _QB, _QB, _QB], [_QB, _QA, _QB, _QB],
                 [_QB, _QB, _QA, _QB], [_QB, _QB, _QB, _QA]])
QP_W = np.full(4, 0.25)

DEFAULT_MATERIAL = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
def p1_gradients(x):
    """Gradients of the four P1 shape functions and the volume of each tet.

    x: (T,4,3) vertex coordinates (real or complex). The affine map is
    x = x0 + Jm xi with Jm = [x1-x0 | x2-x0 | x3-x0]; grad N_k (k=1..3) is row k of
    Jm^{-1}, grad N_0 = -(sum of the others). Jm^{-1} = adj(Jm)/det(Jm) by cofactors.
    Returns grad (T,4,3), vol (T,) = det/6.
    """
    e1 = x[:, 1] - x[:, 0]
    e2 = x[:, 2] - x[:, 0]
    e3 = x[:, 3] - x[:, 0]
    # rows of Jm^{-1}: (e2 x e3, e3 x e1, e1 x e2) / det, with det = e1 . (e2 x e3)
    c1 = np.cross(e2, e3)
    c2 = np.cross(e3, e1)
    c3 = np.cross(e1, e2)
    det = np.sum(e1 * c1, axis=1)
    g = np.empty(x.shape, dtype=x.dtype)
    g[:, 1] = c1 / det[:, None]
    g[:, 2] = c2 / det[:, None]
    g[:, 3] = c3 / det[:, None]
    g[:, 0] = -(g[:, 1] + g[:, 2] + g[:, 3])
    return g, det / 6.0


# ----------------------------------------------------------------------------
# element residuals
# ----------------------------------------------------------------------------
def fluid_element(Xe, ue, pe, de, u1e, d1e, mat, dt, stab=(1.0, 1.0, 1.0)):
    """Fluid-tet residuals: momentum (T,4,3), continuity (T,4), mesh motion (T,4,3).

    Momentum with test v = N_a e_i on the current tet (fully implicit BE, Eq. 3, 9):
        int rho (u - u_old)/dt . v + rho ((u - w) . grad) u . v + sigma(u,p) : grad v
      + SUPG  int tau_M ((a . grad) v) . r_M
      + LSIC  int tau_C rho (div v)(div u)
    continuity with test q = N_a:
        int q div u + PSPG int (tau_M / rho) grad q . r_M
    where w = (d - d_old)/dt is the BE mesh velocity, a = u - w, and
    r_M = rho (u - u_old)/dt + rho (a . grad) u + grad p (the P1 viscous term is 0).
    Stabilisation reading: h = (6 sqrt2 |K_0|)^(1/3) on the reference tet,
    D = sqrt((2 rho/dt)^2 + (2 rho |a_c|/h)^2 + (4 mu/h^2)^2) with a_c = a at the
    centroid, tau_M = rho/D, tau_M/rho = 1/D, tau_C rho = h^2 D / 12. Constant per
    tet; the 4-point rule integrates every term exactly.
    Mesh motion (Eq. 1, reference tet): int grad_X d : grad_X v.
    stab scales the (SUPG, PSPG, LSIC) terms; the solver always uses (1,1,1).
    """
    rho, mu = mat["rho_f"], mat["mu_f"]
    s_supg, s_pspg, s_lsic = stab
    xe = Xe + de                                   # ALE map, Sec. 2.1
    w = (de - d1e) / dt                            # BE mesh velocity
    grad, vol = p1_gradients(xe)
    G = np.einsum("tai,taj->tij", ue, grad)        # G_ij = du_i/dx_j
    divu = G[:, 0, 0] + G[:, 1, 1] + G[:, 2, 2]
    gradp = np.einsum("ta,taj->tj", pe, grad)
    grad0, vol0 = p1_gradients(Xe.astype(np.float64))
    h = (6.0 * np.sqrt(2.0) * vol0) ** (1.0 / 3.0)
    ae = ue - w
    ac = ae.mean(axis=1)
    D = np.sqrt((2.0 * rho / dt) ** 2 + 4.0 * rho * rho * np.sum(ac * ac, axis=1) / (h * h)
                + (4.0 * mu / (h * h)) ** 2)
    tau_m = rho / D
    tau_p = 1.0 / D
    tau_c_rho = h * h * D / 12.0

    Rm = np.zeros(ue.shape, dtype=np.result_type(ue, de, pe))
    Rc = np.zeros(pe.shape, dtype=Rm.dtype)
    for q in range(4):
        N = QP_N[q]
        uq = np.einsum("a,tai->ti", N, ue)
        u1q = np.einsum("a,tai->ti", N, u1e)
        aq = np.einsum("a,tai->ti", N, ae)
        conv = np.einsum("tij,tj->ti", G, aq)                  # (a . grad) u
        inert = rho * (uq - u1q) / dt + rho * conv
        rM = inert + gradp
        adv = np.einsum("ti,tai->ta", aq, grad)                # a . grad N_a
        wv = QP_W[q] * vol
        Rm += wv[:, None, None] * (N[None, :, None] * inert[:, None, :]
                                   + s_supg * tau_m[:, None, None] * adv[:, :, None] * rM[:, None, :])
        Rc += wv[:, None] * (N[None, :] * divu[:, None]
                             + s_pspg * tau_p[:, None] * np.einsum("tai,ti->ta", grad, rM))
    pc = pe.mean(axis=1)
    sym = G + np.transpose(G, (0, 2, 1))
    Rm += vol[:, None, None] * (-pc[:, None, None] * grad
                                + mu * np.einsum("tij,taj->tai", sym, grad)
                                + s_lsic * (tau_c_rho * divu)[:, None, None] * grad)
    Rh = vol0[:, None, None] * np.einsum("taj,tbj,tbi->tai", grad0, grad0, de)
    return Rm, Rc, Rh


def lame_constants(E, nu):
    """mu_s = E/(2(1+nu)), lambda_s = E nu/((1+nu)(1-2nu)) (Sec. 2.1)."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def wall_stress_element(Xe, de, mat):
    """Total-Lagrangian SVK stress term int_K0 Pi(F) : grad_X v, (T,4,3).

    F = I + grad d, E = (F^T F - I)/2, S = lambda tr(E) I + 2 mu E, Pi = F S
    (Sec. 2.1). Pi is constant per P1 tet, so one point is exact.
    """
    mu_s, lam_s = lame_constants(mat["E_s"], mat["nu_s"])
    grad0, vol0 = p1_gradients(Xe.astype(np.float64))
    F = np.eye(3)[None] + np.einsum("tai,taj->tij", de, grad0)
    E = 0.5 * (np.einsum("tki,tkj->tij", F, F) - np.eye(3)[None])
    trE = E[:, 0, 0] + E[:, 1, 1] + E[:, 2, 2]
    S = lam_s * trE[:, None, None] * np.eye(3)[None] + 2.0 * mu_s * E
    Pi = np.einsum("tik,tkj->tij", F, S)
    return vol0[:, None, None] * np.einsum("tij,taj->tai", Pi, grad0)


def wall_element(Xe, de, d1e, d2e, mat, dt):
    """Wall-tet momentum residual (T,4,3), Eq. 2 with BE in time.

    int rho_s (v_s - v_s,old)/dt . v + eta_s v_s . v + Pi : grad_X v on K0, with
    v_s = (d - d_old)/dt, v_s,old = (d_old - d_older)/dt and the consistent P1
    mass rho_s |K0| (1 + delta_ab)/20. f_s = 0 and g_s = 0 (zero outer traction).
    """
    _, vol0 = p1_gradients(Xe.astype(np.float64))
    vs = (de - d1e) / dt
    vs1 = (d1e - d2e) / dt
    M = (np.ones((4, 4)) + np.eye(4)) / 20.0
    acc = np.einsum("ab,tbi->tai", M, mat["rho_s"] * (vs - vs1) / dt + mat["eta_s"] * vs)
    return vol0[:, None, None] * acc + wall_stress_element(Xe, de, mat)


# ----------------------------------------------------------------------------
# global residual
# ----------------------------------------------------------------------------
def inlet_profile(X, inlet, t):
    """Parabolic inflow u = U(t) (1 - r^2/R^2)_+ n, U(t) = peak (1 + amp sin(2 pi f t + phase))."""
    c = np.asarray(inlet["center"])
    n = np.asarray(inlet["normal"])
    rel = X - c
    ax = rel @ n
    r2 = np.sum(rel * rel, axis=1) - ax * ax
    U = inlet["peak"] * (1.0 + inlet["amp"] * np.sin(2.0 * np.pi * inlet["freq"] * t + inlet["phase"]))
    prof = np.maximum(0.0, 1.0 - r2 / inlet["radius"] ** 2)
    return (U * prof)[:, None] * n[None, :]


class Problem:
    """Mesh + material + step data for the oracle's residual and Jacobian.

    mesh arrays: X (N,3), tets (T,4), tet_domain (T,), node_tag (N,),
    node_problem (N,), inlets (list of dicts). rigid_wall=True clamps every wall
    node (d = 0), so the wall does not move (rigid-wall Stokes/NS limit).
    """

    def __init__(self, X, tets, tet_domain, node_tag, node_problem, inlets, mat=None,
                 dt=1e-3, rigid_wall=False, stab=(1.0, 1.0, 1.0)):
        self.X = np.asarray(X, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        self.dom = np.asarray(tet_domain)
        self.tag = np.asarray(node_tag, dtype=np.int64)
        self.prob = np.asarray(node_problem, dtype=np.int64)
        self.inlets = inlets
        self.mat = dict(DEFAULT_MATERIAL if mat is None else mat)
        self.dt = float(dt)
        self.rigid_wall = rigid_wall
        self.stab = stab
        self.N = self.X.shape[0]
        self.ftets = self.tets[self.dom == 0]
        self.wtets = self.tets[self.dom == 1]
        tag = self.tag
        fl = (tag & FLUID) != 0
        wl = (tag & WALL) != 0
        itf = (tag & INTERFACE) != 0
        # rows that are replaced by constraint rows (Dirichlet, kinematic, identity)
        self.u_kin = itf.copy()                                  # u - (d - d_old)/dt
        self.u_ident = wl & ~fl                                   # wall-only: u = 0
        self.p_ident = wl & ~fl                                   # wall-only: p = 0
        self.u_inlet = fl & ((tag & INLET) != 0)                  # u = inflow profile
        self.d_zero = ((tag & (INLET | OUTLET | WALL_END)) != 0)
        if rigid_wall:
            self.d_zero = self.d_zero | wl
        self.u_kin &= ~self.u_inlet
        self.itf = itf

    # element-to-row placement --------------------------------------------------
    @staticmethod
    def route_fluid(Rm, Rc, Rh, itf):
        """Node-row layout (T,4,7) of a fluid tet's residuals (Sec. 2.2, Eq. 6-7).

        Continuity -> p row. Momentum -> u rows at fluid-only nodes; at interface
        nodes (itf (T,4) bool) -> the d rows, where it is added to the wall
        momentum of the wall tets: with one test function shared by both sides,
        the boundary terms of the two weak forms cancel exactly when
        sigma_s n_s = -sigma_f n_f (the traction balance of Sec. 2.1), so the sum
        imposes it weakly. Mesh motion -> d rows at fluid-only nodes. The u rows of
        interface nodes hold the kinematic condition instead (constraint rows).
        """
        itf = itf[:, :, None]
        out = np.zeros(Rm.shape[:2] + (7,), dtype=np.result_type(Rm, Rc, Rh))
        out[:, :, 0:3] = np.where(itf, 0.0, Rm)
        out[:, :, 3] = Rc
        out[:, :, 4:7] = np.where(itf, Rm, Rh)
        return out

    def element_rows(self, y, y1, y2):
        """Per-tet contributions (T_f,4,7) and (T_w,4,7) in the node-row layout.

        Fluid tets: continuity -> p row; momentum -> u rows at fluid-only nodes and
        -> d rows at interface nodes (the shared test function carries the traction
        balance sigma_s n = -sigma_f n, Sec. 2.1); mesh motion -> d rows at
        fluid-only nodes. Wall tets: wall momentum -> d rows.
        """
        X = self.X
        ft, wt = self.ftets, self.wtets
        out_f = out_w = None
        if len(ft):
            Xe = X[ft]
            Rm, Rc, Rh = fluid_element(Xe, y[ft, 0:3], y[ft, 3], y[ft, 4:7], y1[ft, 0:3],
                                       y1[ft, 4:7], self.mat, self.dt, self.stab)
            out_f = self.route_fluid(Rm, Rc, Rh, self.itf[ft])
        if len(wt):
            Rw = wall_element(X[wt], y[wt, 4:7], y1[wt, 4:7], y2[wt, 4:7], self.mat, self.dt)
            out_w = np.zeros(wt.shape + (7,), dtype=Rw.dtype)
            out_w[:, :, 4:7] = Rw
        return out_f, out_w

    def constraint_mask(self):
        """(N,7) bool: rows replaced by constraint rows."""
        m = np.zeros((self.N, 7), dtype=bool)
        m[:, 0:3] = (self.u_kin | self.u_ident | self.u_inlet)[:, None]
        m[:, 3] = self.p_ident
        m[:, 4:7] = self.d_zero[:, None]
        return m

    def residual(self, y, y1, y2, t):
        """F(y) (N,7), Eq. 10, for the step that ends at time t."""
        out_f, out_w = self.element_rows(y, y1, y2)
        F = np.zeros((self.N, 7), dtype=np.result_type(y, out_f if out_f is not None else y))
        if out_f is not None:
            np.add.at(F, self.ftets, out_f)
        if out_w is not None:
            np.add.at(F, self.wtets, out_w)
        F[self.constraint_mask()] = 0.0
        self._constraint_rows(F, y, y1, t)
        return F

    def _constraint_rows(self, F, y, y1, t):
        dt = self.dt
        k = self.u_kin
        F[k, 0:3] = y[k, 0:3] - (y[k, 4:7] - y1[k, 4:7]) / dt     # u_f = d(d_s)/dt, Eq. 3
        k = self.u_ident
        F[k, 0:3] = y[k, 0:3]
        F[self.p_ident, 3] = y[self.p_ident, 3]
        F[self.d_zero, 4:7] = y[self.d_zero, 4:7]                  # d_m = 0 on caps (Eq. 1), d_s = 0 at ends (Eq. 2)
        k = np.nonzero(self.u_inlet)[0]
        if len(k):
            uin = np.zeros((len(k), 3))
            for p, inl in enumerate(self.inlets):
                sel = self.prob[k] == p
                if np.any(sel):
                    uin[sel] = inlet_profile(self.X[k[sel]], inl, t)
            F[k, 0:3] = y[k, 0:3] - uin                            # u_f = v_f^d on the inlet, Eq. 3

    def jacobian(self, y, y1, y2, t, h=1e-30):
        """dF/dy as a scipy CSR matrix of size 7N, by the complex step.

        For every local node b and dof k, the gathered element inputs of all tets
        are perturbed by i h in (b, k); Im(element rows)/h is then column
        (tets[:, b], k) of every element matrix. Constraint rows are written
        directly: identity, or [I, -I/dt] for the kinematic rows.
        """
        N = self.N
        rows, cols, vals = [], [], []
        cmask = self.constraint_mask()
        for tets, which in ((self.ftets, 0), (self.wtets, 1)):
            if not len(tets):
                continue
            keep = ~cmask[tets]                                   # (T,4,7)
            r = 7 * tets[:, :, None] + np.arange(7)[None, None, :]
            for b in range(4):
                for k in range(7):
                    col = self._element_column(tets, which, y, y1, y2, b, k, h)
                    c = np.broadcast_to((7 * tets[:, b] + k)[:, None, None], r.shape)
                    rows.append(r[keep])
                    cols.append(c[keep])
                    vals.append(col[keep])
        kin = np.nonzero(self.u_kin)[0]
        for c in range(3):
            rows += [7 * kin + c, 7 * kin + c]
            cols += [7 * kin + c, 7 * kin + 4 + c]
            vals += [np.ones(len(kin)), np.full(len(kin), -1.0 / self.dt)]
        ident = cmask.copy()
        ident[self.u_kin, 0:3] = False
        idx = np.nonzero(ident.reshape(-1))[0]
        rows.append(idx)
        cols.append(idx)
        vals.append(np.ones(len(idx)))
        r = np.concatenate(rows)
        c = np.concatenate(cols)
        v = np.concatenate(vals)
        return sp.csr_matrix((v, (r, c)), shape=(7 * N, 7 * N))

    def _element_column(self, tets, which, y, y1, y2, b, k, h):
        X = self.X
        ye = y[tets].astype(np.complex128)
        ye[:, b, k] += 1j * h
        if which == 0:
            Rm, Rc, Rh = fluid_element(X[tets], ye[:, :, 0:3], ye[:, :, 3], ye[:, :, 4:7],
                                       y1[tets, 0:3], y1[tets, 4:7], self.mat, self.dt, self.stab)
            out = self.route_fluid(Rm, Rc, Rh, self.itf[tets])
        else:
            Rw = wall_element(X[tets], ye[:, :, 4:7], y1[tets, 4:7], y2[tets, 4:7], self.mat, self.dt)
            out = np.zeros(tets.shape + (7,), dtype=np.complex128)
            out[:, :, 4:7] = Rw
        return out.imag / h


# ----------------------------------------------------------------------------
# Newton (Eq. 11-12) with backtracking and a direct solve
# ----------------------------------------------------------------------------
class LineSearchError(RuntimeError):
    pass


class NewtonDiverged(RuntimeError):
    pass


def newton_solve(prob, y1, y2, t, rtol=1e-10, atol=0.0, maxit=30, armijo=1e-4,
                 alpha_min=2.0 ** -10, stall_rtol=1e-8, verbose=False):
    """Solve F(y) = 0 for the step ending at t, from y^(0) = y_{n-1}.

    Each iteration solves J(y) dy = -F(y) exactly (SuperLU), then backtracks
    alpha = 1, 1/2, 1/4, ... until ||F(y + alpha dy)|| <= (1 - armijo alpha)||F(y)||
    (Dennis-Schnabel backtracking, Sec. 3). Stops when ||F|| <= rtol ||F(y^(0))||
    or ||F|| <= atol. When backtracking finds no decrease although ||F|| is
    already below stall_rtol ||F(y^(0))||, |F| has reached the rounding floor of
    its assembly and the iterate is returned as converged. Returns
    (y, history of ||F||).
    """
    y = y1.copy()
    F = prob.residual(y, y1, y2, t)
    nf0 = np.linalg.norm(F)
    nf = nf0
    hist = [nf]
    for it in range(maxit):
        if nf <= rtol * nf0 or nf <= atol:
            return y, hist
        J = prob.jacobian(y, y1, y2, t)
        dy = spla.spsolve(J.tocsc(), -F.reshape(-1)).reshape(y.shape)
        alpha = 1.0
        while True:
            yt = y + alpha * dy
            Ft = prob.residual(yt, y1, y2, t)
            nft = np.linalg.norm(Ft)
            if nft <= (1.0 - armijo * alpha) * nf:
                break
            alpha *= 0.5
            if alpha < alpha_min:
                if nf <= stall_rtol * nf0:
                    # no decrease is possible any more: |F| sits at its rounding floor
                    return y, hist
                raise LineSearchError(f"backtracking failed at Newton iteration {it}")
        stalled = nft > 0.5 * nf and nft <= stall_rtol * nf0
        y, F, nf = yt, Ft, nft
        hist.append(nf)
        if stalled:
            # the last step no longer reduced |F| markedly and |F| is at the level
            # of its assembly rounding: further iterations only move rounding noise
            return y, hist
        if verbose:
            print(f"  newton {it}: |F| = {nf:.3e} alpha = {alpha}")
    if nf <= rtol * nf0 or nf <= atol:
        return y, hist
    raise NewtonDiverged(f"no convergence in {maxit} iterations: {hist}")


def run_steps(prob, y0, n_steps, t0=0.0, **kw):
    """Advance n_steps backward-Euler steps from y_{-1} = y_{-2} = y0 (initial state)."""
    y1, y2 = y0.copy(), y0.copy()
    out = []
    t = t0
    for n in range(n_steps):
        t = t0 + (n + 1) * prob.dt
        y, hist = newton_solve(prob, y1, y2, t, **kw)
        out.append((y, hist))
        y2, y1 = y1, y
    return out


# ----------------------------------------------------------------------------
# wall shear stress (Sec. 4, results: the WSS and SAWSS formulas)
# ----------------------------------------------------------------------------
def wss_faces(tets, tet_domain, node_problem):
    """The inner wall surface: faces shared by a fluid tet and a wall tet.

    Faces are matched by their sorted vertex triple (a plain dictionary, one pass
    over all faces). Returns an (F, 2) int64 array of (fluid tet, local index of
    the vertex opposite the face), sorted by (problem of the tet's first vertex,
    tet, local index).
    """
    tets = np.asarray(tets)
    owners = {}
    for t in range(tets.shape[0]):
        for f in range(4):
            key = tuple(sorted(int(tets[t, a]) for a in range(4) if a != f))
            owners.setdefault(key, []).append((t, f))
    out = []
    for lst in owners.values():
        if len(lst) != 2:
            continue
        (t0, f0), (t1, f1) = lst
        if tet_domain[t0] == 0 and tet_domain[t1] == 1:
            out.append((t0, f0))
        elif tet_domain[t1] == 0 and tet_domain[t0] == 1:
            out.append((t1, f1))
    prob = np.asarray(node_problem)
    out.sort(key=lambda tf: (int(prob[tets[tf[0], 0]]), tf[0], tf[1]))
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def wall_shear_stress(X, tets, tet_domain, node_problem, y, mu, n_problems=1):
    """Per-face WSS vectors and the spatially averaged WSS of every problem.

    On each inner-wall face, with the fluid stress sigma = -p I + 2 mu eps(u)
    (Eq. 3) of the adjacent fluid tet on the current configuration x = X + d
    (P1: eps constant on the tet, p taken at the face centroid) and n the unit
    normal pointing out of the fluid:
        WSS = sigma n - (sigma n . n) n,
    and SAWSS = (1/A) sum over faces of |WSS| area, A = total face area (the
    surface integral of the WSS magnitude over the inner wall, normalised by its
    area). Returns (faces (F,2), wss (F,3), area (F,), sawss (n_problems,)).
    """
    faces = wss_faces(tets, tet_domain, node_problem)
    y = np.asarray(y, dtype=np.float64)
    F = faces.shape[0]
    wss = np.zeros((F, 3))
    area = np.zeros(F)
    num = np.zeros(n_problems)
    den = np.zeros(n_problems)
    for i, (t, f) in enumerate(faces):
        v = np.asarray(tets[t], dtype=np.int64)
        x = X[v] + y[v, 4:7]
        g, _ = p1_gradients(x[None])
        G = y[v, 0:3].T @ g[0]                      # (grad u)_ij = sum_a u_a,i dN_a/dx_j
        eps = 0.5 * (G + G.T)
        fv = [a for a in range(4) if a != f]
        xa, xb, xc = x[fv[0]], x[fv[1]], x[fv[2]]
        cr = np.cross(xb - xa, xc - xa)
        A = 0.5 * np.linalg.norm(cr)
        n = cr / np.linalg.norm(cr)
        if np.dot(n, (xa + xb + xc) / 3.0 - x[f]) < 0:
            n = -n                                  # out of the fluid tet
        p = np.mean(y[v[fv], 3])
        sn = -p * n + 2.0 * mu * (eps @ n)
        w = sn - np.dot(sn, n) * n
        wss[i] = w
        area[i] = A
        q = int(node_problem[v[0]])
        num[q] += np.linalg.norm(w) * A
        den[q] += A
    sawss = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return faces, wss, area, sawss
