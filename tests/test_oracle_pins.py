"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a closed form,
an invariance, an exact discrete identity, a patch test or a finite-difference
derivative. None of them runs the CUDA solver.
"""
import json
import os

import numpy as np
import pytest

import vesselmesh as vm
from oracle import fsi_oracle as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
MAT = dict(O.DEFAULT_MATERIAL)


def make_problem(m, **kw):
    return O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, **kw)


def interior_nodes(m):
    """Nodes of a box mesh that are not on its boundary surface."""
    lo, hi = m.X.min(axis=0), m.X.max(axis=0)
    eps = 1e-9
    return np.all((m.X > lo + eps) & (m.X < hi - eps), axis=1)


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
def test_p1_gradients_reproduce_linear_fields_and_volume():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(50, 4, 3))
    g, vol = O.p1_gradients(x)
    c = rng.normal(size=3)
    f = x @ c + 0.7                                    # linear field at the vertices
    assert np.allclose(np.einsum("ta,taj->tj", f, g), c[None, :], rtol=1e-10, atol=1e-10)
    # volume against the triple product written as a 4x4 determinant
    M = np.concatenate([x, np.ones((50, 4, 1))], axis=2)
    assert np.allclose(np.abs(vol), np.abs(np.linalg.det(M)) / 6.0, rtol=1e-12)


def test_tube_volume_is_the_polygon_prism():
    # boundary nodes are not jittered, so the meshed lumen is exactly the prism on
    # a regular n-gon inscribed in the circle: area n/2 R^2 sin(2 pi/n)
    m = vm.tube_config("tube-12x8x4")
    _, vol = O.p1_gradients(m.X[m.tets])
    n, R, L = 8, 0.5, 4.0
    fl = m.tet_domain == 0
    assert np.isclose(vol[fl].sum(), 0.5 * n * R * R * np.sin(2 * np.pi / n) * L, rtol=1e-12)
    Rb = 0.6
    assert np.isclose(vol[~fl].sum(), 0.5 * n * (Rb * Rb - R * R) * np.sin(2 * np.pi / n) * L, rtol=1e-12)
    assert vol.min() > 0


# ---------------------------------------------------------------------------
# Jacobian against central differences of the residual
# ---------------------------------------------------------------------------
def _fd_check(m, seed, rigid=False, h_rel=1e-4, tol=2e-5):
    P = make_problem(m, rigid_wall=rigid)
    rng = np.random.default_rng(seed)
    y0 = vm.poiseuille_state(m)
    sc = np.array([3, 3, 3, 10, 1e-3, 1e-3, 1e-3])
    y = y0 + rng.normal(size=y0.shape) * sc
    y1 = y0 + rng.normal(size=y0.shape) * sc
    y2 = y0 + rng.normal(size=y0.shape) * sc
    t = 2e-3
    J = P.jacobian(y, y1, y2, t).toarray()
    step = np.array([1, 1, 1, 10, 1e-3, 1e-3, 1e-3]) * h_rel
    n = J.shape[1]
    Jfd = np.zeros_like(J)
    for j in range(n):
        e = np.zeros(n)
        e[j] = step[j % 7]
        Fp = P.residual(y + e.reshape(-1, 7), y1, y2, t).reshape(-1)
        Fm = P.residual(y - e.reshape(-1, 7), y1, y2, t).reshape(-1)
        Jfd[:, j] = (Fp - Fm) / (2 * e[j])
    err = np.abs(J - Jfd).max(axis=0) / (np.abs(J).max(axis=0) + 1e-300)
    assert err.max() < tol, (err.max(), int(np.argmax(err)))


def test_jacobian_fd_single_fluid_tet():
    m = vm.box_mesh(1, 1.0, domain=0)
    m.tets = m.tets[:1]
    m.tet_domain = m.tet_domain[:1]
    _fd_check(m, 3)


def test_jacobian_fd_single_wall_tet():
    m = vm.box_mesh(1, 1.0, domain=1)
    m.tets = m.tets[:1]
    m.tet_domain = m.tet_domain[:1]
    _fd_check(m, 4)


def test_jacobian_fd_small_tube_with_interface_and_caps():
    _fd_check(vm.tube_mesh(2, 4, 1, 1, seed=5), 6)


def test_jacobian_fd_rigid_wall_tube():
    _fd_check(vm.tube_mesh(2, 4, 2, 1, seed=7), 8, rigid=True)


# ---------------------------------------------------------------------------
# wall: invariance, energy, patch, inertia
# ---------------------------------------------------------------------------
def _rotation(axis, ang):
    a = np.asarray(axis, dtype=float)
    a /= np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def test_wall_stress_vanishes_under_rigid_rotation():
    # SVK is frame invariant: d = (Q - I) X gives F = Q, E = 0, Pi = 0 on every tet
    rng = np.random.default_rng(2)
    X = rng.normal(size=(20, 4, 3))
    X = X[np.linalg.det(np.concatenate([X, np.ones((20, 4, 1))], 2)) > 0.1]
    Q = _rotation([0.3, -1.0, 0.5], 0.8)
    d = X @ Q.T - X
    R = O.wall_stress_element(X, d, MAT)
    scale = MAT["E_s"] * np.abs(O.p1_gradients(X)[1]).max() * 10
    assert np.abs(R).max() < 1e-9 * scale
    # whereas a stretch does load it
    d2 = X * np.array([0.01, 0.0, 0.0])
    assert np.abs(O.wall_stress_element(X, d2, MAT)).max() > 1e-4 * scale


def test_wall_stress_is_gradient_of_svk_energy():
    # the St. Venant-Kirchhoff strain energy |K0| (lambda/2 tr(E)^2 + mu E:E) has
    # nodal gradient int Pi : grad v with Pi = F S
    mu_s, lam_s = O.lame_constants(MAT["E_s"], MAT["nu_s"])
    rng = np.random.default_rng(9)
    X = np.array([[[0, 0, 0], [1, 0.1, 0], [0.2, 1, 0.1], [0.1, 0.3, 1.0]]], dtype=float)
    d = 0.05 * rng.normal(size=(1, 4, 3))

    def energy(dd):
        g, vol = O.p1_gradients(X)
        F = np.eye(3) + np.einsum("ai,aj->ij", dd[0], g[0])
        E = 0.5 * (F.T @ F - np.eye(3))
        return vol[0] * (0.5 * lam_s * np.trace(E) ** 2 + mu_s * np.sum(E * E))

    R = O.wall_stress_element(X, d, MAT)[0]
    h = 1e-7
    G = np.zeros((4, 3))
    for a in range(4):
        for i in range(3):
            e = np.zeros((1, 4, 3))
            e[0, a, i] = h
            G[a, i] = (energy(d + e) - energy(d - e)) / (2 * h)
    assert np.allclose(R, G, rtol=1e-6, atol=1e-6 * np.abs(R).max())


def test_lame_constants_match_golden():
    g = GOLDEN["lame_constants"]
    mu_s, lam_s = O.lame_constants(3.0e6, 0.45)
    assert np.isclose(mu_s, g["mu_s"], rtol=1e-14) and np.isclose(lam_s, g["lambda_s"], rtol=1e-14)


def test_wall_patch_affine_displacement():
    # affine d: F, Pi constant; interior nodes see sum_K |K| Pi grad N_a = 0
    m = vm.box_mesh(3, 1.0 / 3.0, domain=1, jitter=0.2, seed=3)
    A = np.array([[0.01, 0.002, -0.003], [0.004, -0.02, 0.001], [0.0, 0.005, 0.015]])
    d = m.X @ A.T + 0.1
    P = make_problem(m)
    Fe = O.wall_stress_element(m.X[P.wtets], d[P.wtets], MAT)
    R = np.zeros((m.n_nodes, 3))
    np.add.at(R, P.wtets, Fe)
    inner = interior_nodes(m)
    assert inner.sum() == 8
    assert np.abs(R[inner]).max() < 1e-9 * np.abs(R).max()


def test_wall_inertia_total_force_uniform_acceleration():
    # d = g t^2 / 2 on every node: F = I (no stress) and the BE second difference
    # is exactly g, so the summed wall rows equal rho_s g |wall volume|
    m = vm.box_mesh(2, 0.5, domain=1, jitter=0.1, seed=1)
    dt = 1e-3
    g = np.array([3.0, -1.0, 2.0])
    tn = 5 * dt
    y = np.zeros((m.n_nodes, 7))
    y1 = y.copy()
    y2 = y.copy()
    y[:, 4:7] = 0.5 * g * tn ** 2
    y1[:, 4:7] = 0.5 * g * (tn - dt) ** 2
    y2[:, 4:7] = 0.5 * g * (tn - 2 * dt) ** 2
    R = O.wall_element(m.X[m.tets], y[m.tets, 4:7], y1[m.tets, 4:7], y2[m.tets, 4:7], MAT, dt)
    V = O.p1_gradients(m.X[m.tets])[1].sum()
    # the stress part is not exactly zero (F = I only up to the d offset), so
    # compare the total, where the stress part cancels (sum_a grad N_a = 0)
    assert np.allclose(R.sum(axis=(0, 1)), MAT["rho_s"] * g * V, rtol=1e-8)


# ---------------------------------------------------------------------------
# fluid and mesh motion: patch tests, conservation, dissipation
# ---------------------------------------------------------------------------
def _fluid_rows(m, y, y1, mat, dt, stab=(1.0, 1.0, 1.0)):
    T = m.tets
    Rm, Rc, Rh = O.fluid_element(m.X[T], y[T, 0:3], y[T, 3], y[T, 4:7], y1[T, 0:3], y1[T, 4:7],
                                 mat, dt, stab)
    Fm = np.zeros((m.n_nodes, 3))
    Fc = np.zeros(m.n_nodes)
    Fh = np.zeros((m.n_nodes, 3))
    np.add.at(Fm, T, Rm)
    np.add.at(Fc, T, Rc)
    np.add.at(Fh, T, Rh)
    return Fm, Fc, Fh


def test_harmonic_patch_linear_mesh_displacement():
    m = vm.box_mesh(3, 1.0 / 3.0, domain=0, jitter=0.2, seed=4)
    y = np.zeros((m.n_nodes, 7))
    y[:, 4:7] = 1e-3 * (m.X @ np.array([[1, 2, 0], [0, -1, 3], [2, 0, 1.0]]).T)
    _, _, Fh = _fluid_rows(m, y, y, MAT, 1e-3)
    inner = interior_nodes(m)
    assert np.abs(Fh[inner]).max() < 1e-12 * np.abs(Fh).max()


def test_stokes_patch_linear_velocity_constant_pressure():
    # rho = 0 (Stokes limit), u = A x with tr A = 0, p constant, static mesh:
    # every interior momentum and continuity row vanishes
    m = vm.box_mesh(3, 1.0 / 3.0, domain=0, jitter=0.2, seed=5)
    mat = dict(MAT, rho_f=0.0)
    A = np.array([[0.5, 1.0, -2.0], [0.3, -1.5, 0.7], [2.0, 0.1, 1.0]])
    y = np.zeros((m.n_nodes, 7))
    y[:, 0:3] = m.X @ A.T
    y[:, 3] = 4.0
    Fm, Fc, _ = _fluid_rows(m, y, y, mat, 1e-3)
    inner = interior_nodes(m)
    assert np.abs(Fm[inner]).max() < 1e-12 * np.abs(Fm).max()
    assert np.abs(Fc[inner]).max() < 1e-12 * max(np.abs(Fc).max(), 1.0)


def test_unsteady_plug_flow_patch():
    # uniform u accelerating at rate g with p = -rho g . x solves the momentum
    # equation exactly (r_M = 0, viscous and convective terms vanish); interior
    # momentum rows vanish, which ties the mass term to the pressure term
    m = vm.box_mesh(3, 1.0 / 3.0, domain=0, jitter=0.2, seed=6)
    dt = 1e-3
    g = np.array([40.0, -10.0, 25.0])
    y1 = np.zeros((m.n_nodes, 7))
    y1[:, 0:3] = [1.0, 2.0, 3.0]
    y = y1.copy()
    y[:, 0:3] += g * dt
    y[:, 3] = -MAT["rho_f"] * (m.X @ g)
    Fm, Fc, _ = _fluid_rows(m, y, y1, MAT, dt)
    inner = interior_nodes(m)
    assert np.abs(Fm[inner]).max() < 1e-11 * np.abs(Fm).max()
    # continuity: div u = 0 and r_M = 0, so every row is zero up to rounding
    assert np.abs(Fc).max() < 1e-14
    # a wrong mass scaling would leave a residual: check the test can fail
    Fm2, _, _ = _fluid_rows(m, y, y1, MAT, 2 * dt)
    assert np.abs(Fm2[inner]).max() > 1e-3 * np.abs(Fm).max()


def test_ale_oseen_patch_moving_mesh():
    # u = A x (div-free) seen from a mesh moving with w = u - c: the ALE advection
    # velocity is the constant a = c, so (a . grad) u = A c, balanced by the linear
    # pressure p = -rho (A c) . x; with u_old = u at the nodes every term of the
    # interior momentum and continuity rows cancels. A wrong sign of w, u in place
    # of a, or a transposed velocity gradient leaves a residual.
    m = vm.box_mesh(3, 1.0 / 3.0, domain=0, jitter=0.2, seed=21)
    dt = 1e-3
    A = np.array([[0.5, 2.0, -1.0], [0.3, -1.5, 0.7], [1.2, 0.1, 1.0]])
    c = np.array([3.0, -2.0, 1.0])
    # d = dt (A x - c) with x = X + d  =>  d = (I - dt A)^{-1} dt (A X - c)
    M = np.linalg.inv(np.eye(3) - dt * A)
    d = (dt * (m.X @ A.T - c)) @ M.T
    x = m.X + d
    y = np.zeros((m.n_nodes, 7))
    y[:, 0:3] = x @ A.T
    y[:, 3] = -MAT["rho_f"] * (x @ (A @ c))
    y[:, 4:7] = d
    y1 = y.copy()
    y1[:, 4:7] = 0.0
    Fm, Fc, _ = _fluid_rows(m, y, y1, MAT, dt)
    inner = interior_nodes(m)
    assert np.abs(Fm[inner]).max() < 1e-10 * np.abs(Fm).max()
    assert np.abs(Fc).max() < 1e-13          # div u = 0 and r_M = 0 everywhere
    # the same state without the mesh motion is not a solution
    y1b = y1.copy()
    y1b[:, 4:7] = d
    Fm2, _, _ = _fluid_rows(m, y, y1b, MAT, dt)
    assert np.abs(Fm2[inner]).max() > 1e-3 * np.abs(Fm).max()


def test_momentum_rows_first_moment_is_fluid_stress():
    # for rho = 0, linear u and constant p the stress sigma = -p I + 2 mu eps(u) is
    # constant, and the weak form gives sum_a x_a,k R_a,i = int sigma_ik = |Omega| sigma_ik
    # (P1 reproduces the coordinate x_k); this fixes the symmetric strain rate
    m = vm.box_mesh(3, 1.0 / 3.0, domain=0, jitter=0.2, seed=22)
    mat = dict(MAT, rho_f=0.0)
    A = np.array([[0.5, 1.0, -2.0], [0.3, -1.5, 0.7], [2.0, 0.1, 1.0]])
    p0 = 4.0
    y = np.zeros((m.n_nodes, 7))
    y[:, 0:3] = m.X @ A.T
    y[:, 3] = p0
    Fm, _, _ = _fluid_rows(m, y, y, mat, 1e-3)
    mom = np.einsum("ak,ai->ik", m.X, Fm)
    vol = O.p1_gradients(m.X[m.tets])[1].sum()
    sigma = -p0 * np.eye(3) + mat["mu_f"] * (A + A.T)
    assert np.allclose(mom, vol * sigma, rtol=1e-12, atol=1e-12 * np.abs(sigma).max())


def test_continuity_rows_sum_to_boundary_flux():
    # sum over nodes of the continuity rows = int_K div u (PSPG sums to zero since
    # sum_a grad N_a = 0) = boundary flux of u on the current mesh x = X + d
    m = vm.tube_mesh(4, 8, 2, 1, seed=11)
    rng = np.random.default_rng(12)
    y = rng.normal(size=(m.n_nodes, 7))
    y[:, 4:7] *= 0.01
    y1 = rng.normal(size=(m.n_nodes, 7))
    fl = m.tet_domain == 0
    T = m.tets[fl]
    _, Rc, _ = O.fluid_element(m.X[T], y[T, 0:3], y[T, 3], y[T, 4:7], y1[T, 0:3], y1[T, 4:7], MAT, 1e-3)
    # boundary faces of the fluid region (faces used once), outward normals
    faces = T[:, O_faces()].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bnd = faces[cnt[inv.reshape(-1)] == 1]
    x = m.X + y[:, 4:7]
    a, b, c = x[bnd[:, 0]], x[bnd[:, 1]], x[bnd[:, 2]]
    nA = 0.5 * np.cross(b - a, c - a)                       # area-weighted normal
    ubar = (y[bnd[:, 0], 0:3] + y[bnd[:, 1], 0:3] + y[bnd[:, 2], 0:3]) / 3.0
    flux = np.sum(ubar * nA)
    assert np.isclose(Rc.sum(), flux, rtol=1e-11, atol=1e-12)


def O_faces():
    # outward-oriented faces of a positively oriented tet (v0 v1 v2 v3)
    return np.array([[1, 2, 3], [0, 3, 2], [0, 1, 3], [0, 2, 1]])


def _is_psd(S, rel=1e-10):
    w = np.linalg.eigvalsh(0.5 * (S + S.T))
    return w.min() >= -rel * max(np.abs(w).max(), 1e-300)


def test_stabilisation_terms_are_dissipative():
    # at a uniform flow (grad u = 0) on a static mesh, the SUPG u-u block
    # tau_M rho^2 (a.grad v)(a.grad du), the PSPG p-p block (1/D) grad q . grad dp
    # and the LSIC u-u block (h^2 D/12)(div v)(div du) are symmetric positive
    # semidefinite: each stabilisation adds dissipation, never removes it
    m = vm.box_mesh(2, 0.5, domain=0, jitter=0.2, seed=8)
    y = np.zeros((m.n_nodes, 7))
    y[:, 0:3] = [20.0, -5.0, 10.0]
    n = m.n_nodes
    dt = 1e9   # steady: the SUPG test term sees only the convective operator

    def J(stab):
        P = make_problem(m, dt=dt, stab=stab)
        P.u_kin[:] = False
        P.u_ident[:] = False
        P.p_ident[:] = False
        P.u_inlet[:] = False
        P.d_zero[:] = True
        return P.jacobian(y, y, y, 0.0).toarray()

    base = J((0.0, 0.0, 0.0))
    ui = np.array([7 * i + c for i in range(n) for c in range(3)])
    pi = np.array([7 * i + 3 for i in range(n)])
    for which, idx in ((0, ui), (1, pi), (2, ui)):
        s = [0.0, 0.0, 0.0]
        s[which] = 1.0
        dJ = J(tuple(s)) - base
        blk = dJ[np.ix_(idx, idx)]
        assert np.abs(blk).max() > 0
        assert _is_psd(blk), which
        # with the opposite sign the block is negative semidefinite instead
        assert not _is_psd(-blk), which


# ---------------------------------------------------------------------------
# closed-form flows and solids
# ---------------------------------------------------------------------------
def _poiseuille_error(n_axial, n_theta, n_rf):
    g = GOLDEN["poiseuille"]
    m = vm.tube_mesh(n_axial, n_theta, n_rf, 1, radius=g["R"], length=g["L"], jitter=0.0,
                     peak=g["U"], amp=0.0)
    mat = dict(MAT, mu_f=g["mu"])
    P = make_problem(m, mat=mat, dt=1e8, rigid_wall=True)
    y0 = vm.poiseuille_state(m, mu=g["mu"])
    y, hist = O.newton_solve(P, y0, y0, 1e8)
    fl = (m.node_tag & vm.FLUID) != 0
    r2 = m.X[:, 0] ** 2 + m.X[:, 1] ** 2
    uex = g["U"] * np.maximum(0, 1 - r2 / g["R"] ** 2)
    e = np.abs(y[fl, 2] - uex[fl]) / g["U"]
    # pressure drop from the axial pressure slope over the middle half of the tube
    z = m.X[:, 2]
    mid = fl & (z > 0.25 * g["L"]) & (z < 0.75 * g["L"])
    slope = np.polyfit(z[mid], y[mid, 3], 1)[0]
    return e.max(), np.sqrt(np.mean(e * e)), -slope * g["L"]


def test_poiseuille_convergence():
    # steady rigid-wall flow at Re_D = 900 with the exact parabolic inflow: the
    # nodal velocity error falls with h and the pressure drop approaches
    # 4 mu U L / R^2 = 67.2. With P1 elements the stabilised residual r_M lacks the
    # viscous term, a known first-order consistency error of P1-P1 residual
    # stabilisation (Jansen, Collis, Whiting & Shakib, CMAME 1999), so the pin is
    # first order or better, not second.
    g = GOLDEN["poiseuille"]
    m1, r1, dp1 = _poiseuille_error(6, 12, 3)
    m2, r2, dp2 = _poiseuille_error(12, 24, 6)
    assert m2 < m1 / 1.7 and r2 < r1 / 1.7, (m1, m2, r1, r2)
    assert r2 < 0.008 and m2 < 0.015
    assert abs(dp1 - g["dp"]) / g["dp"] < 0.03 and abs(dp2 - g["dp"]) / g["dp"] < 0.03, (dp1, dp2)


def _lame(n_theta, n_rw, n_axial=2):
    g = GOLDEN["lame"]
    mat = dict(MAT, E_s=g["E"], nu_s=g["nu"])
    a, b, Pp = g["a"], g["b"], g["P"]
    full = vm.tube_mesh(n_axial, n_theta, 1, n_rw, radius=a, length=0.2, wall=b - a, jitter=0.0)
    itf_faces = vm.interface_faces(full.tets, full.tet_domain)
    wt = full.tets[full.tet_domain == 1].astype(np.int64)
    used = np.unique(wt)
    remap = -np.ones(full.n_nodes, dtype=np.int64)
    remap[used] = np.arange(len(used))
    X = full.X[used]
    T = remap[wt]
    n = len(used)
    # pressure load on the inner surface: nodal share area/3 of P n, n radial outward
    f = np.zeros((n, 3))
    for fa in itf_faces:
        p = full.X[fa]
        nA = 0.5 * np.cross(p[1] - p[0], p[2] - p[0])
        c = p.mean(axis=0)
        if np.dot(nA[:2], c[:2]) < 0:
            nA = -nA
        for v in fa:
            f[remap[v]] += Pp * nA / 3.0
    z = X[:, 2]
    th = np.arctan2(X[:, 1], X[:, 0])
    fix = np.zeros((n, 3), dtype=bool)
    fix[:, 2] = (z < 1e-12) | (z > 0.2 - 1e-12)               # axial rollers
    fix[:, 0] |= np.isclose(np.abs(np.cos(th)), 0.0, atol=1e-9)  # symmetry planes
    fix[:, 1] |= np.isclose(np.abs(np.sin(th)), 0.0, atol=1e-9)
    free = ~fix.reshape(-1)
    d = np.zeros((n, 3))
    for it in range(6):
        R = np.zeros((n, 3))
        np.add.at(R, T, O.wall_stress_element(X[T], d[T], mat))
        R -= f
        r = R.reshape(-1)[free]
        if np.linalg.norm(r) < 1e-10 * np.linalg.norm(f):
            break
        # complex-step Jacobian of the stress term
        K = np.zeros((3 * n, 3 * n))
        for bb in range(4):
            for k in range(3):
                dc = d[T].astype(np.complex128)
                dc[:, bb, k] += 1e-30j
                col = O.wall_stress_element(X[T], dc, mat).imag / 1e-30
                for aa in range(4):
                    np.add.at(K, (3 * T[:, aa, None] + np.arange(3)[None, :], 3 * T[:, bb, None] + k),
                              col[:, aa, :])
        Kf = K[np.ix_(free, free)]
        dd = np.zeros(3 * n)
        dd[free] = np.linalg.solve(Kf, -r)
        d += dd.reshape(n, 3)
    rr = np.hypot(X[:, 0], X[:, 1])
    ur = (d[:, 0] * X[:, 0] + d[:, 1] * X[:, 1]) / rr
    inner = np.isclose(rr, a)
    outer = np.isclose(rr, b)
    return ur[inner].mean(), ur[outer].mean()


def test_lame_thick_cylinder_small_strain():
    g = GOLDEN["lame"]
    ua1, ub1 = _lame(16, 2)
    ua2, ub2 = _lame(32, 4)
    ea1, ea2 = abs(ua1 - g["u_r_a"]), abs(ua2 - g["u_r_a"])
    eb1, eb2 = abs(ub1 - g["u_r_b"]), abs(ub2 - g["u_r_b"])
    # second order (the polygonal section and P1 both err by O(h^2))
    assert ea2 < ea1 / 3.0 and eb2 < eb1 / 3.0, (ua1, ua2, ub1, ub2)
    assert ea2 / g["u_r_a"] < 0.02 and eb2 / g["u_r_b"] < 0.02


# ---------------------------------------------------------------------------
# the step as a whole
# ---------------------------------------------------------------------------
def test_newton_step_quadratic_and_volume_balance():
    # lumen volume change over a step equals the net inflow through the caps
    # (the kinematic rows make the wall move with the fluid): Q_in - Q_out = dV/dt
    m = vm.tube_config("tube-12x8x4")
    P = make_problem(m)
    y0 = vm.poiseuille_state(m)
    out = O.run_steps(P, y0, 2)
    hist = out[0][1]
    assert hist[2] < 1e-3 * hist[1] and len(hist) <= 5
    y1, y2 = out[0][0], out[1][0]
    fl = m.tet_domain == 0
    T = m.tets[fl]

    def volume(y):
        return O.p1_gradients((m.X + y[:, 4:7])[T])[1].sum()

    faces = T[:, O_faces()].reshape(-1, 3)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    bnd = faces[cnt[inv.reshape(-1)] == 1]

    def cap_flux(y, tagbit):
        sel = np.all((m.node_tag[bnd] & tagbit) != 0, axis=1)
        x = m.X + y[:, 4:7]
        f = bnd[sel]
        nA = 0.5 * np.cross(x[f[:, 1]] - x[f[:, 0]], x[f[:, 2]] - x[f[:, 0]])
        ub = y[f, 0:3].mean(axis=1)
        return np.sum(ub * nA)

    q_net = -(cap_flux(y2, vm.INLET) + cap_flux(y2, vm.OUTLET))    # net inflow
    dV = (volume(y2) - volume(y1)) / P.dt
    q_in = -cap_flux(y2, vm.INLET)
    assert abs(dV) > 1e-4 * q_in          # the wall does move
    assert abs(q_net - dV) < 1e-6 * q_in, (q_net, dV, q_in)


# ---------------------------------------------------------------------------
# wall shear stress (results section: WSS = sigma n - (sigma n . n) n, SAWSS)
# ---------------------------------------------------------------------------
def test_wss_poiseuille_converges_to_closed_form():
    """Rigid-tube Poiseuille u = U (1 - r^2/R^2) e_z: the wall shear stress is
    mu |du/dr| at r = R = 2 mu U / R = 4.2 dyn/cm^2 (textbook). The P1 gradient in
    the wall-adjacent tets is a secant slope, so SAWSS converges at first order.
    The inner wall of the polygonal tube has area L n_theta 2R sin(pi/n_theta)
    exactly, and the traction the wall puts on the fluid opposes the flow (-z),
    which fixes the orientation of n."""
    mu, U, R, L = 0.035, 30.0, 0.5, 4.0
    exact = 2.0 * mu * U / R
    errs = []
    for nz, nt, nrf, nrw in ((12, 8, 3, 1), (24, 16, 6, 2), (48, 32, 12, 4)):
        m = vm.tube_mesh(nz, nt, nrf, nrw, jitter=0.0)
        y = vm.poiseuille_state(m)
        _, w, a, s = O.wall_shear_stress(m.X, m.tets, m.tet_domain, m.node_problem, y, mu)
        assert abs(a.sum() - L * nt * 2 * R * np.sin(np.pi / nt)) < 1e-12 * a.sum()
        assert (w[:, 2] < 0).all()
        errs.append(abs(s[0] - exact))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 1.5 and errs[2] < 0.05 * exact


def test_wss_ignores_pressure_and_rigid_rotation():
    """The tangential projection removes -p n whatever p is, and a rigid rotation
    u = omega x X has eps(u) = 0, so its WSS vanishes (a transposed or unsymmetrised
    velocity gradient would not)."""
    m = vm.tube_config("tube-12x8x4")
    y = vm.poiseuille_state(m)
    _, w, _, _ = O.wall_shear_stress(m.X, m.tets, m.tet_domain, m.node_problem, y, 0.035)
    y2 = y.copy()
    y2[:, 3] += 100.0 + 3.0 * m.X[:, 0] - 7.0 * m.X[:, 2]
    _, w2, _, _ = O.wall_shear_stress(m.X, m.tets, m.tet_domain, m.node_problem, y2, 0.035)
    assert np.abs(w2 - w).max() < 1e-12 * np.abs(w).max() * 100
    y3 = np.zeros_like(y)
    y3[:, 0:3] = np.cross(np.array([0.3, -1.2, 0.7]), m.X)
    _, w3, _, _ = O.wall_shear_stress(m.X, m.tets, m.tet_domain, m.node_problem, y3, 0.035)
    assert np.abs(w3).max() < 1e-13


def test_wss_face_set_is_the_algorithm_1_interface():
    """The oracle's inner-wall faces (a dictionary over sorted vertex triples) are
    exactly the interface faces of the mesh generator's Algorithm 1 walk (a sort
    of all faces), on a single tube and on a batch of three."""
    parts = [vm.tube_config("tube-12x8x4"), vm.tube_mesh(6, 8, 2, 1, radius=0.6, length=2.0, seed=9)]
    for m in parts + [vm.concat_meshes(parts)]:
        faces = O.wss_faces(m.tets, m.tet_domain, m.node_problem)
        mine = {tuple(sorted(int(m.tets[t, a]) for a in range(4) if a != f)) for t, f in faces}
        ref = {tuple(sorted(int(v) for v in tri)) for tri in vm.interface_faces(m.tets, m.tet_domain)}
        assert mine == ref and len(mine) == len(faces)


# ---------------------------------------------------------------------------
# interface traction balance through the coupled rows (Sec. 2.1 interface
# conditions, Sec. 2.2 Eq. 6-7): a pressurised lumen loads the wall only through
# the fluid momentum that the interface d rows receive
# ---------------------------------------------------------------------------
def _coupled_lame(n_theta, n_rw):
    """Coupled ring under a lumen at rest with uniform pressure P.

    Fluid and wall of a short tube segment; u is held at 0 and p at P by leaving
    their rows and columns out of the solve, and the d unknowns are solved from
    the oracle's own d rows: wall momentum at wall nodes, fluid + wall momentum at
    interface nodes, harmonic mesh motion at fluid-only nodes. The end planes are
    axial rollers (d_z = 0) and the x = 0 / y = 0 planes symmetry planes, so the
    wall is in plane strain, which is the Lame closed form's setting. dt is huge
    and the previous levels are the reference state, so inertia and the mesh
    velocity vanish. The fluid's traction reaches the wall only through the
    interface routing: nothing else puts a load on it.
    """
    g = GOLDEN["lame"]
    a, b, Pp = g["a"], g["b"], g["P"]
    mat = dict(MAT, E_s=g["E"], nu_s=g["nu"])
    L = 0.2
    m = vm.tube_mesh(2, n_theta, 2, n_rw, radius=a, length=L, wall=b - a, jitter=0.0)
    tag = m.node_tag & ~np.uint32(vm.INLET | vm.OUTLET | vm.WALL_END)   # the test sets its own ends
    P = O.Problem(m.X, m.tets, m.tet_domain, tag, m.node_problem, m.inlets, mat=mat, dt=1e8)
    N = m.n_nodes
    fl = (tag & vm.FLUID) != 0
    y = np.zeros((N, 7))
    y[fl, 3] = Pp
    yref = y.copy()
    z = m.X[:, 2]
    rr = np.hypot(m.X[:, 0], m.X[:, 1])
    th = np.arctan2(m.X[:, 1], m.X[:, 0])
    axis = rr < 1e-12
    fix = np.zeros((N, 3), dtype=bool)
    fix[:, 2] = (z < 1e-12) | (z > L - 1e-12)
    fix[:, 0] = axis | np.isclose(np.abs(np.cos(th)), 0.0, atol=1e-9)
    fix[:, 1] = axis | np.isclose(np.abs(np.sin(th)), 0.0, atol=1e-9)
    dof = (7 * np.arange(N)[:, None] + np.arange(4, 7)[None, :])[~fix]
    load = None
    for _ in range(8):
        F = P.residual(y, yref, yref, 1.0).reshape(-1)[dof]
        if load is None:
            load = np.linalg.norm(F)
        if np.linalg.norm(F) <= 1e-11 * load:
            break
        J = P.jacobian(y, yref, yref, 1.0)[dof][:, dof].tocsc()
        import scipy.sparse.linalg as spla
        yv = y.reshape(-1)
        yv[dof] -= spla.spsolve(J, F)
        y = yv.reshape(N, 7)
    d = y[:, 4:7]
    ur = np.where(axis, 0.0, (d[:, 0] * m.X[:, 0] + d[:, 1] * m.X[:, 1]) / np.where(axis, 1.0, rr))
    return ur[np.isclose(rr, a)].mean(), ur[np.isclose(rr, b)].mean()


def test_interface_traction_balance_coupled_lame():
    """The wall displacement under the fluid's pressure converges at O(h^2) to
    the plane-strain Lame values u_r(a) = 8.458e-5 cm, u_r(b) = 7.250e-5 cm: the
    fluid momentum that the interface d rows receive is the traction -sigma_f n_f
    = P n_f that the wall must balance (sigma_s n_s = -sigma_f n_f, Sec. 2.1)."""
    g = GOLDEN["lame"]
    ua1, ub1 = _coupled_lame(16, 2)
    ua2, ub2 = _coupled_lame(32, 4)
    ea1, ea2 = abs(ua1 - g["u_r_a"]), abs(ua2 - g["u_r_a"])
    eb1, eb2 = abs(ub1 - g["u_r_b"]), abs(ub2 - g["u_r_b"])
    assert ua2 > 0 and ub2 > 0
    assert ea2 < ea1 / 3.0 and eb2 < eb1 / 3.0, (ua1, ua2, ub1, ub2)
    assert ea2 / g["u_r_a"] < 0.02 and eb2 / g["u_r_b"] < 0.02, (ua2, ub2)


@pytest.mark.parametrize("mutation", ["dropped", "flipped", "to_u_rows"])
def test_interface_traction_pin_catches_wrong_routing(monkeypatch, mutation):
    """A routing that drops the fluid momentum at interface nodes, flips its sign
    or sends it to the u rows fails the coupled Lame pin (the mistake is planted in
    the oracle, on the CPU)."""
    def routed(Rm, Rc, Rh, itf):
        i3 = itf[:, :, None]
        out = np.zeros(Rm.shape[:2] + (7,), dtype=np.result_type(Rm, Rc, Rh))
        out[:, :, 3] = Rc
        if mutation == "dropped":
            out[:, :, 0:3] = np.where(i3, 0.0, Rm)
            out[:, :, 4:7] = np.where(i3, 0.0, Rh)
        elif mutation == "flipped":
            out[:, :, 0:3] = np.where(i3, 0.0, Rm)
            out[:, :, 4:7] = np.where(i3, -Rm, Rh)
        else:
            out[:, :, 0:3] = Rm
            out[:, :, 4:7] = np.where(i3, 0.0, Rh)
        return out

    monkeypatch.setattr(O.Problem, "route_fluid", staticmethod(routed))
    g = GOLDEN["lame"]
    ua, ub = _coupled_lame(16, 2)
    assert abs(ua - g["u_r_a"]) / g["u_r_a"] > 0.5 and abs(ub - g["u_r_b"]) / g["u_r_b"] > 0.5, (ua, ub)


# ---------------------------------------------------------------------------
# inflow waveform (Eq. 3 inlet condition u_f = v_f^d; the workloads' pulsatile
# waveform with period 0.8 s)
# ---------------------------------------------------------------------------
def test_inlet_waveform_and_profile():
    """U(t) = 30 (1 + 0.5 sin(2 pi t/0.8)) at t = 0, T/8, T/4, T/2, 3T/4 where the
    sine takes the values 0, sqrt2/2, 1, 0, -1; the parabola is U on the axis, 3U/4
    at r = R/2 and 0 from r = R on; the direction is the inlet normal."""
    g = GOLDEN["inlet_waveform"]
    R = g["R"]
    n = np.array([0.0, 0.6, 0.8])
    e1 = np.array([1.0, 0.0, 0.0])
    c = np.array([0.3, -0.2, 1.0])
    inlet = dict(center=c, normal=n, radius=R, peak=g["peak"], amp=g["amp"], freq=1.0 / g["period"], phase=0.0)
    X = np.stack([c + 2.0 * n, c + 0.5 * R * e1 - 1.0 * n, c + R * e1, c + 1.5 * R * e1])
    for t, U in g["t_U"]:
        u = O.inlet_profile(X, inlet, t)
        assert np.allclose(u[0], U * n, rtol=1e-13, atol=1e-12), (t, u[0], U)
        assert np.allclose(u[1], g["profile_half_radius"] * U * n, rtol=1e-13, atol=1e-12)
        assert np.all(u[2:] == 0.0)


def test_inlet_rows_use_the_waveform_at_the_step_end():
    """The inlet constraint rows of F(y) hold u - u_in(t) at the time the step
    ends: at y = 0 an inlet node on the axis has F_u = -U(t) n."""
    g = GOLDEN["inlet_waveform"]
    m = vm.tube_mesh(2, 4, 1, 1, radius=0.5, length=1.0, jitter=0.0, peak=g["peak"], amp=g["amp"],
                     freq=1.0 / g["period"])
    P = make_problem(m)
    on_axis = (np.hypot(m.X[:, 0], m.X[:, 1]) < 1e-12) & ((m.node_tag & vm.INLET) != 0)
    assert on_axis.sum() == 1
    y = np.zeros((m.n_nodes, 7))
    for t, U in g["t_U"]:
        F = P.residual(y, y, y, t)
        assert np.allclose(F[on_axis, 0:3], [0.0, 0.0, -U], rtol=1e-13, atol=1e-12), (t, F[on_axis])
