"""Many independent vessel problems advanced together in one set of launches.

The unknowns of the problems are stored one after another; assembly, the
Schwarz preconditioner, the Krylov scalars and the Newton stopping tests are all
per problem, so a batched run must reproduce the independent runs: residuals
bit for bit (element-wise assembly with an ordered gather does not see the
other problems) and Newton solutions within the Newton tolerance. The batched
solution is also checked against the FP64 oracle on the stacked problem.
"""
import numpy as np
import pytest

import vesselmesh as vm
from oracle import fsi_oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1810_04289_gb300 import fsi  # noqa: E402

MAT = dict(O.DEFAULT_MATERIAL)
GROUPS = {"u": [0, 1, 2], "p": [3], "d": [4, 5, 6]}


def rel_by_group(a, b):
    return {g: np.abs(a[:, c] - b[:, c]).max() / max(np.abs(b[:, c]).max(), 1e-300) for g, c in GROUPS.items()}


@pytest.fixture(scope="module")
def parts():
    a = vm.tube_config("tube-12x8x4")
    b = vm.tube_mesh(10, 6, 3, 1, radius=0.35, length=3.0, jitter=0.08, seed=5, peak=20.0, phase=1.3)
    c = vm.tube_mesh(6, 8, 2, 1, radius=0.6, length=2.0, jitter=0.0, seed=9, peak=45.0, amp=0.2, phase=4.0)
    return [a, b, c]


def solver(m, **opt):
    return fsi.Solver(m, MAT, fsi.fsi_default_options(**opt))


def split(y, parts):
    out, off = [], 0
    for m in parts:
        out.append(y[off:off + m.n_nodes])
        off += m.n_nodes
    return out


def test_batched_residual_is_bitwise_concatenation(parts):
    batch = vm.concat_meshes(parts)
    rng = np.random.default_rng(3)
    ys = []
    for m in parts:
        y = vm.poiseuille_state(m)
        y = y + rng.normal(size=y.shape) * np.array([2, 2, 2, 5, 1e-4, 1e-4, 1e-4])
        y[:, 0:4] *= ((m.node_tag & vm.FLUID) != 0)[:, None]
        ys.append(y)
    yb = np.concatenate(ys)
    Sb = solver(batch)
    Sb.set_state(yb, t=0.1)
    Fb = split(Sb.residual(yb), parts)
    for m, y, f in zip(parts, ys, Fb):
        S = solver(m)
        S.set_state(y, t=0.1)
        assert np.array_equal(S.residual(y), f)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_batched_steps_match_independent_and_oracle(parts, precision, tol):
    batch = vm.concat_meshes(parts)
    opts = dict(precision=precision, newton_rtol=1e-10, gmres_rtol=1e-6 if precision == 0 else 1e-4)
    nsteps = 3
    yb0 = np.concatenate([vm.poiseuille_state(m) for m in parts])
    Sb = solver(batch, n_subdomains=6, **opts)
    Sb.set_state(yb0, t=0.0)
    batched = []
    for _ in range(nsteps):
        st = Sb.step()
        assert st.converged == 1
        batched.append(Sb.state()[0].copy())

    for p, m in enumerate(parts):
        S = solver(m, n_subdomains=2, **opts)
        S.set_state(vm.poiseuille_state(m), t=0.0)
        for k in range(nsteps):
            assert S.step().converged == 1
            rel = rel_by_group(split(batched[k], parts)[p], S.state()[0])
            assert all(v < tol for v in rel.values()), (p, k, rel)

    P = O.Problem(batch.X, batch.tets, batch.tet_domain, batch.node_tag, batch.node_problem, batch.inlets, mat=MAT,
                  dt=1e-3)
    ref = [y for y, _ in O.run_steps(P, yb0, nsteps)]
    for k in range(nsteps):
        for p, (yg, yo) in enumerate(zip(split(batched[k], parts), split(ref[k], parts))):
            rel = rel_by_group(yg, yo)
            assert all(v < tol for v in rel.values()), (p, k, rel)


def test_batched_linear_solve_meets_every_problem_tolerance(parts):
    """Each problem's own residual reaches gmres_rtol * ||b_p||, whatever the
    scale of the other problems' right-hand sides."""
    batch = vm.concat_meshes(parts)
    S = solver(batch, n_subdomains=6, gmres_rtol=1e-6)
    y = np.concatenate([vm.poiseuille_state(m) for m in parts])
    S.set_state(y, t=0.0)
    yv = S.vec(y)
    F = S.vec()
    fsi.fsi_residual(S.ctx, yv, F)
    rng = np.random.default_rng(1)
    b = rng.normal(size=(batch.n_nodes, 7))
    scales = [1.0, 1e-6, 1e4]
    off = 0
    for m, s in zip(parts, scales):
        b[off:off + m.n_nodes] *= s
        off += m.n_nodes
    fsi.fsi_jacobian(S.ctx, yv)
    x = S.vec()
    st = fsi.fsi_linear_solve(S.ctx, S.vec(b), x)
    assert st.converged == 1
    r = S.vec()
    fsi.fsi_spmv(S.ctx, x, r)
    rr = b - r.cpu().numpy().reshape(-1, 7)
    for bp, rp in zip(split(b, parts), split(rr, parts)):
        assert np.linalg.norm(rp) <= 1.0001e-6 * np.linalg.norm(bp)
