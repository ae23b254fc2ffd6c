"""Parity of the CUDA solver (through the C ABI) with the CPU FP64 oracle.

Tolerances: FP64 assembly 1e-12 relative (max norm per field row group), FP64
Newton solutions 1e-8 relative, mixed-precision Newton solutions 1e-6 relative.
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


def oracle_problem(m, dt=1e-3, rigid=False):
    return O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MAT, dt=dt,
                     rigid_wall=rigid)


def perturbed_states(m, seed, scale=(3, 3, 3, 10, 1e-4, 1e-4, 1e-4)):
    rng = np.random.default_rng(seed)
    y0 = vm.poiseuille_state(m)
    fl = ((m.node_tag & vm.FLUID) != 0)[:, None]
    sc = np.array(scale)
    out = []
    for _ in range(3):
        y = y0 + rng.normal(size=y0.shape) * sc
        y[:, 0:4] *= fl                     # wall-only u, p slots stay 0
        out.append(y)
    return out


def rel_by_group(a, b):
    """max |a-b| / max |b| over each field group of the node-major (N,7) arrays."""
    return {g: np.abs(a[:, c] - b[:, c]).max() / max(np.abs(b[:, c]).max(), 1e-300) for g, c in GROUPS.items()}


def jac_rel_by_group(Jg, Jo):
    D = (Jg - Jo).tocsr()
    out = {}
    for g, cols in GROUPS.items():
        rows = np.concatenate([np.arange(c, Jo.shape[0], 7) for c in cols])
        dm = abs(D[rows]).max() if D[rows].nnz else 0.0
        om = abs(Jo[rows]).max()
        out[g] = dm / om
    return out


@pytest.fixture(scope="module")
def tube0():
    return vm.tube_config("tube-12x8x4")


def make_solver(m, **opt):
    o = fsi.fsi_default_options(**opt)
    return fsi.Solver(m, MAT, o)


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_residual_matches_oracle(tube0, seed):
    m = tube0
    y, y1, y2 = perturbed_states(m, seed)
    t1 = 0.25
    P = oracle_problem(m)
    Fo = P.residual(y, y1, y2, t1 + P.dt)
    S = make_solver(m)
    S.set_state(y1, y2, None, t=t1)
    Fg = S.residual(y)
    rel = rel_by_group(Fg, Fo)
    assert all(v < 1e-12 for v in rel.values()), rel


def test_residual_small_meshes_and_rigid_wall():
    for m, rigid in ((vm.tube_mesh(2, 4, 1, 1, seed=5), False), (vm.tube_mesh(3, 6, 2, 2, seed=6), True)):
        y, y1, y2 = perturbed_states(m, 3)
        P = oracle_problem(m, rigid=rigid)
        Fo = P.residual(y, y1, y2, 0.5 + P.dt)
        S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=2), rigid_wall=rigid)
        S.set_state(y1, y2, None, t=0.5)
        rel = rel_by_group(S.residual(y), Fo)
        assert all(v < 1e-12 for v in rel.values()), rel


@pytest.mark.parametrize("seed", [0, 1])
def test_jacobian_fp64_matches_oracle(tube0, seed):
    m = tube0
    y, y1, y2 = perturbed_states(m, 10 + seed)
    P = oracle_problem(m)
    Jo = P.jacobian(y, y1, y2, 0.25 + P.dt)
    S = make_solver(m)
    S.set_state(y1, y2, None, t=0.25)
    S.jacobian(y)
    Jg = S.jacobian_csr()
    rel = jac_rel_by_group(Jg, Jo)
    assert all(v < 1e-12 for v in rel.values()), rel


def test_jacobian_mixed_is_fp32_accurate(tube0):
    m = tube0
    y, y1, y2 = perturbed_states(m, 20)
    P = oracle_problem(m)
    Jo = P.jacobian(y, y1, y2, 0.25 + P.dt)
    S = make_solver(m, precision=1)
    S.set_state(y1, y2, None, t=0.25)
    S.jacobian(y)
    rel = jac_rel_by_group(S.jacobian_csr(), Jo)
    assert all(v < 2e-5 for v in rel.values()), rel


def test_spmv_matches_oracle_product(tube0):
    m = tube0
    y, y1, y2 = perturbed_states(m, 30)
    P = oracle_problem(m)
    Jo = P.jacobian(y, y1, y2, 0.25 + P.dt)
    S = make_solver(m)
    S.set_state(y1, y2, None, t=0.25)
    S.jacobian(y)
    x = np.random.default_rng(31).normal(size=(m.n_nodes, 7))
    out = S.vec()
    fsi.fsi_spmv(S.ctx, S.vec(x), out)
    ref = (Jo @ x.reshape(-1)).reshape(-1, 7)
    rel = rel_by_group(out.cpu().numpy(), ref)
    assert all(v < 1e-12 for v in rel.values()), rel


# ---------------------------------------------------------------------------
# linear solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision,nsub", [(0, 1), (0, 4), (1, 4)])
def test_linear_solve_matches_direct_solve(tube0, precision, nsub):
    import scipy.sparse.linalg as spla
    m = tube0
    y, y1, y2 = perturbed_states(m, 40)
    P = oracle_problem(m)
    Jo = P.jacobian(y, y1, y2, 0.25 + P.dt)
    b = P.residual(y, y1, y2, 0.25 + P.dt)
    xo = spla.spsolve(Jo.tocsc(), b.reshape(-1)).reshape(-1, 7)
    # an FP32 operator limits the attainable relative residual to ~1e-6
    rtol = 1e-10 if precision == 0 else 1e-5
    S = make_solver(m, precision=precision, n_subdomains=nsub, gmres_rtol=rtol, gmres_maxit=600)
    S.set_state(y1, y2, None, t=0.25)
    S.jacobian(y)
    x = S.vec()
    st = fsi.fsi_linear_solve(S.ctx, S.vec(b), x)
    assert st.converged == 1 and st.rnorm <= rtol * st.rnorm0 * 1.0001
    xg = x.cpu().numpy()
    tol = 1e-6 if precision == 0 else 1e-2
    rel = rel_by_group(xg, xo)
    assert all(v < tol for v in rel.values()), (rel, st.iterations)


# ---------------------------------------------------------------------------
# Newton steps
# ---------------------------------------------------------------------------
def _oracle_steps(m, n):
    P = oracle_problem(m)
    y0 = vm.poiseuille_state(m)
    return y0, [y for y, _ in O.run_steps(P, y0, n)]


@pytest.fixture(scope="module")
def oracle_tube0_steps(tube0):
    return _oracle_steps(tube0, 5)


def test_newton_steps_fp64_match_oracle(tube0, oracle_tube0_steps):
    y0, ref = oracle_tube0_steps
    S = make_solver(tube0, newton_rtol=1e-10, gmres_rtol=1e-6, n_subdomains=4)
    S.set_state(y0, t=0.0)
    for k in range(5):
        st = S.step()
        y, t = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert all(v < 1e-8 for v in rel.values()), (k, rel)
        assert abs(t - (k + 1) * 1e-3) < 1e-15


def test_newton_steps_mixed_match_oracle(tube0, oracle_tube0_steps):
    y0, ref = oracle_tube0_steps
    S = make_solver(tube0, precision=1, newton_rtol=1e-10, gmres_rtol=1e-4, n_subdomains=4)
    S.set_state(y0, t=0.0)
    for k in range(5):
        st = S.step()
        y, _ = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert all(v < 1e-6 for v in rel.values()), (k, rel)


@pytest.mark.parametrize("precision,ilu,ordering", [(0, 1, 1), (1, 2, 1), (0, 2, 3), (1, 1, 3)])
def test_factor_shared_memory_modes_are_bitwise_identical(tube0, precision, ilu, ordering):
    """The shared-memory modes of the ILU factorisation (pivots and sources
    prefetched / sources only / neither) and the nested-dissection grouped
    kernel (ordering 3) do the same arithmetic in the same order, so the
    preconditioner applies agree bit for bit."""
    y = vm.poiseuille_state(tube0)
    r = torch.randn((tube0.n_nodes, 7), dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    outs = []
    for mode in ((1, 2, 3) if ordering != 3 else (3, 4)):
        S = make_solver(tube0, precision=precision, ilu_level=ilu, n_subdomains=4, ordering=ordering,
                        factor_mode=mode)
        S.set_state(y, t=0.0)
        S.jacobian(y)
        z = S.vec()
        fsi.fsi_pc_apply(S.ctx, r, z)
        outs.append(z.cpu().numpy())
        S.close()
    assert np.isfinite(outs[0]).all()
    assert all(np.array_equal(outs[0], o) for o in outs[1:])


def test_newton_steps_with_jacobian_lag_match_oracle(tube0, oracle_tube0_steps):
    """Reusing one Jacobian and its factors for three Newton iterations (Eq. 12,
    the paper's Jacobian lag) changes the path, not the solution: the steps still
    match the oracle's exact-Newton steps to 1e-8."""
    y0, ref = oracle_tube0_steps
    S = make_solver(tube0, newton_rtol=1e-10, gmres_rtol=1e-6, n_subdomains=4, jac_lag=3)
    S.set_state(y0, t=0.0)
    for k in range(5):
        st = S.step()
        y, _ = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert st.jacobian_evaluations <= -(-st.newton_iterations // 3)
        assert all(v < 1e-8 for v in rel.values()), (k, rel)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_newton_steps_with_selective_reorthogonalisation_match_oracle(tube0, oracle_tube0_steps, precision, tol):
    """orth = 1 (Gram-Schmidt with a second pass only where the first lost more
    than 1 - 1/sqrt(2) of the norm) changes the Krylov basis only at rounding
    level: the Newton steps still match the oracle's."""
    y0, ref = oracle_tube0_steps
    S = make_solver(tube0, precision=precision, newton_rtol=1e-10, gmres_rtol=1e-6 if precision == 0 else 1e-4,
                    n_subdomains=4, orth=1)
    S.set_state(y0, t=0.0)
    for k in range(5):
        st = S.step()
        y, _ = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert all(v < tol for v in rel.values()), (k, rel)


@pytest.mark.parametrize("precision", [0, 1])
def test_chunked_jacobian_assembly_is_bitwise_identical(tube0, precision):
    """The element Jacobians assembled in chunks of tets (jac_chunk; the default
    chunk holds what the factor storage holds) sum into the same BSR values in the
    same order: the matrices are equal bit for bit."""
    y, y1, y2 = perturbed_states(tube0, 90)
    mats = []
    for chunk in (0, 97, 1000):
        S = make_solver(tube0, precision=precision, jac_chunk=chunk)
        S.set_state(y1, y2, None, t=0.25)
        S.jacobian(y)
        mats.append(fsi.fsi_jacobian_export(S.ctx)[2])
        S.close()
    assert np.array_equal(mats[0], mats[1]) and np.array_equal(mats[0], mats[2])


# ---------------------------------------------------------------------------
# Gram-Schmidt forms
# ---------------------------------------------------------------------------
def _solve_fp64_operator(m, **opt):
    """GMRES on the FP64 Jacobian (FP64 preconditioner) to a relative residual of
    1e-10: reachable only if the Arnoldi relation holds to about that accuracy,
    so it measures the orthogonalisation."""
    y, y1, y2 = perturbed_states(m, 40)
    P = oracle_problem(m)
    b = P.residual(y, y1, y2, 0.25 + P.dt)
    S = make_solver(m, n_subdomains=4, gmres_rtol=1e-10, gmres_maxit=600, **opt)
    S.set_state(y1, y2, None, t=0.25)
    S.jacobian(y)
    x = S.vec()
    st = fsi.fsi_linear_solve(S.ctx, S.vec(b), x)
    S.close()
    return st, x.cpu().numpy()


@pytest.mark.parametrize("fault_test", [0, 2])
def test_pythagorean_norm_gram_schmidt_matches_six_sweep_form(tube0, fault_test):
    """orth = 0 takes the new Arnoldi vector's norm from the second pass,
    sqrt(||w||^2 - ||h2||^2), and scales in the second update's sweep. On the
    FP64 operator it reaches a 1e-10 relative residual in the iterations of the
    six-sweep form (orth = 2) and the direct solve's solution; fault_test = 2
    forms every norm from the updated vector instead (the fallback path)."""
    import scipy.sparse.linalg as spla
    m = tube0
    st2, x2 = _solve_fp64_operator(m, orth=2)
    st0, x0 = _solve_fp64_operator(m, orth=0, fault_test=fault_test)
    for st in (st2, st0):
        assert st.converged == 1 and st.rnorm <= 1e-10 * st.rnorm0 * 1.0001
    assert abs(st0.iterations - st2.iterations) <= 1, (st2.iterations, st0.iterations)
    y, y1, y2 = perturbed_states(m, 40)
    P = oracle_problem(m)
    Jo = P.jacobian(y, y1, y2, 0.25 + P.dt)
    b = P.residual(y, y1, y2, 0.25 + P.dt)
    xo = spla.spsolve(Jo.tocsc(), b.reshape(-1)).reshape(-1, 7)
    for x in (x0, x2):
        rel = rel_by_group(x, xo)
        assert all(v < 1e-6 for v in rel.values()), rel


def test_orth_option_range(tube0):
    with pytest.raises(fsi.FsiError):
        make_solver(tube0, orth=3, n_subdomains=4)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 1e-6)])
def test_newton_steps_with_six_sweep_gram_schmidt_match_oracle(tube0, oracle_tube0_steps, precision, tol):
    """The six-sweep form (orth = 2) gives the oracle's Newton steps too."""
    y0, ref = oracle_tube0_steps
    S = make_solver(tube0, precision=precision, newton_rtol=1e-10, gmres_rtol=1e-6 if precision == 0 else 1e-4,
                    n_subdomains=4, orth=2)
    S.set_state(y0, t=0.0)
    for k in range(5):
        st = S.step()
        y, _ = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert all(v < tol for v in rel.values()), (k, rel)
