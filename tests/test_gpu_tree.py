"""Newton parity on a bifurcating tree (Kuhn-voxel mesh, Algorithm 1 interface,
junctions, four outlets, voxel caps, clamped wall ends), the geometry of the
tree workloads at a size the oracle solves in seconds.

Both sides start from the same steady rigid-wall Stokes state, computed by the
oracle (the initial state of the tree workloads), and take backward-Euler steps
to Newton rtol 1e-10; the GPU uses ILU(2), the level the tree workloads run
with. Tolerances: 1e-8 relative per field group in FP64, 1e-6 in mixed
precision.
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
N_STEPS = 2


def rel_by_group(a, b):
    return {g: np.abs(a[:, c] - b[:, c]).max() / max(np.abs(b[:, c]).max(), 1e-300) for g, c in GROUPS.items()}


@pytest.fixture(scope="module")
def tree_case():
    m = vm.tree_mesh(generations=3, r0=0.2, h=0.08, seed=7)
    assert ((m.node_tag & vm.OUTLET) != 0).sum() > 0 and m.info["leaves"] == 4
    Ps = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=dict(MAT, rho_f=0.0),
                   dt=1e8, rigid_wall=True)
    z = np.zeros((m.n_nodes, 7))
    y0, _ = O.newton_solve(Ps, z, z, 0.0, rtol=1e-10)
    y0[:, 4:7] = 0.0
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MAT, dt=1e-3)
    ref = [y for y, _ in O.run_steps(P, y0, N_STEPS)]
    return m, y0, ref


@pytest.mark.parametrize("precision,tol,gmres_rtol", [(0, 1e-8, 1e-6), (1, 1e-6, 1e-4)])
def test_tree_newton_steps_match_oracle(tree_case, precision, tol, gmres_rtol):
    m, y0, ref = tree_case
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(precision=precision, newton_rtol=1e-10, gmres_rtol=gmres_rtol,
                                                  n_subdomains=16, ilu_level=2))
    S.set_state(y0, t=0.0)
    for k in range(N_STEPS):
        st = S.step()
        y, _ = S.state()
        rel = rel_by_group(y, ref[k])
        assert st.converged == 1
        assert all(v < tol for v in rel.values()), (k, rel)


def test_tree_residual_matches_oracle(tree_case):
    """F at a state off the solution (the step's solution plus noise), where F is
    not small, so the comparison is not one of rounding noise."""
    m, y0, ref = tree_case
    rng = np.random.default_rng(70)
    fl = ((m.node_tag & vm.FLUID) != 0)[:, None]
    y = ref[0] + rng.normal(size=ref[0].shape) * np.array([1, 1, 1, 3, 1e-5, 1e-5, 1e-5])
    y[:, 0:4] *= fl
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MAT, dt=1e-3)
    Fo = P.residual(y, y0, y0, 1e-3)
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=16))
    S.set_state(y0, t=0.0)
    rel = rel_by_group(S.residual(y), Fo)
    assert all(v < 1e-12 for v in rel.values()), rel
