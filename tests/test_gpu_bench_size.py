"""Assembly and SpMV parity at the size of the benchmarked tube (96 x 32 x (12 + 3)
cells, 46,657 nodes, 267,264 tets) with the options the benchmark runs (512
subdomains, ILU(1), RCM), through the C ABI.

The residual is compared with the oracle's residual (Eq. 10) and the SpMV with
the oracle's directional derivative of the residual taken by the complex step,
J(y) x = Im F(y + i h x) / h (h = 1e-30; exact up to rounding because every
residual routine of the oracle is analytic), so no matrix is formed on the CPU.
Tolerance 1e-12 relative per field group (FP64 assembly parity).
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
OPTS = dict(n_subdomains=512, ilu_level=1, ordering=1, jac_lag=3)


def rel_by_group(a, b):
    return {g: np.abs(a[:, c] - b[:, c]).max() / max(np.abs(b[:, c]).max(), 1e-300) for g, c in GROUPS.items()}


@pytest.fixture(scope="module")
def bench_tube():
    m = vm.tube_config("tube-96x32x15")
    rng = np.random.default_rng(60)
    y0 = vm.poiseuille_state(m)
    fl = ((m.node_tag & vm.FLUID) != 0)[:, None]
    sc = np.array([1, 1, 1, 3, 1e-5, 1e-5, 1e-5])
    y = y0 + rng.normal(size=y0.shape) * sc
    y[:, 0:4] *= fl
    y1 = y0 + rng.normal(size=y0.shape) * sc * 0.1
    y1[:, 0:4] *= fl
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MAT, dt=1e-3)
    return m, P, y, y1


def test_bench_size_residual_matches_oracle(bench_tube):
    m, P, y, y1 = bench_tube
    Fo = P.residual(y, y1, y1, 0.3 + 1e-3)
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(**OPTS))
    S.set_state(y1, t=0.3)
    rel = rel_by_group(S.residual(y), Fo)
    assert all(v < 1e-12 for v in rel.values()), rel


@pytest.mark.parametrize("threads_per_row", [32, 16])
def test_bench_size_spmv_matches_complex_step(bench_tube, threads_per_row):
    m, P, y, y1 = bench_tube
    x = np.random.default_rng(61).normal(size=(m.n_nodes, 7)) * np.array([1, 1, 1, 3, 1e-5, 1e-5, 1e-5])
    h = 1e-30
    Jx = P.residual(y + 1j * h * x, y1, y1, 0.3 + 1e-3).imag / h
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(threads_per_row=threads_per_row, **OPTS))
    S.set_state(y1, t=0.3)
    S.jacobian(y)
    out = S.vec()
    fsi.fsi_spmv(S.ctx, S.vec(x), out)
    rel = rel_by_group(out.cpu().numpy(), Jx)
    assert all(v < 1e-12 for v in rel.values()), rel
