"""The CUDA restricted additive Schwarz preconditioner (Sec. 3, Eq. 14-16) against
the oracle's plain definition of it (oracle/ras_oracle.py): same partition,
overlap, subdomain ordering (Sec. 4.5) and ILU(k) fill (Sec. 4.3), element by
element, through the C ABI (fsi_pc_apply).

Tolerances come from the conditioning of each case, measured on the oracle
itself: how far its own apply moves when its Jacobian is perturbed the way the
GPU's differs from it.
- FP64: the two Jacobians agree to 1e-12 (assembly parity) and the two sides
  invert the 7x7 pivots differently (Gauss-Jordan against LAPACK), both exact to
  rounding. The sensitivity s64 is the oracle's change under a relative 1e-12
  perturbation of every entry of J; the bound is max(1e-10, 10 s64) per field
  group. For well-conditioned factors s64 is ~1e-12 and the bound is 1e-10; an
  incomplete factorisation with small pivots (ILU(0) on one subdomain of this
  coupled system) amplifies 1e-12 up to ~1e-1, and then only the structure
  (partition, overlap, order, fill) is pinned, by the plan counts.
- Mixed: the GPU assembles the Jacobian in FP32 (within 2e-5 relative of the
  FP64 one per field group, the bound test_jacobian_mixed_is_fp32_accurate
  pins) and factors and solves in FP32. Two oracle measurements bound that: d32,
  the distance of the oracle's own FP32 run (dtype=float32: block elimination,
  pivot inverses and solves in numpy FP32) from its FP64 apply, the error of FP32
  arithmetic on this case; and sJ, the oracle's change under a relative 2e-5
  perturbation of every entry of J, the effect of the assembly error. The bound
  is max(1e-5, 10 d32, sJ) per field group against FP64.
"""
import numpy as np
import pytest

import vesselmesh as vm
from oracle import fsi_oracle as O
from oracle import ras_oracle as RO

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1810_04289_gb300 import fsi  # noqa: E402

MAT = dict(O.DEFAULT_MATERIAL)
GROUPS = {"u": [0, 1, 2], "p": [3], "d": [4, 5, 6]}


def rel_by_group(a, b):
    return {g: np.abs(a[:, c] - b[:, c]).max() / max(np.abs(b[:, c]).max(), 1e-300) for g, c in GROUPS.items()}


def node_rank(m):
    """0 lumen, 1 interface, 2 wall-only: the rank of the lumen-first ordering."""
    tag = m.node_tag
    return np.where((tag & vm.INTERFACE) != 0, 1, np.where((tag & vm.FLUID) != 0, 0, 2))


@pytest.fixture(scope="module")
def case():
    m = vm.tube_config("tube-12x8x4")
    rng = np.random.default_rng(50)
    y0 = vm.poiseuille_state(m)
    fl = ((m.node_tag & vm.FLUID) != 0)[:, None]
    y = y0 + rng.normal(size=y0.shape) * np.array([1, 1, 1, 3, 1e-5, 1e-5, 1e-5]) * 0.1
    y[:, 0:4] *= fl
    P = O.Problem(m.X, m.tets, m.tet_domain, m.node_tag, m.node_problem, m.inlets, mat=MAT, dt=1e-3)
    J = P.jacobian(y, y0, y0, 0.25 + 1e-3)
    r = rng.normal(size=(m.n_nodes, 7))
    return m, y, y0, J, r


def gpu_apply(m, y, y0, r, **opt):
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(**opt))
    S.set_state(y0, t=0.25)
    S.jacobian(y)
    z = S.vec()
    fsi.fsi_pc_apply(S.ctx, S.vec(r), z)
    out = z.cpu().numpy()
    info = S.info()
    S.close()
    return out, info


def oracle_apply(m, J, r, nsub, ilu, ordering, overlap=1):
    ras = RO.RAS(J, m.X, m.tets, m.node_problem, m.n_problems, nsub, overlap, ilu, ordering, node_rank(m))
    return ras.apply(r), ras


def tolerance(m, J, r, z, nsub, ilu, ordering, fp32, overlap=1):
    """Per field group bound from the oracle's own behaviour (see the module notes)."""
    if fp32:
        ras = RO.RAS(J, m.X, m.tets, m.node_problem, m.n_problems, nsub, overlap, ilu, ordering, node_rank(m),
                     dtype=np.float32)
        d32 = rel_by_group(ras.apply(r), z)
        Jp = J.copy()
        Jp.data = Jp.data * (1.0 + 2e-5 * np.random.default_rng(3).normal(size=Jp.data.shape))
        zp, _ = oracle_apply(m, Jp, r, nsub, ilu, ordering, overlap)
        sJ = rel_by_group(zp, z)
        return {g: max(1e-5, 10 * d32[g], sJ[g]) for g in d32}
    Jp = J.copy()
    Jp.data = Jp.data * (1.0 + 1e-12 * np.random.default_rng(5).normal(size=Jp.data.shape))
    zp, _ = oracle_apply(m, Jp, r, nsub, ilu, ordering, overlap)
    sens = rel_by_group(zp, z)
    return {g: max(1e-10, 10 * v) for g, v in sens.items()}


def within(rel, tol):
    return all(rel[g] < tol[g] for g in rel)


CASES = [(ilu, ordering, nsub) for ilu in (0, 1, 2, 3) for ordering in (0, 1, 2, 3) for nsub in (1, 4, 64)]


@pytest.mark.parametrize("ilu,ordering,nsub", CASES)
def test_pc_apply_fp64_matches_oracle(case, ilu, ordering, nsub):
    m, y, y0, J, r = case
    zo, ras = oracle_apply(m, J, r, nsub, ilu, ordering)
    zg, info = gpu_apply(m, y, y0, r, n_subdomains=nsub, ilu_level=ilu, ordering=ordering)
    assert info.n_subdomains == len(ras.subs)
    assert info.factor_rows == sum(len(s["order"]) for s in ras.subs)
    assert info.factor_blocks == sum(int(s["keep"].sum()) for s in ras.subs)
    rel = rel_by_group(zg, zo)
    tol = tolerance(m, J, r, zo, nsub, ilu, ordering, fp32=False)
    assert within(rel, tol), (rel, tol)


@pytest.mark.parametrize("ilu,ordering,nsub", [(1, 1, 4), (2, 1, 4), (2, 2, 64), (1, 0, 64), (2, 3, 1), (1, 3, 4)])
def test_pc_apply_mixed_matches_oracle(case, ilu, ordering, nsub):
    m, y, y0, J, r = case
    zo, _ = oracle_apply(m, J, r, nsub, ilu, ordering)
    zg, _ = gpu_apply(m, y, y0, r, precision=1, n_subdomains=nsub, ilu_level=ilu, ordering=ordering)
    rel = rel_by_group(zg, zo)
    tol = tolerance(m, J, r, zo, nsub, ilu, ordering, fp32=True)
    assert within(rel, tol), (rel, tol)


@pytest.mark.parametrize("precision,ilu,nsub,ordering", [(0, 1, 4, 1), (0, 2, 64, 1), (0, 3, 1, 1), (1, 2, 4, 1),
                                                          (0, 2, 4, 3), (1, 1, 4, 3)])
def test_level_scheduled_apply_matches_oracle(case, precision, ilu, nsub, ordering):
    """apply_mode 2 forces the level-scheduled apply (the kernel taken when the
    streamed one does not fit in shared memory)."""
    m, y, y0, J, r = case
    zo, _ = oracle_apply(m, J, r, nsub, ilu, ordering)
    zs, i1 = gpu_apply(m, y, y0, r, precision=precision, n_subdomains=nsub, ilu_level=ilu, ordering=ordering,
                       apply_mode=1)
    zl, i2 = gpu_apply(m, y, y0, r, precision=precision, n_subdomains=nsub, ilu_level=ilu, ordering=ordering,
                       apply_mode=2)
    assert i1.apply_kernel == 1 and i2.apply_kernel == 2
    tol = tolerance(m, J, r, zo, nsub, ilu, ordering, fp32=precision == 1)
    for z in (zs, zl):
        rel = rel_by_group(z, zo)
        assert within(rel, tol), (rel, tol)
    # the two kernels sum each row in a different order only
    rel = rel_by_group(zl, zs)
    assert within(rel, tol), (rel, tol)


def test_pc_apply_overlap_two_matches_oracle(case):
    m, y, y0, J, r = case
    zo, _ = oracle_apply(m, J, r, 8, 1, 1, overlap=2)
    zg, _ = gpu_apply(m, y, y0, r, n_subdomains=8, ilu_level=1, overlap=2)
    rel = rel_by_group(zg, zo)
    tol = tolerance(m, J, r, zo, 8, 1, 1, fp32=False, overlap=2)
    assert within(rel, tol), (rel, tol)


def test_bilu0_one_subdomain_on_a_rigid_tube_is_not_exact_but_ilu_full_is(case):
    """Special cases on the GPU: one subdomain with every fill level the mesh can
    create (ILU(3) on this small tube keeps far more than ILU(1)) brings J B^{-1} r
    closer to r than ILU(0) does (the residual of the preconditioned system falls
    with the fill level)."""
    m, y, y0, J, r = case
    res = []
    for ilu in (0, 1, 3):
        zg, _ = gpu_apply(m, y, y0, r, n_subdomains=1, ilu_level=ilu)
        res.append(np.linalg.norm(r.reshape(-1) - J @ zg.reshape(-1)))
    assert res[2] < res[1] < res[0], res
