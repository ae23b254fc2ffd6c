"""Wall shear stress through the C ABI (fsi_wss, fsi_wss_faces) against the FP64
oracle's WSS and SAWSS on the same states: same faces in the same order, per-face
WSS vectors and per-problem SAWSS to 1e-12 relative."""
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


def _state(m, seed):
    rng = np.random.default_rng(seed)
    y = vm.poiseuille_state(m)
    y = y + rng.normal(size=y.shape) * np.array([3, 3, 3, 10, 1e-3, 1e-3, 1e-3])
    y[:, 0:4] *= ((m.node_tag & vm.FLUID) != 0)[:, None]
    return y


def _check(m, y, n_problems):
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    faces, w, sawss = S.wss(y)
    of, ow, oa, osawss = O.wall_shear_stress(m.X, m.tets, m.tet_domain, m.node_problem, y, MAT["mu_f"],
                                             n_problems)
    assert np.array_equal(faces.astype(np.int64), of)
    assert np.abs(w - ow).max() <= 1e-12 * np.abs(ow).max()
    assert np.all(np.abs(sawss - osawss) <= 1e-12 * np.abs(osawss))
    assert S.info().n_wss_faces == len(of)
    S.close()
    return osawss


@pytest.mark.parametrize("seed", [0, 1])
def test_wss_matches_oracle_on_a_moving_tube(seed):
    m = vm.tube_config("tube-12x8x4")
    s = _check(m, _state(m, seed), 1)
    assert s[0] > 0


def test_wss_per_problem_in_a_batch():
    parts = [vm.tube_config("tube-12x8x4"),
             vm.tube_mesh(10, 6, 3, 1, radius=0.35, length=3.0, jitter=0.08, seed=5, peak=20.0, phase=1.3),
             vm.tube_mesh(6, 8, 2, 1, radius=0.6, length=2.0, jitter=0.0, seed=9, peak=45.0, amp=0.2, phase=4.0)]
    batch = vm.concat_meshes(parts)
    y = np.concatenate([_state(p, k) for k, p in enumerate(parts)])
    s = _check(batch, y, 3)
    # each problem's SAWSS is its own: equal to the single-tube value
    off = 0
    for k, p in enumerate(parts):
        yp = y[off:off + p.n_nodes]
        off += p.n_nodes
        _, _, _, sp = O.wall_shear_stress(p.X, p.tets, p.tet_domain, p.node_problem, yp, MAT["mu_f"], 1)
        assert abs(sp[0] - s[k]) <= 1e-12 * abs(sp[0])
