"""The allocation-free residual entry point gives the same F(y) as fsi_residual.

fsi_residual_noalloc serves callers that must not have the library allocate
device memory; its assembly scratch is a fixed array inside the library. It is
checked through the C ABI against fsi_residual on two calls in a row (the second
call reuses the array the first one left behind). This file is collected last.
"""
import numpy as np
import pytest

import vesselmesh as vm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("CUDA device required", allow_module_level=True)

from paper_1810_04289_gb300 import fsi  # noqa: E402

MAT = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)


def test_residual_noalloc_matches_residual_twice():
    m = vm.tube_config("tube-12x8x4")
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=4))
    rng = np.random.default_rng(77)
    y0 = vm.poiseuille_state(m)
    fl = ((m.node_tag & vm.FLUID) != 0)[:, None]
    sc = np.array([3, 3, 3, 10, 1e-4, 1e-4, 1e-4])
    S.set_state(y0 + rng.normal(size=y0.shape) * sc * fl, t=0.1)
    for call in range(2):
        y = S.vec(y0 + rng.normal(size=y0.shape) * sc * fl)
        F_ref = S.vec()
        F_new = S.vec()
        fsi.fsi_residual(S.ctx, y, F_ref)
        F_new.fill_(np.nan)
        fsi.fsi_residual_noalloc(S.ctx, y, F_new)
        a, b = F_new.cpu().numpy(), F_ref.cpu().numpy()
        for cols in ([0, 1, 2], [3], [4, 5, 6]):
            err = np.abs(a[:, cols] - b[:, cols]).max() / np.abs(b[:, cols]).max()
            assert err < 1e-12, (call, cols, err)
    S.close()


def test_residual_noalloc_rejects_large_meshes():
    m = vm.tube_config("tube-96x32x15")      # 267,264 tets > 32,768
    S = fsi.Solver(m, MAT, fsi.fsi_default_options(n_subdomains=64))
    y = S.vec(vm.poiseuille_state(m))
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_residual_noalloc(S.ctx, y, S.vec())
    assert "32768" in str(e.value)
    S.close()
