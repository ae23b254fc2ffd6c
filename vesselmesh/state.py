"""Initial states (inputs): the Poiseuille field of a straight tube."""
import numpy as np
from .mesh import FLUID, WALL


def poiseuille_state(mesh, mu=0.035, t=0.0, problem_params=None):
    """u = U(t)(1 - r^2/R^2) n, p = dp (1 - s/L), d = 0 on every tube of the mesh.

    U(t) is the inflow peak at time t, dp = 4 mu U L / R^2 is the Poiseuille
    pressure drop over the tube length L, s is the distance along the axis from the
    inlet. Wall-only nodes get u = 0, p = 0. Returns y (N,7).
    """
    y = np.zeros((mesh.n_nodes, 7))
    fl = (mesh.node_tag & FLUID) != 0
    infos = mesh.info.get("problems", [mesh.info])
    for p, inl in enumerate(mesh.inlets):
        sel = np.nonzero(fl & (mesh.node_problem == p))[0]
        c, n, R = np.asarray(inl["center"]), np.asarray(inl["normal"]), inl["radius"]
        L = infos[p].get("length", 1.0)
        U = inl["peak"] * (1.0 + inl["amp"] * np.sin(2 * np.pi * inl["freq"] * t + inl["phase"]))
        rel = mesh.X[sel] - c
        s = rel @ n
        r2 = np.sum(rel * rel, axis=1) - s * s
        y[sel, 0:3] = (U * np.maximum(0.0, 1.0 - r2 / R ** 2))[:, None] * n[None, :]
        dp = 4.0 * mu * U * L / R ** 2
        y[sel, 3] = dp * (1.0 - s / L)
    return y
