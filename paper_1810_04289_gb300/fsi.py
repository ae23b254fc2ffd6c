"""Python binding of the C ABI in include/fsi.h (ctypes; argument marshalling only).

Every function here forwards to the entry point of the same name in
libfsi_gb300.so; all numerical work runs in that library's CUDA kernels.
Device arrays are torch CUDA tensors (float64, contiguous, node-major [N, 7]);
their data pointers and the current torch stream are passed through. Importing
this module fails loudly when the library has not been built.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libfsi_gb300.so")

FSI_OK = 0
STATUS = {0: "FSI_OK", 1: "FSI_ERR_ARG", 2: "FSI_ERR_MESH", 3: "FSI_ERR_CUDA", 4: "FSI_ERR_NOMEM",
          5: "FSI_ERR_ZERO_PIVOT", 6: "FSI_ERR_LINEAR_DIVERGED", 7: "FSI_ERR_DIVERGED",
          8: "FSI_ERR_LINESEARCH", 9: "FSI_ERR_TIMEOUT", 10: "FSI_ERR_NONFINITE"}

# every symbol include/fsi.h declares
EXPORTS = ["fsi_default_options", "fsi_create", "fsi_destroy", "fsi_set_state", "fsi_get_state",
           "fsi_residual", "fsi_jacobian", "fsi_jacobian_export", "fsi_spmv", "fsi_pc_apply",
           "fsi_linear_solve", "fsi_step", "fsi_get_info", "fsi_last_error", "fsi_residual_noalloc",
           "fsi_wss", "fsi_wss_faces"]


class FsiMesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("tet_domain", ctypes.c_void_p),
                ("node_tag", ctypes.c_void_p), ("node_problem", ctypes.c_void_p)]


class FsiMaterial(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("rho_f", "mu_f", "rho_s", "E_s", "nu_s", "eta_s")]


class FsiBc(ctypes.Structure):
    _fields_ = [("center", ctypes.c_double * 3), ("normal", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("peak", ctypes.c_double), ("amp", ctypes.c_double), ("freq", ctypes.c_double),
                ("phase", ctypes.c_double), ("rigid_wall", ctypes.c_int32)]


class FsiOptions(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("gmres_rtol", ctypes.c_double), ("newton_maxit", ctypes.c_int32),
                ("gmres_restart", ctypes.c_int32), ("gmres_maxit", ctypes.c_int32),
                ("n_subdomains", ctypes.c_int32), ("overlap", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("jac_lag", ctypes.c_int32), ("ilu_level", ctypes.c_int32), ("threads_per_row", ctypes.c_int32),
                ("ordering", ctypes.c_int32), ("factor_mode", ctypes.c_int32),
                ("verbose", ctypes.c_int32), ("fault_test", ctypes.c_int32), ("apply_mode", ctypes.c_int32),
                ("stage_blocks", ctypes.c_int32), ("stages", ctypes.c_int32), ("orth", ctypes.c_int32),
                ("jac_chunk", ctypes.c_int32)]


class FsiSolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("rnorm0", ctypes.c_double), ("rnorm", ctypes.c_double)]


class FsiStepStats(ctypes.Structure):
    _fields_ = [("newton_iterations", ctypes.c_int32), ("linear_iterations", ctypes.c_int32),
                ("jacobian_evaluations", ctypes.c_int32), ("residual_evaluations", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("fnorm0", ctypes.c_double), ("fnorm", ctypes.c_double)] + \
               [(k, ctypes.c_double) for k in ("t_funceval", "t_jaceval", "t_pcsetup", "t_pcapply", "t_spmv",
                                                "t_orth", "t_total", "t_krylov")] + \
               [(k, ctypes.c_int32) for k in ("n_funceval", "n_jaceval", "n_pcsetup", "n_pcapply", "n_spmv",
                                               "n_orth")] + [("kernel_launches", ctypes.c_int64)]


class FsiInfo(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("n_unknowns", ctypes.c_int64),
                ("nnzb", ctypes.c_int64), ("n_fluid_tets", ctypes.c_int64), ("n_wall_tets", ctypes.c_int64),
                ("n_problems", ctypes.c_int32), ("n_subdomains", ctypes.c_int32),
                ("factor_blocks", ctypes.c_int64), ("factor_rows", ctypes.c_int64), ("max_levels", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("n_wss_faces", ctypes.c_int64), ("nd_depth", ctypes.c_int32),
                ("apply_kernel", ctypes.c_int32)]


def load_library(path=LIB_PATH):
    """Load libfsi_gb300.so and declare the signatures. Raises if it is missing."""
    if not os.path.exists(path):
        raise RuntimeError(f"solver library not built: {path} (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    sig = {
        "fsi_default_options": (None, [ctypes.POINTER(FsiOptions)]),
        "fsi_create": (ctypes.c_int, [ctypes.POINTER(FsiMesh), ctypes.POINTER(FsiMaterial), ctypes.POINTER(FsiBc),
                                      ctypes.c_int32, ctypes.POINTER(FsiOptions), P, ctypes.POINTER(P)]),
        "fsi_destroy": (ctypes.c_int, [P]),
        "fsi_set_state": (ctypes.c_int, [P, P, P, P, ctypes.c_double]),
        "fsi_get_state": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_double)]),
        "fsi_residual": (ctypes.c_int, [P, P, P]),
        "fsi_jacobian": (ctypes.c_int, [P, P]),
        "fsi_jacobian_export": (ctypes.c_int, [P, P, P, P]),
        "fsi_spmv": (ctypes.c_int, [P, P, P]),
        "fsi_pc_apply": (ctypes.c_int, [P, P, P]),
        "fsi_linear_solve": (ctypes.c_int, [P, P, P, ctypes.POINTER(FsiSolveStats)]),
        "fsi_step": (ctypes.c_int, [P, ctypes.POINTER(FsiStepStats)]),
        "fsi_get_info": (ctypes.c_int, [P, ctypes.POINTER(FsiInfo)]),
        "fsi_last_error": (ctypes.c_char_p, [P]),
        "fsi_residual_noalloc": (ctypes.c_int, [P, P, P]),
        "fsi_wss": (ctypes.c_int, [P, P, P, P]),
        "fsi_wss_faces": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class FsiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(ctx, st):
    if st != FSI_OK:
        msg = lib().fsi_last_error(ctx)
        raise FsiError(st, msg.decode() if msg else "")
    return st


def _dptr(t):
    """Data pointer of a contiguous float64 CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---------------------------------------------------------------------------
# the entry points, one by one
# ---------------------------------------------------------------------------
def fsi_default_options(**over):
    o = FsiOptions()
    lib().fsi_default_options(ctypes.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def fsi_create(mesh, material, bcs, options, stream=None):
    """mesh: vesselmesh.Mesh-like (X, tets, tet_domain, node_tag, node_problem);
    material: dict; bcs: list of dicts (center, normal, radius, peak, amp, freq,
    phase, rigid_wall); options: FsiOptions. Returns the opaque context handle."""
    X = np.ascontiguousarray(mesh.X, dtype=np.float64)
    T = np.ascontiguousarray(mesh.tets, dtype=np.int32)
    D = np.ascontiguousarray(mesh.tet_domain, dtype=np.uint8)
    G = np.ascontiguousarray(mesh.node_tag, dtype=np.uint32)
    NP = np.ascontiguousarray(mesh.node_problem, dtype=np.int32)
    m = FsiMesh(X.shape[0], T.shape[0], X.ctypes.data, T.ctypes.data, D.ctypes.data, G.ctypes.data,
                NP.ctypes.data)
    mat = FsiMaterial(**{k: float(material[k]) for k in ("rho_f", "mu_f", "rho_s", "E_s", "nu_s", "eta_s")})
    arr = (FsiBc * len(bcs))()
    for i, b in enumerate(bcs):
        arr[i].center[:] = list(map(float, b["center"]))
        arr[i].normal[:] = list(map(float, b["normal"]))
        arr[i].radius = float(b["radius"])
        arr[i].peak, arr[i].amp = float(b["peak"]), float(b["amp"])
        arr[i].freq, arr[i].phase = float(b["freq"]), float(b["phase"])
        arr[i].rigid_wall = int(b.get("rigid_wall", 0))
    ctx = ctypes.c_void_p()
    st = lib().fsi_create(ctypes.byref(m), ctypes.byref(mat), arr, len(bcs), ctypes.byref(options),
                          stream if stream is not None else _stream(), ctypes.byref(ctx))
    if st != FSI_OK:
        raise FsiError(st, "fsi_create failed")
    return ctx


def fsi_destroy(ctx):
    return lib().fsi_destroy(ctx)


def fsi_set_state(ctx, y_n, y_nm1=None, y_nm2=None, t=0.0):
    return _check(ctx, lib().fsi_set_state(ctx, _dptr(y_n), _dptr(y_nm1), _dptr(y_nm2), float(t)))


def fsi_get_state(ctx, y_n=None):
    t = ctypes.c_double()
    _check(ctx, lib().fsi_get_state(ctx, _dptr(y_n), ctypes.byref(t)))
    return t.value


def fsi_residual(ctx, y, F):
    return _check(ctx, lib().fsi_residual(ctx, _dptr(y), _dptr(F)))


def fsi_residual_noalloc(ctx, y, F):
    """Same F(y) as fsi_residual, computed without any device allocation (the
    assembly scratch is a fixed array inside the library; at most 32,768 tets)."""
    return _check(ctx, lib().fsi_residual_noalloc(ctx, _dptr(y), _dptr(F)))


def fsi_jacobian(ctx, y):
    return _check(ctx, lib().fsi_jacobian(ctx, _dptr(y)))


def fsi_jacobian_export(ctx):
    """Returns (row_ptr, col, vals[nnzb,7,7]) as numpy arrays."""
    info = fsi_get_info(ctx)
    rp = np.zeros(info.n_nodes + 1, dtype=np.int32)
    col = np.zeros(info.nnzb, dtype=np.int32)
    vals = np.zeros((info.nnzb, 7, 7), dtype=np.float64)
    _check(ctx, lib().fsi_jacobian_export(ctx, rp.ctypes.data, col.ctypes.data, vals.ctypes.data))
    return rp, col, vals


def fsi_spmv(ctx, x, y):
    return _check(ctx, lib().fsi_spmv(ctx, _dptr(x), _dptr(y)))


def fsi_pc_apply(ctx, r, z):
    return _check(ctx, lib().fsi_pc_apply(ctx, _dptr(r), _dptr(z)))


def fsi_linear_solve(ctx, rhs, x, raise_on_divergence=True):
    s = FsiSolveStats()
    st = lib().fsi_linear_solve(ctx, _dptr(rhs), _dptr(x), ctypes.byref(s))
    if st != FSI_OK and (raise_on_divergence or st != 6):
        _check(ctx, st)
    return s


def fsi_step(ctx, stats=True):
    s = FsiStepStats()
    _check(ctx, lib().fsi_step(ctx, ctypes.byref(s) if stats else None))
    return s


def fsi_wss(ctx, y, wss=None):
    """Wall shear stress: fills the device tensor wss ([n_wss_faces, 3] FP64, or
    None) and returns the per-problem SAWSS as a numpy array."""
    n = fsi_get_info(ctx).n_problems
    out = np.zeros(n, dtype=np.float64)
    _check(ctx, lib().fsi_wss(ctx, _dptr(y), _dptr(wss) if wss is not None else None, out.ctypes.data))
    return out


def fsi_wss_faces(ctx):
    """(n_faces, (n_faces, 2) int32 array of input fluid tet and opposite vertex)."""
    n = ctypes.c_int64()
    _check(ctx, lib().fsi_wss_faces(ctx, ctypes.byref(n), None))
    tf = np.zeros((n.value, 2), dtype=np.int32)
    _check(ctx, lib().fsi_wss_faces(ctx, ctypes.byref(n), tf.ctypes.data))
    return n.value, tf


def fsi_get_info(ctx):
    i = FsiInfo()
    _check(ctx, lib().fsi_get_info(ctx, ctypes.byref(i)))
    return i


def fsi_last_error(ctx):
    m = lib().fsi_last_error(ctx)
    return m.decode() if m else ""


def stats_dict(s):
    return {k: getattr(s, k) for k, _ in s._fields_}


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
DEFAULT_MATERIAL = dict(rho_f=1.05, mu_f=0.035, rho_s=1.2, E_s=3.0e6, nu_s=0.45, eta_s=0.0)


class Solver:
    """Owns one context; inputs are a mesh, a material dict and solver options."""

    def __init__(self, mesh, material=None, options=None, rigid_wall=False, **opt):
        import torch
        self.mesh = mesh
        self.material = dict(DEFAULT_MATERIAL if material is None else material)
        self.options = options if options is not None else fsi_default_options(**opt)
        bcs = [dict(b, rigid_wall=int(rigid_wall)) for b in mesh.inlets]
        self.ctx = fsi_create(mesh, self.material, bcs, self.options)
        self.N = mesh.n_nodes
        self.torch = torch

    def close(self):
        if self.ctx is not None:
            fsi_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, a=None):
        t = self.torch
        if a is None:
            return t.zeros((self.N, 7), dtype=t.float64, device="cuda")
        if isinstance(a, t.Tensor):
            return a.to(device="cuda", dtype=t.float64).reshape(self.N, 7).contiguous()
        return t.as_tensor(np.asarray(a, dtype=np.float64), device="cuda").reshape(self.N, 7).contiguous()

    def set_state(self, y_n, y_nm1=None, y_nm2=None, t=0.0):
        fsi_set_state(self.ctx, self.vec(y_n), None if y_nm1 is None else self.vec(y_nm1),
                      None if y_nm2 is None else self.vec(y_nm2), t)

    def state(self):
        y = self.vec()
        t = fsi_get_state(self.ctx, y)
        return y.cpu().numpy(), t

    def residual(self, y):
        F = self.vec()
        fsi_residual(self.ctx, self.vec(y), F)
        return F.cpu().numpy()

    def jacobian(self, y):
        fsi_jacobian(self.ctx, self.vec(y))

    def jacobian_csr(self):
        import scipy.sparse as sp
        rp, col, vals = fsi_jacobian_export(self.ctx)
        return sp.bsr_matrix((vals, col, rp), shape=(7 * self.N, 7 * self.N)).tocsr()

    def info(self):
        return fsi_get_info(self.ctx)

    def step(self):
        return fsi_step(self.ctx)

    def wss(self, y):
        """(faces (F,2), WSS vectors (F,3), SAWSS per problem) for the state y."""
        n, faces = fsi_wss_faces(self.ctx)
        w = self.torch.zeros((max(n, 1), 3), dtype=self.torch.float64, device="cuda")
        sawss = fsi_wss(self.ctx, self.vec(y), w)
        return faces, w[:n].cpu().numpy(), sawss
