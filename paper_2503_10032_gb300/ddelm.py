"""Thin ctypes binding of libddelm (include/ddelm.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device memory (the workspace and the
input/output tensors) and the stream.  If the shared library is missing the
import of this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libddelm.so")

DDELM_OK = 0
DDELM_ERR_INVALID_ARG = -1
DDELM_ERR_RANK_DEFICIENT = -2
DDELM_ERR_NOT_CONVERGED = -3
DDELM_ERR_CUDA = -4
DDELM_ERR_TIMEOUT = -5
DDELM_ERR_UNSUPPORTED = -6
DDELM_OP_POISSON = 0
DDELM_OP_DIFFUSION = 1
DDELM_OP_BIHARMONIC = 2
DDELM_PREC_FP64 = 0
DDELM_PREC_MIXED = 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class ddelm_options(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("eps_rel", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("use_change_of_vars", ctypes.c_int),
                ("precision", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("keep_matrices", ctypes.c_int), ("setup_wave", ctypes.c_int),
                ("setup_scheme", ctypes.c_int), ("setup_passes", ctypes.c_int),
                ("disable_graphs", ctypes.c_int), ("barrier_timeout_ms", ctypes.c_int),
                ("inject_barrier_stall", ctypes.c_int), ("plain_flux_corners", ctypes.c_int),
                ("vanilla", ctypes.c_int), ("autotune", ctypes.c_int), ("trim_levels", ctypes.c_int),
                ("trim_mask", ctypes.c_int), ("chol_blocked", ctypes.c_int), ("tc_tiles", ctypes.c_int)]


class ddelm_problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("op", ctypes.c_int), ("n_rhs", ctypes.c_int),
                ("M", _ip), ("w_hat", _dp), ("b_hat", _dp), ("scale", ctypes.c_double),
                ("n_int", _ip), ("x_int", _dp), ("a_int", _dp), ("grad_a_int", _dp),
                ("edge_pts", _ip), ("n_eval", _ip), ("x_eval", _dp),
                ("opt", ddelm_options)]


class ddelm_sizes(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int), ("n_edges", ctypes.c_int), ("n_bnd", ctypes.c_int),
                ("n_pi", ctypes.c_int), ("n_delta", ctypes.c_int),
                ("sum_M", ctypes.c_longlong), ("sum_int", ctypes.c_longlong),
                ("sum_eval", ctypes.c_longlong), ("workspace_bytes", ctypes.c_size_t),
                ("upload_bytes", ctypes.c_size_t)]


class ddelm_solve_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("ms_total", ctypes.c_double)]


EXPORTS = ("ddelm_query", "ddelm_setup", "ddelm_refactor", "ddelm_solve", "ddelm_backward",
           "ddelm_interface_residual", "ddelm_interface_solve",
           "ddelm_inspect", "ddelm_profile", "ddelm_local_lstsq_static", "ddelm_destroy",
           "ddelm_status_string", "ddelm_last_error")
DDELM_STATIC_SCRATCH_DOUBLES = 1048576
DDELM_SCHEME_AUTO, DDELM_SCHEME_FP64CQR3, DDELM_SCHEME_FP32, DDELM_SCHEME_CQR2_SERIES = 0, 1, 2, 3
DDELM_SCHEME_CQR2_SERIES_DW = 4
DDELM_PROF_CLASSES = 8
PROF_CLASS_NAMES = ("features", "gemm_f64", "chol_inv", "cg_persistent", "other", "slicing", "tc_gemm")


def load_library(path: str = LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(f"libddelm.so not built ({path}); run paper_2503_10032_gb300.build.build()")
    lib = ctypes.CDLL(path)
    lib.ddelm_query.argtypes = [ctypes.POINTER(ddelm_problem), ctypes.POINTER(ddelm_sizes)]
    lib.ddelm_query.restype = ctypes.c_int
    lib.ddelm_setup.argtypes = [ctypes.POINTER(ddelm_problem), ctypes.c_void_p, ctypes.c_size_t,
                                ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), _ip]
    lib.ddelm_setup.restype = ctypes.c_int
    lib.ddelm_refactor.argtypes = [ctypes.c_void_p, ctypes.c_void_p, _ip]
    lib.ddelm_refactor.restype = ctypes.c_int
    lib.ddelm_profile.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp,
                                  ctypes.POINTER(ctypes.c_longlong)]
    lib.ddelm_profile.restype = ctypes.c_int
    lib.ddelm_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ddelm_solve_info),
                                ctypes.c_void_p]
    lib.ddelm_solve.restype = ctypes.c_int
    lib.ddelm_backward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, _dp, ctypes.POINTER(ddelm_solve_info), ctypes.c_void_p]
    lib.ddelm_backward.restype = ctypes.c_int
    lib.ddelm_interface_residual.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 6 + [ctypes.c_void_p]
    lib.ddelm_interface_residual.restype = ctypes.c_int
    lib.ddelm_interface_solve.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ddelm_solve_info), ctypes.c_void_p]
    lib.ddelm_interface_solve.restype = ctypes.c_int
    lib.ddelm_inspect.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_size_t]
    lib.ddelm_inspect.restype = ctypes.c_int
    lib.ddelm_local_lstsq_static.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    lib.ddelm_local_lstsq_static.restype = ctypes.c_int
    lib.ddelm_destroy.argtypes = [ctypes.c_void_p]
    lib.ddelm_destroy.restype = None
    lib.ddelm_status_string.argtypes = [ctypes.c_int]
    lib.ddelm_status_string.restype = ctypes.c_char_p
    lib.ddelm_last_error.argtypes = []
    lib.ddelm_last_error.restype = ctypes.c_char_p
    return lib


_lib = load_library()


class DDELMError(RuntimeError):
    def __init__(self, status, what=""):
        msg = f"{what}: {ddelm_status_string(status)} ({status})"
        last = _lib.ddelm_last_error().decode()
        if status == DDELM_ERR_CUDA or (status == DDELM_ERR_INVALID_ARG and last.startswith("problem rejected")):
            msg += f": {last}"
        super().__init__(msg)
        self.status = status


def ddelm_status_string(status: int) -> str:
    return _lib.ddelm_status_string(status).decode()


def make_options(theta=0.999, eps_rel=1e-8, tol=1e-8, max_iters=5000, use_change_of_vars=True,
                 precision=DDELM_PREC_FP64, max_refine=8, keep_matrices=False, setup_wave=0,
                 setup_scheme=DDELM_SCHEME_AUTO, setup_passes=0, graphs=True, barrier_timeout_ms=0,
                 inject_barrier_stall=False, use_Am=True, use_coarse=True, autotune=True, trim_levels=0,
                 trim_mask=0, chol_blocked=False, tc_tiles=0):
    return ddelm_options(theta, eps_rel, tol, max_iters, int(use_change_of_vars), precision,
                         max_refine, int(keep_matrices), int(setup_wave), int(setup_scheme),
                         int(setup_passes), int(not graphs), int(barrier_timeout_ms),
                         int(inject_barrier_stall), int(not use_Am), int(not use_coarse), int(autotune),
                         int(trim_levels), int(trim_mask), int(chol_blocked), int(tc_tiles))


class ProblemArgs:
    """Keeps the numpy arrays of a problem alive while a ddelm_problem points at them."""

    def __init__(self, prob, opts: ddelm_options):
        def d(a):
            return np.ascontiguousarray(a, dtype=np.float64)

        def i(a):
            return np.ascontiguousarray(a, dtype=np.int32)
        self.M, self.n_int, self.edge_pts, self.n_eval = i(prob.M), i(prob.n_int), i(prob.edge_pts), i(prob.n_eval)
        self.w_hat, self.b_hat, self.x_int = d(prob.w_hat), d(prob.b_hat), d(prob.x_int)
        self.a_int, self.grad_a_int, self.x_eval = d(prob.a_int), d(prob.grad_a_int), d(prob.x_eval)
        c = ddelm_problem()
        c.nx, c.ny = prob.nx, prob.ny
        c.x0, c.x1, c.y0, c.y1 = prob.box
        c.op = prob.op
        c.n_rhs = prob.n_rhs
        c.M = self.M.ctypes.data_as(_ip)
        c.w_hat = self.w_hat.ctypes.data_as(_dp)
        c.b_hat = self.b_hat.ctypes.data_as(_dp)
        c.scale = prob.scale
        c.n_int = self.n_int.ctypes.data_as(_ip)
        c.x_int = self.x_int.ctypes.data_as(_dp)
        c.a_int = self.a_int.ctypes.data_as(_dp) if prob.op == DDELM_OP_DIFFUSION else None
        c.grad_a_int = self.grad_a_int.ctypes.data_as(_dp) if prob.op == DDELM_OP_DIFFUSION else None
        c.edge_pts = self.edge_pts.ctypes.data_as(_ip)
        c.n_eval = self.n_eval.ctypes.data_as(_ip)
        c.x_eval = self.x_eval.ctypes.data_as(_dp)
        c.opt = opts
        self.c = c


def ddelm_query(pa: ProblemArgs) -> ddelm_sizes:
    sz = ddelm_sizes()
    rc = _lib.ddelm_query(ctypes.byref(pa.c), ctypes.byref(sz))
    if rc != DDELM_OK:
        raise DDELMError(rc, "ddelm_query")
    return sz


def ddelm_setup(pa: ProblemArgs, ws_ptr: int, ws_bytes: int, stream: int):
    h = ctypes.c_void_p()
    info = ctypes.c_int(-1)
    rc = _lib.ddelm_setup(ctypes.byref(pa.c), ctypes.c_void_p(ws_ptr), ws_bytes, ctypes.c_void_p(stream),
                          ctypes.byref(h), ctypes.byref(info))
    return rc, h, info.value


def ddelm_refactor(h, stream):
    info = ctypes.c_int(-1)
    rc = _lib.ddelm_refactor(h, ctypes.c_void_p(stream), ctypes.byref(info))
    return rc, info.value


def ddelm_profile(h, enable: bool, reset: bool):
    ms = np.zeros(DDELM_PROF_CLASSES, np.float64)
    n = np.zeros(DDELM_PROF_CLASSES, np.int64)
    rc = _lib.ddelm_profile(h, int(enable), int(reset), ms.ctypes.data_as(_dp),
                            n.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    if rc != DDELM_OK:
        raise DDELMError(rc, "ddelm_profile")
    return ms, n


def ddelm_solve(h, f_ptr, g_ptr, c_ptr, mu_ptr, u_ptr, stream):
    info = ddelm_solve_info()
    rc = _lib.ddelm_solve(h, ctypes.c_void_p(f_ptr), ctypes.c_void_p(g_ptr), ctypes.c_void_p(c_ptr),
                          ctypes.c_void_p(mu_ptr), ctypes.c_void_p(u_ptr), ctypes.byref(info),
                          ctypes.c_void_p(stream))
    return rc, info


def ddelm_backward(h, grad_c_ptr, grad_u_ptr, grad_f_ptr, grad_g_ptr, stream, want_scale=False):
    """(status, info, dL/ds or None)."""
    info = ddelm_solve_info()
    gs = ctypes.c_double(0.0)
    rc = _lib.ddelm_backward(h, ctypes.c_void_p(grad_c_ptr), ctypes.c_void_p(grad_u_ptr),
                             ctypes.c_void_p(grad_f_ptr), ctypes.c_void_p(grad_g_ptr),
                             ctypes.byref(gs) if want_scale else None, ctypes.byref(info),
                             ctypes.c_void_p(stream))
    return rc, info, (gs.value if want_scale else None)


def ddelm_interface_residual(h, f_ptr, g_ptr, mu_ptr, r_ptr, c_ptr, u_ptr, stream):
    return _lib.ddelm_interface_residual(h, *(ctypes.c_void_p(x) for x in (f_ptr, g_ptr, mu_ptr, r_ptr, c_ptr,
                                                                          u_ptr)), ctypes.c_void_p(stream))


def ddelm_interface_solve(h, b_ptr, mu_ptr, stream):
    info = ddelm_solve_info()
    rc = _lib.ddelm_interface_solve(h, ctypes.c_void_p(b_ptr), ctypes.c_void_p(mu_ptr), ctypes.byref(info),
                                    ctypes.c_void_p(stream))
    return rc, info


def ddelm_inspect(h, sub: int, which: int, n: int) -> np.ndarray:
    out = np.zeros(max(n, 1), np.float64)
    rc = _lib.ddelm_inspect(h, sub, which, out.ctypes.data_as(_dp), out.size)
    if rc != DDELM_OK:
        raise DDELMError(rc, "ddelm_inspect")
    return out[:n]


def ddelm_local_lstsq_static(k_ptr, m, M, f_ptr, R, eps_rel, c_ptr, stream):
    """C = K^+ F for one local system with scratch in a static device array (no allocation)."""
    return _lib.ddelm_local_lstsq_static(ctypes.c_void_p(k_ptr), m, M, ctypes.c_void_p(f_ptr), R, eps_rel,
                                         ctypes.c_void_p(c_ptr), ctypes.c_void_p(stream))


def ddelm_destroy(h):
    _lib.ddelm_destroy(h)


class Solver:
    """A DDELM-NN handle with its torch-allocated workspace on one CUDA device."""

    def __init__(self, prob, *, device="cuda:0", stream=None, **opt_kw):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.prob = prob
        self.opt_kw = dict(opt_kw)
        self.opts = make_options(**opt_kw)
        self.pa = ProblemArgs(prob, self.opts)
        self.sizes = ddelm_query(self.pa)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = int(self.sizes.workspace_bytes)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) // 256 * 256
        rc, h, sub = ddelm_setup(self.pa, self.ws_ptr, nbytes, self.stream.cuda_stream)
        if rc != DDELM_OK:
            if h.value:
                ddelm_destroy(h)
            raise DDELMError(rc, f"ddelm_setup (subdomain {sub})")
        self.h = h

    def refactor(self):
        rc, sub = ddelm_refactor(self.h, self.stream.cuda_stream)
        if rc != DDELM_OK:
            raise DDELMError(rc, f"ddelm_refactor (subdomain {sub})")

    def profile(self, enable=True, reset=True):
        return ddelm_profile(self.h, enable, reset)

    def solve(self, f_int, g_bnd):
        """f_int [sum n_int, R], g_bnd [n_bnd, R] float64 CUDA tensors -> (c, mu, u_eval, info)."""
        torch = self.torch
        R = self.prob.n_rhs
        sz = self.sizes
        c = torch.empty((sz.sum_M, R), dtype=torch.float64, device=self.device)
        mu = torch.empty((sz.n_pi + sz.n_delta, R), dtype=torch.float64, device=self.device)
        u = torch.empty((max(sz.sum_eval, 1), R), dtype=torch.float64, device=self.device)
        f_int = f_int.contiguous()
        g_bnd = g_bnd.contiguous()
        rc, info = ddelm_solve(self.h, f_int.data_ptr(), g_bnd.data_ptr(), c.data_ptr(), mu.data_ptr(),
                               u.data_ptr(), self.stream.cuda_stream)
        if rc not in (DDELM_OK, DDELM_ERR_NOT_CONVERGED):
            raise DDELMError(rc, "ddelm_solve")
        return c, mu, u[:sz.sum_eval], info, rc

    def interface_residual(self, f_int, g_bnd, mu_delta):
        """(r = b_theta - S_theta mu_Delta, c, u_eval) at a given mu_Delta [n_delta, R]."""
        torch = self.torch
        R = self.prob.n_rhs
        sz = self.sizes
        r = torch.empty((max(sz.n_delta, 1), R), dtype=torch.float64, device=self.device)
        c = torch.empty((sz.sum_M, R), dtype=torch.float64, device=self.device)
        u = torch.empty((max(sz.sum_eval, 1), R), dtype=torch.float64, device=self.device)
        mu = mu_delta.contiguous()
        rc = ddelm_interface_residual(self.h, f_int.contiguous().data_ptr(), g_bnd.contiguous().data_ptr(),
                                      mu.data_ptr(), r.data_ptr(), c.data_ptr(), u.data_ptr(),
                                      self.stream.cuda_stream)
        if rc != DDELM_OK:
            raise DDELMError(rc, "ddelm_interface_residual")
        return r[:sz.n_delta], c, u[:sz.sum_eval]

    def interface_solve(self, b):
        """mu_Delta with S_theta mu_Delta = b (b: [n_delta, R] device tensor)."""
        torch = self.torch
        mu = torch.empty((max(self.sizes.n_delta, 1), self.prob.n_rhs), dtype=torch.float64, device=self.device)
        rc, info = ddelm_interface_solve(self.h, b.contiguous().data_ptr(), mu.data_ptr(), self.stream.cuda_stream)
        if rc not in (DDELM_OK, DDELM_ERR_NOT_CONVERGED):
            raise DDELMError(rc, "ddelm_interface_solve")
        return mu[:self.sizes.n_delta], info

    def backward(self, grad_c=None, grad_u=None, scale=False):
        """(dL/df [sum n_int, R], dL/dg [n_bnd, R], info) for cotangents of c and/or u;
        with scale=True also dL/ds for the hidden-layer scale at the last solve
        (a float, the fourth element)."""
        torch = self.torch
        R = self.prob.n_rhs
        sz = self.sizes
        gf = torch.empty((max(sz.sum_int, 1), R), dtype=torch.float64, device=self.device)
        gg = torch.empty((max(sz.n_bnd, 1), R), dtype=torch.float64, device=self.device)
        gc = grad_c.contiguous() if grad_c is not None else None
        gu = grad_u.contiguous() if grad_u is not None else None
        rc, info, gs = ddelm_backward(self.h, gc.data_ptr() if gc is not None else 0,
                                      gu.data_ptr() if gu is not None else 0, gf.data_ptr(), gg.data_ptr(),
                                      self.stream.cuda_stream, want_scale=scale)
        if rc not in (DDELM_OK, DDELM_ERR_NOT_CONVERGED):
            raise DDELMError(rc, "ddelm_backward")
        if scale:
            return gf[:sz.sum_int], gg[:sz.n_bnd], info, gs
        return gf[:sz.sum_int], gg[:sz.n_bnd], info

    def inspect(self, sub, which):
        sizes = ddelm_inspect(self.h, sub, 7, 4)
        m, M, nG, nDl = (int(v) for v in sizes)
        shapes = {0: (m, M), 1: (m, M), 2: (nG, M), 3: (nG, nG), 4: (nG, nG), 5: (nDl, nDl),
                  6: (self.sizes.n_pi, self.sizes.n_pi), 10: (M, M)}
        shp = shapes[which]
        return ddelm_inspect(self.h, sub, which, shp[0] * shp[1]).reshape(shp)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            ddelm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
