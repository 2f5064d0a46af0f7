"""Thin Python binding of the MG-CCCS C ABI (include/mgcccs.h).

Argument marshalling only: every numerical step runs in the CUDA library
``_lib/libmgcccs.so``.  PyTorch supplies device memory and the stream.  There is
no CPU path: if the library is missing or no GPU is present, calls raise.

The module-level functions carry the C names (``mgcccs_setup``, ``mgcccs_vcycle``,
...); ``Solver`` bundles a handle with its workspace tensor.
"""
from __future__ import annotations

import ctypes
import math
import os
import re

import numpy as np

from . import build as _build

HEADER = os.path.join(_build.ROOT, "include", "mgcccs.h")

OK, EINVAL, ECUDA, ENOSPACE, EBREAKDOWN, ENONFINITE, ENOTCONV, EDIVERGED = 0, -1, -2, -3, -4, -5, -6, -7


class MGCCCSError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {mgcccs_strerror(code)} (code {code})")


class mgcccs_c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class mgcccs_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("R0x", ctypes.c_double), ("R0y", ctypes.c_double),
                ("theta", ctypes.c_double), ("E", ctypes.c_double),
                ("levels", ctypes.c_int), ("nu1", ctypes.c_int), ("nu2", ctypes.c_int),
                ("omega", ctypes.c_double), ("n_b", ctypes.c_int),
                ("coarse_gamma", ctypes.c_double), ("krylov_restart", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_rtol", ctypes.c_double)]


COARSE_GAMMA_DEFAULT = 14.6 * math.pi / 180.0

_LIB = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_SIGS = {
    "mgcccs_workspace_size": (ctypes.c_size_t, [ctypes.POINTER(mgcccs_params)]),
    "mgcccs_setup": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(mgcccs_params), _vp, _vp, _vp, _vp,
                          ctypes.c_size_t, _vp]),
    "mgcccs_setup_with_states": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(mgcccs_params), _vp, _vp, _vp,
                                      _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "mgcccs_vcycle": (_i, [_vp, _vp, _vp]),
    "mgcccs_cccs": (_i, [_vp, _vp, _vp]),
    "mgcccs_solve": (_i, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d), _vp]),
    "mgcccs_solve_host": (_i, [_vp, _vp, _vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d)]),
    "mgcccs_precond_apply": (_i, [_vp, _vp, _vp]),
    "mgcccs_set_solve_driver": (_i, [_vp, _i]),
    "mgcccs_set_tile_rows": (_i, [_vp, _i]),
    "mgcccs_axis_spectrum": (_i, [_vp, _i, _i, _vp]),
    "mgcccs_eig_fallbacks": (_i, [_vp]),
    "mgcccs_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp),
                                 ctypes.POINTER(_vp), _vp]),
    "mgcccs_batch_run": (_i, [_vp, _d, _i, ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "mgcccs_batch_destroy": (None, [_vp]),
    "mgcccs_batch_solve": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _d, _i,
                                ctypes.POINTER(_i), ctypes.POINTER(_d), ctypes.POINTER(_i)]),
    "mgcccs_residual": (_i, [_vp, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "mgcccs_matvec": (_i, [_vp, _vp, _vp]),
    "mgcccs_weighted_dot": (_i, [_vp, _vp, _vp, _vp, mgcccs_c128, _vp]),
    "mgcccs_weighted_product": (_i, [_vp, _vp, _vp, mgcccs_c128, _vp]),
    "mgcccs_smooth": (_i, [_vp, _i, _vp, _vp, _i]),
    "mgcccs_level_residual": (_i, [_vp, _i, _vp, _vp, _vp]),
    "mgcccs_restrict": (_i, [_vp, _i, _vp, _vp]),
    "mgcccs_prolong_add": (_i, [_vp, _i, _vp, _vp]),
    "mgcccs_coarse_solve": (_i, [_vp, _vp, _vp]),
    "mgcccs_get_bound_states": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "mgcccs_gs_dots": (_i, [_vp, _vp, ctypes.c_longlong, _i, _vp, _vp]),
    "mgcccs_gs_update": (_i, [_vp, _vp, ctypes.c_longlong, _i, _vp, _vp]),
    "mgcccs_gs_dots_c64": (_i, [_vp, _vp, ctypes.c_longlong, _i, _vp, _vp]),
    "mgcccs_gs_update_c64": (_i, [_vp, _vp, ctypes.c_longlong, _i, _vp, _vp]),
    "mgcccs_launch_count": (ctypes.c_longlong, [_vp]),
    "mgcccs_norm2_noalloc": (_i, [_vp, ctypes.c_size_t, _vp, _vp]),
    "mgcccs_fp64_probe": (_i, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "mgcccs_strerror": (ctypes.c_char_p, [_i]),
    "mgcccs_destroy": (None, [_vp]),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/mgcccs.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgcccs_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB_PATH):
            raise RuntimeError(f"MG-CCCS CUDA library missing at {_build.LIB_PATH}; "
                               "build it with paper_1412_1953_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def mgcccs_strerror(code: int) -> str:
    return lib().mgcccs_strerror(int(code)).decode()


def _check(code: int, where: str) -> int:
    if code != OK:
        raise MGCCCSError(code, where)
    return code


NOALLOC_MAX_N = 8388608


def mgcccs_norm2_noalloc(v, out, stream=None):
    """Squared 2-norm of a complex128 CUDA tensor into a float64 CUDA tensor `out`
    (one element), without any workspace (see include/mgcccs.h)."""
    import torch
    if v.dtype != torch.complex128 or not v.is_cuda or not v.is_contiguous():
        raise TypeError("v must be a contiguous complex128 CUDA tensor")
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < 1:
        raise TypeError("out must be a float64 CUDA tensor")
    if out.device != v.device:
        raise TypeError("out must be on the device of v")
    # the scratch address is looked up for the current device: make it v's
    with torch.cuda.device(v.device):
        st = stream if stream is not None else torch.cuda.current_stream(v.device)
        _check(lib().mgcccs_norm2_noalloc(v.data_ptr(), v.numel(), out.data_ptr(), st.cuda_stream),
               "mgcccs_norm2_noalloc")


PROBE_CHAINS = 8


def mgcccs_fp64_probe(blocks, iters, out, m=0.9999999, b=1e-9, stream=None):
    """Launch the FP64 throughput probe (see include/mgcccs.h) into the float64 CUDA tensor
    `out` (>= blocks elements) on `stream` (default: the current stream of out's device).
    Returns the FP64 lane operations it executes."""
    import torch
    if out.dtype != torch.float64 or not out.is_cuda or out.numel() < blocks:
        raise TypeError("out must be a float64 CUDA tensor of at least `blocks` elements")
    with torch.cuda.device(out.device):
        st = stream if stream is not None else torch.cuda.current_stream(out.device)
        _check(lib().mgcccs_fp64_probe(int(blocks), int(iters), float(m), float(b), out.data_ptr(), st.cuda_stream),
               "mgcccs_fp64_probe")
    return int(blocks) * 256 * int(iters) * PROBE_CHAINS


def make_params(nx, ny, Lx, Ly, R0x, R0y, theta, E, levels=5, nu1=1, nu2=1, omega=2.0 / 3.0, n_b=3,
                coarse_gamma=COARSE_GAMMA_DEFAULT, krylov_restart=0, precision=0,
                inner_rtol=0.0) -> mgcccs_params:
    return mgcccs_params(int(nx), int(ny), float(Lx), float(Ly), float(R0x), float(R0y), float(theta),
                         float(E), int(levels), int(nu1), int(nu2), float(omega), int(n_b), float(coarse_gamma),
                         int(krylov_restart), int(precision), float(inner_rtol))


def params_for(prob, **kw) -> mgcccs_params:
    return make_params(prob.nx, prob.ny, prob.Lx, prob.Ly, prob.R0x, prob.R0y, prob.theta, prob.E, **kw)


def mgcccs_workspace_size(p: mgcccs_params) -> int:
    return int(lib().mgcccs_workspace_size(ctypes.byref(p)))


def _ptr(t) -> int:
    return t.data_ptr()


def _dev_c128(t, n: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.complex128 or not t.is_cuda:
        raise TypeError(f"{name} must be a complex128 CUDA tensor")
    if not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name} must be contiguous with {n} elements")
    return t


# Bound states by (grid, contour, n_b, V1, V2): they do not depend on E or V12, so a
# handle for another energy on the same grid reuses them (mgcccs_setup_with_states).
_STATE_CACHE: dict = {}


def _state_key(p: mgcccs_params, v1, v2):
    import hashlib
    h = hashlib.sha1()
    for a in (v1, v2):
        arr = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
        h.update(np.ascontiguousarray(arr, dtype=np.complex128).tobytes())
    return (p.nx, p.ny, p.Lx, p.Ly, p.R0x, p.R0y, p.theta, p.n_b, h.hexdigest())


class Solver:
    """A setup handle plus its workspace.  u, f, r, z are complex128 CUDA tensors of
    shape (ny-1, nx-1) (or any contiguous shape with that many elements).  With
    reuse_states, bound states of an earlier handle on the same grid and V1, V2 are
    supplied to the setup instead of being recomputed."""

    def __init__(self, p: mgcccs_params, v1, v2, v12, stream=None, reuse_states=False):
        import torch
        self.p = p
        self.mx, self.my = p.nx - 1, p.ny - 1
        self.n = self.mx * self.my
        dev = torch.device("cuda", torch.cuda.current_device())
        as_dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.complex128).to(dev) \
            if not isinstance(a, torch.Tensor) else a.to(dev, torch.complex128).contiguous()
        v1d, v2d, v12d = as_dev(v1), as_dev(v2), as_dev(v12)
        _dev_c128(v1d, self.mx, "v1"), _dev_c128(v2d, self.my, "v2"), _dev_c128(v12d, self.n, "v12")
        nbytes = mgcccs_workspace_size(p)
        if nbytes == 0:
            raise MGCCCSError(EINVAL, "mgcccs_workspace_size")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = ctypes.c_void_p()
        key = _state_key(p, v1, v2) if (reuse_states and p.n_b > 0) else None
        cached = _STATE_CACHE.get(key) if key is not None else None
        if cached is not None:
            lam, phi, mu, vphi = cached
            _check(lib().mgcccs_setup_with_states(ctypes.byref(h), ctypes.byref(p), _ptr(v1d), _ptr(v2d),
                                                  _ptr(v12d), lam.ctypes.data, phi.data_ptr(), mu.ctypes.data,
                                                  vphi.data_ptr(), self._ws_ptr, nbytes, self.stream.cuda_stream),
                   "mgcccs_setup_with_states")
        else:
            _check(lib().mgcccs_setup(ctypes.byref(h), ctypes.byref(p), _ptr(v1d), _ptr(v2d), _ptr(v12d),
                                      self._ws_ptr, nbytes, self.stream.cuda_stream), "mgcccs_setup")
        self.h = h
        if key is not None and cached is None:
            _STATE_CACHE[key] = self.bound_states()

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            lib().mgcccs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _f(self, t, name="array", n=None):
        return _ptr(_dev_c128(t, self.n if n is None else n, name))

    # -- hot path
    def vcycle(self, u, f):
        _check(lib().mgcccs_vcycle(self.h, self._f(u, "u"), self._f(f, "f")), "mgcccs_vcycle")

    def cccs(self, u, f):
        _check(lib().mgcccs_cccs(self.h, self._f(u, "u"), self._f(f, "f")), "mgcccs_cccs")

    def precond_apply(self, z, r):
        _check(lib().mgcccs_precond_apply(self.h, self._f(z, "z"), self._f(r, "r")), "mgcccs_precond_apply")

    def solve(self, u, f, rtol=1e-10, max_iter=1000, history=False, raise_on_notconv=True):
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        hist = np.zeros(max_iter) if history else None
        code = lib().mgcccs_solve(self.h, self._f(u, "u"), self._f(f, "f"), float(rtol), int(max_iter),
                                  ctypes.byref(it), ctypes.byref(rr),
                                  hist.ctypes.data if hist is not None else None)
        if code != OK and not (code == ENOTCONV and not raise_on_notconv):
            raise MGCCCSError(code, "mgcccs_solve")
        out = (it.value, rr.value)
        if history:
            out = out + (hist[: it.value].copy(),)
        return out

    def solve_host(self, u: np.ndarray, f: np.ndarray, rtol=1e-10, max_iter=1000):
        """End-to-end call with host arrays (complex128, C-contiguous); u is updated in place."""
        if u.dtype != np.complex128 or f.dtype != np.complex128 or not u.flags.c_contiguous \
                or not f.flags.c_contiguous or u.size != self.n or f.size != self.n:
            raise ValueError("u and f must be C-contiguous complex128 arrays of the grid size")
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        _check(lib().mgcccs_solve_host(self.h, u.ctypes.data, f.ctypes.data, float(rtol), int(max_iter),
                                       ctypes.byref(it), ctypes.byref(rr)), "mgcccs_solve_host")
        return it.value, rr.value

    def residual(self, u, f, r, norm=False):
        n2 = ctypes.c_double(0.0)
        _check(lib().mgcccs_residual(self.h, self._f(u, "u"), self._f(f, "f"), self._f(r, "r"),
                                     ctypes.byref(n2) if norm else None), "mgcccs_residual")
        return n2.value if norm else None

    def matvec(self, x, y):
        _check(lib().mgcccs_matvec(self.h, self._f(x, "x"), self._f(y, "y")), "mgcccs_matvec")

    def weighted_dot(self, a, b, out, d=None, scale=1.0):
        """out[0] = scale * sum_k w_k a_k b_k (d_k); out is a complex128 CUDA tensor."""
        sc = mgcccs_c128(complex(scale).real, complex(scale).imag)
        _check(lib().mgcccs_weighted_dot(self.h, self._f(a, "a"), self._f(b, "b"),
                                         self._f(d, "d") if d is not None else None, sc,
                                         _ptr(_dev_c128(out, out.numel(), "out"))), "mgcccs_weighted_dot")

    def weighted_product(self, a, b, out, scale=1.0):
        sc = mgcccs_c128(complex(scale).real, complex(scale).imag)
        _check(lib().mgcccs_weighted_product(self.h, self._f(a, "a"), self._f(b, "b"), sc, self._f(out, "out")),
               "mgcccs_weighted_product")

    # -- Gram-Schmidt halves of an Arnoldi step (fine-level vectors)
    def _basis(self, V, k, dtype=None):
        import torch
        dtype = dtype or torch.complex128
        if not isinstance(V, torch.Tensor) or V.dtype != dtype or not V.is_cuda:
            raise TypeError(f"V must be a {dtype} CUDA tensor")
        if V.dim() != 2 or V.shape[0] < k or V.shape[1] < self.n or V.stride(1) != 1:
            raise ValueError(f"V must be a (>= {k}, >= {self.n}) {dtype} tensor with unit column stride")
        return V.data_ptr(), V.stride(0)

    def _c64(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64 or not t.is_cuda:
            raise TypeError(f"{name} must be a complex64 CUDA tensor")
        if not t.is_contiguous() or t.numel() != self.n:
            raise ValueError(f"{name} must be contiguous with {self.n} elements")
        return t.data_ptr()

    def gs_dots(self, V, k, w, out):
        """out[i] = sum_p conj(V[i, p]) w[p] for i < k (out: k-element complex128 CUDA tensor)."""
        vp, ld = self._basis(V, k)
        _check(lib().mgcccs_gs_dots(self.h, vp, ld, int(k), self._f(w, "w"), _ptr(_dev_c128(out, k, "out"))),
               "mgcccs_gs_dots")

    def gs_update(self, V, k, coef, w):
        """w -= sum_{i<k} coef[i] V[i] (coef: k-element complex128 CUDA tensor)."""
        vp, ld = self._basis(V, k)
        _check(lib().mgcccs_gs_update(self.h, vp, ld, int(k), _ptr(_dev_c128(coef, k, "coef")), self._f(w, "w")),
               "mgcccs_gs_update")

    def gs_dots_c64(self, V, k, w, out):
        """The complex64 multi-dot of the mixed form: V, w complex64, out k-element complex128."""
        import torch
        vp, ld = self._basis(V, k, torch.complex64)
        _check(lib().mgcccs_gs_dots_c64(self.h, vp, ld, int(k), self._c64(w, "w"), _ptr(_dev_c128(out, k, "out"))),
               "mgcccs_gs_dots_c64")

    def gs_update_c64(self, V, k, coef, w):
        """The complex64 update of the mixed form: V, w complex64, coef k-element complex128."""
        import torch
        vp, ld = self._basis(V, k, torch.complex64)
        _check(lib().mgcccs_gs_update_c64(self.h, vp, ld, int(k), _ptr(_dev_c128(coef, k, "coef")),
                                          self._c64(w, "w")), "mgcccs_gs_update_c64")

    # -- single steps
    def level_size(self, level: int) -> int:
        return ((self.p.nx >> level) - 1) * ((self.p.ny >> level) - 1)

    def smooth(self, level, u, f, sweeps=1):
        n = self.level_size(level)
        _check(lib().mgcccs_smooth(self.h, level, self._f(u, "u", n), self._f(f, "f", n), sweeps), "mgcccs_smooth")

    def level_residual(self, level, u, f, r):
        n = self.level_size(level)
        _check(lib().mgcccs_level_residual(self.h, level, self._f(u, "u", n), self._f(f, "f", n),
                                           self._f(r, "r", n)), "mgcccs_level_residual")

    def restrict(self, level, r, rc):
        _check(lib().mgcccs_restrict(self.h, level, self._f(r, "r", self.level_size(level)),
                                     self._f(rc, "rc", self.level_size(level + 1))), "mgcccs_restrict")

    def prolong_add(self, level, ec, u):
        _check(lib().mgcccs_prolong_add(self.h, level, self._f(ec, "ec", self.level_size(level + 1)),
                                        self._f(u, "u", self.level_size(level))), "mgcccs_prolong_add")

    def coarse_solve(self, f, u):
        n = self.level_size(self.p.levels - 1)
        _check(lib().mgcccs_coarse_solve(self.h, self._f(f, "f", n), self._f(u, "u", n)), "mgcccs_coarse_solve")

    def bound_states(self):
        import torch
        nb = self.p.n_b
        lam = np.zeros(nb, dtype=np.complex128)
        mu = np.zeros(nb, dtype=np.complex128)
        dev = self.workspace.device
        phi = torch.empty((nb, self.mx), dtype=torch.complex128, device=dev)
        vphi = torch.empty((nb, self.my), dtype=torch.complex128, device=dev)
        _check(lib().mgcccs_get_bound_states(self.h, lam.ctypes.data, phi.data_ptr(), mu.ctypes.data,
                                             vphi.data_ptr()), "mgcccs_get_bound_states")
        return lam, phi, mu, vphi

    def axis_spectrum(self, axis: int = 0, method: int = 0) -> np.ndarray:
        """All eigenvalues of the fine-grid H1 of one axis (0: x, 1: y); method 0 is the
        Ehrlich-Aberth iteration setup uses, 1 the FP64 QR."""
        n = self.mx if axis == 0 else self.my
        out = np.zeros(n, dtype=np.complex128)
        _check(lib().mgcccs_axis_spectrum(self.h, int(axis), int(method), out.ctypes.data), "mgcccs_axis_spectrum")
        return out

    def eig_fallbacks(self) -> int:
        return int(lib().mgcccs_eig_fallbacks(self.h))

    def set_tile_rows(self, rows: int):
        """Block height of the passes on the levels too small to fill the GPU (2, 4, 8; 0 =
        default); results do not depend on it."""
        _check(lib().mgcccs_set_tile_rows(self.h, int(rows)), "mgcccs_set_tile_rows")

    def launch_count(self) -> int:
        return int(lib().mgcccs_launch_count(self.h))


def mgcccs_batch_solve(solvers, us, fs, rtol=1e-10, max_iter=1000):
    """Solve the problems of several Solver handles together (see include/mgcccs.h).
    Returns (iterations, relres, status) lists; raises only on argument errors."""
    K = len(solvers)
    hs = (_vp * K)(*[s.h.value for s in solvers])
    up = (_vp * K)(*[s._f(u, "u") for s, u in zip(solvers, us)])
    fp = (_vp * K)(*[s._f(f, "f") for s, f in zip(solvers, fs)])
    its = (_i * K)()
    rr = (_d * K)()
    st = (_i * K)()
    code = lib().mgcccs_batch_solve(hs, K, up, fp, float(rtol), int(max_iter), its, rr, st)
    if code not in (OK, ENOTCONV, ENONFINITE, EDIVERGED):
        raise MGCCCSError(code, "mgcccs_batch_solve")
    return list(its), list(rr), list(st)


DRIVER_GRAPH, DRIVER_HOST = 0, 1


def mgcccs_set_solve_driver(solver, driver: int):
    _check(lib().mgcccs_set_solve_driver(solver.h, int(driver)), "mgcccs_set_solve_driver")


class Batch:
    """mgcccs_batch_create / _run / _destroy: the device-driven solves of several Solver
    handles as one CUDA graph, launched once per run()."""

    def __init__(self, solvers, us, fs, stream=None):
        import torch
        self.solvers, self.us, self.fs = list(solvers), list(us), list(fs)
        K = len(self.solvers)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        hs = (_vp * K)(*[s.h.value for s in self.solvers])
        up = (_vp * K)(*[s._f(u, "u") for s, u in zip(self.solvers, self.us)])
        fp = (_vp * K)(*[s._f(f, "f") for s, f in zip(self.solvers, self.fs)])
        b = _vp()
        _check(lib().mgcccs_batch_create(ctypes.byref(b), hs, K, up, fp, self.stream.cuda_stream),
               "mgcccs_batch_create")
        self.b = b

    def run(self, rtol=1e-10, max_iter=1000):
        K = len(self.solvers)
        its, rr, st = (_i * K)(), (_d * K)(), (_i * K)()
        code = lib().mgcccs_batch_run(self.b, float(rtol), int(max_iter), its, rr, st)
        if code not in (OK, ENOTCONV, ENONFINITE, EDIVERGED):
            raise MGCCCSError(code, "mgcccs_batch_run")
        return list(its), list(rr), list(st)

    def close(self):
        if getattr(self, "b", None):
            lib().mgcccs_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
