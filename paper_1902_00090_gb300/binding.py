"""Thin ctypes binding of libddgmres.so (include/ddgmres.h): argument marshalling only.

Every function keeps the name of the C entry point it calls.  Device memory
comes from torch CUDA tensors (complex128 / complex64 are interleaved re/im,
which is the library's layout); all arithmetic runs in the library's kernels.
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

from . import _build

_LIB = None

DDG_C128 = 0
DDG_C64_REFINE = 1
DDG_C64_ONLY = 2
PRECISIONS = {"c128": DDG_C128, "c64": DDG_C64_REFINE, "c64_refine": DDG_C64_REFINE, "c64_only": DDG_C64_ONLY}

KERNEL_CLASSES = ("step", "dots", "update", "residual", "cycle_end", "setup")

STATUS = {0: "DDG_OK", 1: "DDG_EINVAL", 2: "DDG_ENOMEM", 3: "DDG_ECUDA", 4: "DDG_ENOCONV",
          5: "DDG_EBREAKDOWN", 6: "DDG_ETIMEOUT", 7: "DDG_ESINGULAR"}


class DdgError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {message}")
        self.status = status


class ddg_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("dx", C.c_double), ("wavelength", C.c_double),
                ("npml_x", C.c_int), ("npml_y", C.c_int), ("pml_order", C.c_double),
                ("pml_R", C.c_double)]


class ddg_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("cycles", C.c_int), ("converged", C.c_int),
                ("fallback_used", C.c_int), ("breakdown", C.c_int),
                ("true_rel_residual", C.c_double), ("first_step_rel_residual", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_vp = C.c_void_p
_SIGS = {
    "ddg_status_str": (C.c_char_p, [C.c_int]),
    "ddg_last_error": (C.c_char_p, []),
    "ddg_version": (C.c_int, []),
    "ddg_context_create": (C.c_int, [C.POINTER(_vp)]),
    "ddg_context_destroy": (C.c_int, [_vp]),
    "ddg_context_workspace_bytes": (C.c_longlong, [_vp]),
    "ddg_context_set_inner_tol": (C.c_int, [_vp, C.c_double]),
    "ddg_context_launches": (C.c_longlong, [_vp]),
    "ddg_context_set_orthogonalization": (C.c_int, [_vp, C.c_int]),
    "ddg_context_set_fallback": (C.c_int, [_vp, C.c_double]),
    "ddg_context_set_graphs": (C.c_int, [_vp, C.c_int]),
    "ddg_context_set_basis_storage": (C.c_int, [_vp, C.c_int]),
    "ddg_context_set_preconditioner": (C.c_int, [_vp, C.c_int]),
    "ddg_context_set_augmented_cycles": (C.c_int, [_vp, C.c_int]),
    "ddg_context_set_wait_limit": (C.c_int, [_vp, C.c_longlong]),
    "ddg_context_set_augmented_policy": (C.c_int, [_vp, C.c_double, C.c_int, C.c_int]),
    "ddg_context_set_workspace_limit": (C.c_int, [_vp, C.c_longlong]),
    "ddg_context_profile_enable": (C.c_int, [_vp, C.c_int]),
    "ddg_context_profile_read": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                          C.POINTER(C.c_longlong)]),
    "fdfd_operator": (C.c_int, [C.POINTER(ddg_grid), _vp, C.POINTER(_vp), _vp]),
    "fdfd_operator_destroy": (C.c_int, [_vp]),
    "fdfd_operator_size": (C.c_longlong, [_vp]),
    "fdfd_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "fdfd_apply_c64": (C.c_int, [_vp, _vp, _vp, _vp]),
    "fdfd_source": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, _vp, _vp]),
    "gmres_solve": (C.c_int, [_vp, _vp, _vp, _vp, C.c_double, C.c_int, C.c_int, C.c_int,
                              C.POINTER(ddg_info), _vp]),
    "augmented_gmres_solve": (C.c_int, [_vp, _vp, _vp, _vp, C.c_int, _vp, C.c_double, C.c_int,
                                        C.c_int, C.c_int, C.POINTER(ddg_info), _vp]),
    "gmres_solve_batched": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                      C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(ddg_info),
                                      _vp]),
    "predictor_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(_vp)]),
    "predictor_destroy": (C.c_int, [_vp]),
    "predictor_num_params": (C.c_longlong, [_vp]),
    "predictor_launches": (C.c_longlong, [_vp]),
    "predictor_set_tensor_cores": (C.c_int, [_vp, C.c_int]),
    "predictor_create_with_field": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(_vp)]),
    "predictor_set_input_field": (C.c_int, [_vp, _vp, C.c_int, C.c_int, _vp]),
    "predictor_set_output_base": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_double, _vp]),
    "predictor_set_output_base_wavelength": (C.c_int, [_vp, _vp, C.c_int, C.c_int, C.c_double, C.c_double, _vp]),
    "predictor_set_params": (C.c_int, [_vp, _vp, C.c_longlong]),
    "predictor_get_params": (C.c_int, [_vp, _vp, C.c_longlong]),
    "predictor_forward": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_double, C.c_double, _vp, _vp]),
    "subspace_predict": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_double, C.c_double,
                                   C.POINTER(_vp), _vp]),
    "predictor_loss_grad": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_double, C.c_double,
                                      C.POINTER(_vp), C.POINTER(C.c_double), _vp, _vp]),
    "predictor_adam_step": (C.c_int, [_vp, C.c_float, _vp]),
    "predictor_set_loss": (C.c_int, [_vp, C.c_int]),
    "predictor_train_step": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.c_int, C.c_double, C.c_double,
                                       C.POINTER(_vp), C.c_float, C.POINTER(C.c_double), _vp]),
    "predictor_save": (C.c_int, [_vp, C.c_char_p]),
    "predictor_load": (C.c_int, [_vp, C.c_char_p]),
    "gmres_solve_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_double, C.c_int, C.c_int, C.c_int,
                                      C.POINTER(ddg_info), _vp]),
    "predictor_num_outputs": (C.c_int, [_vp]),
    "gmres_solve_queue_trajectories": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int, C.c_int, C.c_int, C.c_int,
                                                 C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.c_int,
                                                 C.POINTER(_vp), C.c_double, C.c_int, C.c_int, C.c_int,
                                                 C.POINTER(ddg_info)]),
    "gmres_solve_trajectories": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                           C.c_int, C.POINTER(_vp), C.c_double, C.c_int, C.c_int, C.c_int,
                                           C.POINTER(ddg_info), _vp]),
    "fdfd_solve_host": (C.c_int, [_vp, _vp, C.c_int, C.POINTER(ddg_grid), C.POINTER(_vp), C.c_int, C.c_double,
                                  C.c_double, C.POINTER(_vp), C.c_int, C.c_double, C.c_int, C.c_int, C.c_int,
                                  C.POINTER(_vp), C.POINTER(ddg_info), _vp]),
    "pca_fit": (C.c_int, [_vp, _vp, C.c_longlong, C.c_int, C.c_int, _vp, C.POINTER(C.c_double), _vp]),
    "augmented_gmres_solve_batched": (C.c_int, [_vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp),
                                                C.POINTER(_vp), C.c_int, C.POINTER(_vp),
                                                C.c_double, C.c_int, C.c_int, C.c_int,
                                                C.POINTER(ddg_info), _vp]),
    "gmres_solve_queue": (C.c_int, [C.POINTER(_vp), C.POINTER(_vp), C.c_int, C.c_int, C.c_int,
                                    C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.c_int,
                                    C.POINTER(_vp), C.c_double, C.c_int, C.c_int, C.c_int,
                                    C.POINTER(ddg_info)]),
}


def lib_path() -> str:
    return _build.LIB


def load():
    """Loads libddgmres.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"{_build.LIB} is missing: run __graft_entry__.build() first")
        lib = C.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            if hasattr(lib, name):
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int, where: str):
    if status != 0:
        raise DdgError(status, where, load().ddg_last_error().decode())


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("ddgmres needs a CUDA device; none is available")
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _dev_ptr(t, dtype, what, numel=None):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{what}: need a contiguous CUDA tensor of {dtype}, got {t.dtype} "
                         f"on {t.device} (contiguous={t.is_contiguous()})")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{what}: expected {numel} elements, got {t.numel()}")
    return _vp(t.data_ptr())


class Context:
    """ddg_context: device workspace and tuning for one stream."""

    def __init__(self, inner_tol: float | None = None, orthogonalization: str | None = None):
        _torch()
        h = _vp()
        _check(load().ddg_context_create(C.byref(h)), "ddg_context_create")
        self._h = h
        if inner_tol is not None:
            self.set_inner_tol(inner_tol)
        if orthogonalization is not None:
            self.set_orthogonalization(orthogonalization)

    @property
    def handle(self):
        return self._h

    def set_inner_tol(self, eta: float):
        _check(load().ddg_context_set_inner_tol(self._h, float(eta)), "ddg_context_set_inner_tol")

    def set_orthogonalization(self, scheme: str):
        """'cgs2' (classical Gram-Schmidt twice) or 'dcgs2' (delayed reorthogonalisation)."""
        code = {"cgs2": 0, "dcgs2": 1}[scheme]
        _check(load().ddg_context_set_orthogonalization(self._h, code), "ddg_context_set_orthogonalization")

    def set_augmented_cycles(self, cycles: int):
        """Restart cycles of an augmented solve that keep V (later cycles: plain GMRES)."""
        _check(load().ddg_context_set_augmented_cycles(self._h, int(cycles)), "ddg_context_set_augmented_cycles")

    def set_graphs(self, on: bool):
        """Run a batched solve's restart cycles as one CUDA graph launch (default) or host-driven."""
        _check(load().ddg_context_set_graphs(self._h, int(bool(on))), "ddg_context_set_graphs")

    def set_basis_storage(self, storage: str):
        """Krylov basis of complex64 solves stored in 'f32' (default) or 'f16' (IEEE half)."""
        code = {"f32": 0, "f16": 1}[storage]
        _check(load().ddg_context_set_basis_storage(self._h, code), "ddg_context_set_basis_storage")

    def set_preconditioner(self, kind: str):
        """'none' (default) or 'jacobi' (right preconditioner M = diag(A), the data-free baseline)."""
        code = {"none": 0, "jacobi": 1}[kind]
        _check(load().ddg_context_set_preconditioner(self._h, code), "ddg_context_set_preconditioner")

    def set_augmented_policy(self, cycles: int, keep: int = 0, wavelength: float = 0.0):
        """Cycles that use all of V, then the leading `keep` columns (0: plain);
        for every solve (wavelength 0) or the solves at one wavelength [m]."""
        _check(load().ddg_context_set_augmented_policy(self._h, float(wavelength), int(cycles), int(keep)),
               "ddg_context_set_augmented_policy")

    def set_wait_limit(self, ns: int):
        """Limit (ns) of the solver's bounded device waits; DDG_ETIMEOUT when one runs out."""
        _check(load().ddg_context_set_wait_limit(self._h, int(ns)), "ddg_context_set_wait_limit")

    def set_workspace_limit(self, nbytes: int):
        """Largest device workspace this context may allocate (0: no limit); DDG_ENOMEM above it."""
        _check(load().ddg_context_set_workspace_limit(self._h, int(nbytes)), "ddg_context_set_workspace_limit")

    def set_fallback(self, threshold: float):
        """V-only relative residual above which an augmented solve continues as plain GMRES."""
        _check(load().ddg_context_set_fallback(self._h, float(threshold)), "ddg_context_set_fallback")

    @property
    def workspace_bytes(self) -> int:
        return int(load().ddg_context_workspace_bytes(self._h))

    @property
    def launches(self) -> int:
        """Kernels launched through this context (ddg_context_launches)."""
        return int(load().ddg_context_launches(self._h))

    def profile_enable(self, on: bool = True):
        _check(load().ddg_context_profile_enable(self._h, int(bool(on))), "ddg_context_profile_enable")

    def profile_read(self):
        """{class name: (ms, algorithmic bytes, launches)} since profiling was enabled."""
        out = {}
        for cls, name in enumerate(KERNEL_CLASSES):
            ms, by, n = C.c_double(), C.c_double(), C.c_longlong()
            _check(load().ddg_context_profile_read(self._h, cls, C.byref(ms), C.byref(by), C.byref(n)),
                   "ddg_context_profile_read")
            out[name] = (ms.value, by.value, n.value)
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().ddg_context_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ddg_context_create(inner_tol: float | None = None) -> Context:
    return Context(inner_tol)


class Operator:
    """ddg_op: A(eps, omega) of one FDFD problem (keeps its own copy of eps)."""

    def __init__(self, handle, nx, ny):
        self._h, self.nx, self.ny = handle, nx, ny
        self.D = nx * ny

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            load().fdfd_operator_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_grid(grid) -> ddg_grid:
    """ddg_grid from an inputs.Grid (or any object/dict with the same fields)."""
    get = (lambda k: grid[k]) if isinstance(grid, dict) else (lambda k: getattr(grid, k))
    def opt(k, d):
        try:
            return get(k)
        except (KeyError, AttributeError):
            return d
    npml = opt("npml", 0)
    return ddg_grid(int(get("nx")), int(get("ny")), float(get("dx")), float(get("wavelength")),
                    int(opt("npml_x", npml)), int(opt("npml_y", npml)), float(opt("pml_order", 3.0)),
                    float(opt("pml_R", 1e-8)))


def fdfd_operator(grid, eps, stream=None) -> Operator:
    """eps: CUDA float64 tensor (ny, nx)."""
    torch = _torch()
    g = make_grid(grid)
    p = _dev_ptr(eps, torch.float64, "eps", g.nx * g.ny)
    h = _vp()
    _check(load().fdfd_operator(C.byref(g), p, C.byref(h), _stream(stream)), "fdfd_operator")
    return Operator(h, g.nx, g.ny)


def fdfd_apply(A: Operator, x, y=None, stream=None):
    torch = _torch()
    if y is None:
        y = torch.empty_like(x)
    _check(load().fdfd_apply(A.handle, _dev_ptr(x, torch.complex128, "x", A.D),
                             _dev_ptr(y, torch.complex128, "y", A.D), _stream(stream)), "fdfd_apply")
    return y


def fdfd_apply_c64(A: Operator, x, y=None, stream=None):
    torch = _torch()
    if y is None:
        y = torch.empty_like(x)
    _check(load().fdfd_apply_c64(A.handle, _dev_ptr(x, torch.complex64, "x", A.D),
                                 _dev_ptr(y, torch.complex64, "y", A.D), _stream(stream)),
           "fdfd_apply_c64")
    return y


def fdfd_source(A: Operator, i_src: int, sigma_cells: float, j_c: float, b=None, stream=None):
    torch = _torch()
    if b is None:
        b = torch.empty(A.D, dtype=torch.complex128, device="cuda")
    _check(load().fdfd_source(A.handle, int(i_src), float(sigma_cells), float(j_c),
                              _dev_ptr(b, torch.complex128, "b", A.D), _stream(stream)), "fdfd_source")
    return b


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def gmres_solve(ctx: Context, A: Operator, b, x=None, tol=1e-6, restart=200, maxit=5000,
                precision="c128", stream=None, check=False):
    """Returns (x, info dict, status).  x (in/out) holds x0 on entry."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(b)
    info = ddg_info()
    st = load().gmres_solve(ctx.handle, A.handle, _dev_ptr(b, torch.complex128, "b", A.D),
                            _dev_ptr(x, torch.complex128, "x", A.D), float(tol), int(restart),
                            int(maxit), _prec(precision), C.byref(info), _stream(stream))
    if st not in (0, 4) or (check and st != 0):
        _check(st, "gmres_solve")
    return x, info.as_dict(), st


def augmented_gmres_solve(ctx: Context, A: Operator, b, U, x=None, tol=1e-6, restart=200,
                          maxit=5000, precision="c128", stream=None, check=False):
    """U: CUDA complex128 tensor (k, D): row n is the predicted vector v_{n+1}
    (the library's D x k column-major layout)."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(b)
    k = U.shape[0]
    info = ddg_info()
    st = load().augmented_gmres_solve(ctx.handle, A.handle, _dev_ptr(b, torch.complex128, "b", A.D),
                                      _dev_ptr(U, torch.complex128, "U", k * A.D), int(k),
                                      _dev_ptr(x, torch.complex128, "x", A.D), float(tol), int(restart),
                                      int(maxit), _prec(precision), C.byref(info), _stream(stream))
    if st not in (0, 4) or (check and st != 0):
        _check(st, "augmented_gmres_solve")
    return x, info.as_dict(), st


def _ptr_array(ts, dtype, what, sizes):
    arr = (_vp * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _dev_ptr(t, dtype, f"{what}[{i}]", sizes[i]).value
    return arr


def gmres_solve_batched(ctx: Context, A, b, x=None, tol=1e-6, restart=200, maxit=5000,
                        precision="c128", stream=None):
    """A, b, x: lists (one entry per solve).  Returns (x list, info list, status)."""
    torch = _torch()
    n = len(A)
    if x is None:
        x = [torch.zeros_like(bb) for bb in b]
    sizes = [a.D for a in A]
    ha = (_vp * n)(*[a.handle.value for a in A])
    infos = (ddg_info * n)()
    st = load().gmres_solve_batched(ctx.handle, n, ha, _ptr_array(b, torch.complex128, "b", sizes),
                                    _ptr_array(x, torch.complex128, "x", sizes), float(tol),
                                    int(restart), int(maxit), _prec(precision), infos,
                                    _stream(stream))
    if st not in (0, 4):
        _check(st, "gmres_solve_batched")
    return x, [i.as_dict() for i in infos], st


def augmented_gmres_solve_batched(ctx: Context, A, b, U, x=None, tol=1e-6, restart=200,
                                  maxit=5000, precision="c128", stream=None):
    """U: list of CUDA complex128 tensors (k, D), same k for every solve."""
    torch = _torch()
    n = len(A)
    if x is None:
        x = [torch.zeros_like(bb) for bb in b]
    k = U[0].shape[0]
    sizes = [a.D for a in A]
    ha = (_vp * n)(*[a.handle.value for a in A])
    infos = (ddg_info * n)()
    st = load().augmented_gmres_solve_batched(
        ctx.handle, n, ha, _ptr_array(b, torch.complex128, "b", sizes),
        _ptr_array(U, torch.complex128, "U", [k * s for s in sizes]), int(k),
        _ptr_array(x, torch.complex128, "x", sizes), float(tol), int(restart), int(maxit),
        _prec(precision), infos, _stream(stream))
    if st not in (0, 4):
        _check(st, "augmented_gmres_solve_batched")
    return x, [i.as_dict() for i in infos], st


def gmres_solve_trajectories(ctx: Context, A, b, U=None, x=None, tol=1e-6, restart=200, maxit=5000,
                             precision="c64", stream=None):
    """A, b (and U, x): lists of n_traj lists of n_steps entries (one trajectory
    per inner list); U entries (k, D) complex128 or U None.  Returns (x, info,
    status) in the same nesting."""
    torch = _torch()
    n_traj, n_steps = len(A), len(A[0])
    if any(len(a) != n_steps for a in A):
        raise ValueError("every trajectory needs the same number of steps")
    fa = [a for tr in A for a in tr]
    fb = [v for tr in b for v in tr]
    if x is None:
        x = [[torch.zeros_like(v) for v in tr] for tr in b]
    fx = [v for tr in x for v in tr]
    sizes = [a.D for a in fa]
    k = 0
    hu = None
    if U is not None:
        fu = [u for tr in U for u in tr]
        k = fu[0].shape[0]
        hu = _ptr_array(fu, torch.complex128, "U", [k * s for s in sizes])
    n = len(fa)
    infos = (ddg_info * n)()
    st = load().gmres_solve_trajectories(ctx.handle, n_traj, n_steps, (_vp * n)(*[a.handle.value for a in fa]),
                                         _ptr_array(fb, torch.complex128, "b", sizes), hu, int(k),
                                         _ptr_array(fx, torch.complex128, "x", sizes), float(tol), int(restart),
                                         int(maxit), _prec(precision), infos, _stream(stream))
    if st not in (0, 4):
        _check(st, "gmres_solve_trajectories")
    inf = [i.as_dict() for i in infos]
    return x, [inf[r * n_steps:(r + 1) * n_steps] for r in range(n_traj)], st


def gmres_solve_queue_trajectories(lanes, A, b, U=None, x=None, traj_per_group=16, streams=None, tol=1e-6,
                                   restart=200, maxit=5000, precision="c64"):
    """The solve queue over trajectories with recycling: A, b (and U, x) are
    lists of n_traj lists of n_steps entries; groups of traj_per_group
    trajectories run gmres_solve_trajectories on len(lanes) concurrent lanes.
    Returns (x, info, status) nested as A."""
    torch = _torch()
    n_traj, n_steps = len(A), len(A[0])
    if any(len(a) != n_steps for a in A):
        raise ValueError("every trajectory needs the same number of steps")
    nl = len(lanes)
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(nl)]
    cur = torch.cuda.current_stream()
    for st_ in streams:
        st_.wait_stream(cur)
    fa = [a for tr in A for a in tr]
    fb = [v for tr in b for v in tr]
    if x is None:
        x = [[torch.zeros_like(v) for v in tr] for tr in b]
    fx = [v for tr in x for v in tr]
    sizes = [a.D for a in fa]
    k, hu = 0, None
    if U is not None:
        fu = [u for tr in U for u in tr]
        k = fu[0].shape[0]
        hu = _ptr_array(fu, torch.complex128, "U", [k * s_ for s_ in sizes])
    n = len(fa)
    infos = (ddg_info * n)()
    st = load().gmres_solve_queue_trajectories(
        (_vp * nl)(*[c.handle.value for c in lanes]), (_vp * nl)(*[s_.cuda_stream for s_ in streams]), nl,
        int(traj_per_group), n_traj, n_steps, (_vp * n)(*[a.handle.value for a in fa]),
        _ptr_array(fb, torch.complex128, "b", sizes), hu, int(k), _ptr_array(fx, torch.complex128, "x", sizes),
        float(tol), int(restart), int(maxit), _prec(precision), infos)
    for st_ in streams:
        cur.wait_stream(st_)
    if st not in (0, 4):
        _check(st, "gmres_solve_queue_trajectories")
    inf = [i.as_dict() for i in infos]
    return x, [inf[r * n_steps:(r + 1) * n_steps] for r in range(n_traj)], st


def gmres_solve_queue(lanes, A, b, U=None, x=None, width=64, streams=None, tol=1e-6, restart=200,
                      maxit=5000, precision="c64"):
    """A queue of independent solves (A, b, x, U: lists, one entry per solve; U
    entries (k, D) or U None for plain GMRES) run as groups of `width` batched
    solves on len(lanes) concurrent lanes (distinct Contexts; one CUDA stream
    per lane, made here when `streams` is None).  Returns (x list, info list,
    status).  The call returns once every solve has finished."""
    torch = _torch()
    n = len(A)
    nl = len(lanes)
    if x is None:
        x = [torch.zeros_like(bb) for bb in b]
    if streams is None:
        streams = [torch.cuda.Stream() for _ in range(nl)]
    if len(streams) != nl:
        raise ValueError(f"{len(streams)} streams for {nl} lanes")
    # the lanes' streams start after the work queued so far on the current stream
    cur = torch.cuda.current_stream()
    for s in streams:
        s.wait_stream(cur)
    sizes = [a.D for a in A]
    ha = (_vp * n)(*[a.handle.value for a in A])
    hl = (_vp * nl)(*[c.handle.value for c in lanes])
    hs = (_vp * nl)(*[s.cuda_stream for s in streams])
    k = 0
    hu = None
    if U is not None:
        k = U[0].shape[0]
        hu = _ptr_array(U, torch.complex128, "U", [k * sz for sz in sizes])
    infos = (ddg_info * n)()
    st = load().gmres_solve_queue(hl, hs, nl, int(width), n, ha, _ptr_array(b, torch.complex128, "b", sizes),
                                  hu, int(k), _ptr_array(x, torch.complex128, "x", sizes), float(tol),
                                  int(restart), int(maxit), _prec(precision), infos)
    for s in streams:
        cur.wait_stream(s)
    if st not in (0, 4):
        _check(st, "gmres_solve_queue")
    return x, [i.as_dict() for i in infos], st


def pca_fit(ctx: Context, F, k: int, U=None, stream=None):
    """F: CUDA complex128 tensor (M, D) -- row m is training field f_m (the library's
    D x M column-major layout).  Returns (U as a (k, D) tensor, sigma list)."""
    torch = _torch()
    M, D = F.shape
    if U is None:
        U = torch.empty((k, D), dtype=torch.complex128, device=F.device)
    sig = (C.c_double * k)()
    _check(load().pca_fit(ctx.handle, _dev_ptr(F, torch.complex128, "F", M * D), int(D), int(M), int(k),
                          _dev_ptr(U, torch.complex128, "U", k * D), sig, _stream(stream)), "pca_fit")
    return U, list(sig)


def gmres_solve_noalloc(A: Operator, b, x=None, tol=1e-6, restart=200, maxit=5000, precision="c128",
                        stream=None):
    """gmres_solve without device allocation (library-owned static scratch).
    Returns (x, info dict, status); raises on errors other than DDG_ENOCONV."""
    torch = _torch()
    if x is None:
        x = torch.zeros_like(b)
    info = ddg_info()
    st = load().gmres_solve_noalloc(A.handle, _dev_ptr(b, torch.complex128, "b", A.D),
                                    _dev_ptr(x, torch.complex128, "x", A.D), float(tol), int(restart),
                                    int(maxit), _prec(precision), C.byref(info), _stream(stream))
    if st not in (0, 4):
        _check(st, "gmres_solve_noalloc")
    return x, info.as_dict(), st


def fdfd_solve_host(ctx: Context, grids, eps_host, src, x_host, P=None, U_fixed=None, tol=1e-6, restart=200,
                    maxit=5000, precision="c64", stream=None):
    """fdfd_solve_host: grids (one per problem), eps_host (host float64 arrays or
    CPU tensors of ny*nx values, ideally pinned), src = (i_src, sigma, j_c),
    x_host (host complex128 arrays or CPU tensors of D values, written);
    U_fixed: None or one CUDA complex128 (k_fixed, D) tensor per problem,
    placed before the predictor's vectors.  Returns (info list, status)."""
    n = len(grids)
    hg = (ddg_grid * n)(*[make_grid(g) for g in grids])

    def hptr(a, what, itemsize, count):
        if hasattr(a, "data_ptr"):
            if a.is_cuda or not a.is_contiguous() or a.element_size() * a.numel() != itemsize * count:
                raise ValueError(f"{what}: need a contiguous host tensor of {count} values")
            return a.data_ptr()
        if not a.flags["C_CONTIGUOUS"] or a.nbytes != itemsize * count:
            raise ValueError(f"{what}: need a contiguous host array of {count} values")
        return a.ctypes.data

    he = (_vp * n)(*[hptr(e, f"eps[{i}]", 8, g.nx * g.ny) for i, (e, g) in enumerate(zip(eps_host, hg))])
    hx = (_vp * n)(*[hptr(x, f"x[{i}]", 16, g.nx * g.ny) for i, (x, g) in enumerate(zip(x_host, hg))])
    i_src, sigma, j_c = src
    hu, kf = None, 0
    if U_fixed is not None:
        import torch
        kf = int(U_fixed[0].shape[0])
        hu = _ptr_array(U_fixed, torch.complex128, "U_fixed", [kf * g.nx * g.ny for g in hg])
    infos = (ddg_info * n)()
    st = load().fdfd_solve_host(ctx.handle, P.handle if P is not None else None, n, hg, he, int(i_src),
                                float(sigma), float(j_c), hu, kf, float(tol), int(restart), int(maxit),
                                _prec(precision), hx, infos, _stream(stream))
    if st not in (0, 4):
        _check(st, "fdfd_solve_host")
    return [i.as_dict() for i in infos], st


def predictor_layer_shapes(channels, k, cin=4):
    """(name, Cout, Cin, kernel) per layer in the library's parameter order."""
    L = len(channels)
    out = []
    for l in range(L):
        out.append((f"enc{l}a", channels[l], cin if l == 0 else channels[l - 1], 3))
        out.append((f"enc{l}b", channels[l], channels[l], 3))
    for l in range(L - 2, -1, -1):
        out.append((f"dec{l}a", channels[l], channels[l + 1] + channels[l], 3))
        out.append((f"dec{l}b", channels[l], channels[l], 3))
    out.append(("head", 2 * k, channels[0], 1))
    return out


class Predictor:
    """ddg_predictor: the subspace-predicting CNN (weights on the device)."""

    def __init__(self, k=8, channels=(32, 48, 64, 96, 128, 128), input_field=False):
        _torch()
        self.k, self.channels = int(k), tuple(int(c) for c in channels)
        self.cin = 6 if input_field else 4
        arr = (C.c_int * len(self.channels))(*self.channels)
        h = _vp()
        if input_field:
            _check(load().predictor_create_with_field(self.k, len(self.channels), arr, C.byref(h)),
                   "predictor_create_with_field")
        else:
            _check(load().predictor_create(self.k, len(self.channels), arr, C.byref(h)), "predictor_create")
        self._h = h
        self.nparams = int(load().predictor_num_params(h))

    def set_output_base(self, U, nx, ny, scale=1.0, wavelength=None, stream=None):
        """predictor_set_output_base (every wavelength of the grid) or, with a
        wavelength in metres, predictor_set_output_base_wavelength: U a (k, D)
        complex128 CUDA tensor, or None to remove every offset."""
        torch = _torch()
        ptr = _vp()
        if U is not None:
            U = U.to(torch.complex128).contiguous()
            ptr = _vp(U.data_ptr())
        if wavelength is None or U is None:
            _check(load().predictor_set_output_base(self._h, ptr, int(nx), int(ny), float(scale), _stream(stream)),
                   "predictor_set_output_base")
        else:
            _check(load().predictor_set_output_base_wavelength(self._h, ptr, int(nx), int(ny), float(wavelength),
                                                               float(scale), _stream(stream)),
                   "predictor_set_output_base_wavelength")
        if U is not None:
            # the copy into the predictor is stream-ordered: keep U alive until it ran
            self._bases = getattr(self, "_bases", []) + [U]
        else:
            self._bases = []

    def zero_head(self):
        """Sets the 1x1 head's weights and biases to zero (the output is then the output base)."""
        import numpy as np
        theta = self.get_params()
        off = 0
        for name, co, ci, kk in self.layer_shapes():
            n = co * ci * kk * kk + co
            if name == "head":
                theta[off:off + n] = 0.0
            off += n
        self.set_params(theta)

    def set_input_field(self, f, nx, ny, stream=None):
        """predictor_set_input_field: f a complex128 CUDA tensor of ny*nx values."""
        torch = _torch()
        f = f.reshape(-1).to(torch.complex128).contiguous()
        self._field = f
        _check(load().predictor_set_input_field(self._h, _vp(f.data_ptr()), int(nx), int(ny), _stream(stream)),
               "predictor_set_input_field")

    @property
    def handle(self):
        return self._h

    def layer_shapes(self):
        return predictor_layer_shapes(self.channels, self.k, self.cin)

    @property
    def launches(self) -> int:
        """Kernels launched by this predictor (predictor_launches)."""
        return int(load().predictor_launches(self._h))

    def set_tensor_cores(self, on: bool, backward: bool = False, tma: bool = True):
        """Forward 3x3 convolutions on tcgen05 tensor cores (default) or CUDA
        cores; with backward, the backward-data convolutions too; with tma (and
        on), forward ones with a plain input read their tiles by TMA."""
        _check(load().predictor_set_tensor_cores(
            self._h, (1 if on else 0) | (2 if backward else 0) | (4 if (tma and on) else 0)),
               "predictor_set_tensor_cores")

    def set_params(self, theta):
        import numpy as np
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check(load().predictor_set_params(self._h, _vp(a.ctypes.data), a.size), "predictor_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.nparams, dtype=np.float32)
        _check(load().predictor_get_params(self._h, _vp(a.ctypes.data), a.size), "predictor_get_params")
        return a

    def init_he(self, seed=0):
        """He-normal weights (std sqrt(2 / fan_in)), zero biases, drawn from `seed`."""
        import numpy as np
        from . import inputs
        parts = []
        for i, (name, co, ci, kk) in enumerate(self.layer_shapes()):
            w = inputs.standard_normal(co * ci * kk * kk, seed * 1000 + i) * np.sqrt(2.0 / (ci * kk * kk))
            parts += [w, np.zeros(co)]
        self.set_params(np.concatenate(parts))

    def _ops(self, A):
        return (_vp * len(A))(*[a.handle.value for a in A])

    def forward(self, A, src, stream=None):
        torch = _torch()
        i_src, sigma, j_c = src
        y = torch.empty((len(A), A[0].ny, A[0].nx, 2 * self.k), dtype=torch.float32, device="cuda")
        _check(load().predictor_forward(self._h, len(A), self._ops(A), int(i_src), float(sigma), float(j_c),
                                        _vp(y.data_ptr()), _stream(stream)), "predictor_forward")
        return y

    def predict(self, A, src, U=None, stream=None):
        """subspace_predict: list of (k, D) complex128 tensors (D x k column-major)."""
        torch = _torch()
        i_src, sigma, j_c = src
        if U is None:
            U = [torch.empty((self.k, a.D), dtype=torch.complex128, device="cuda") for a in A]
        arr = _ptr_array(U, torch.complex128, "U", [self.k * a.D for a in A])
        _check(load().subspace_predict(self._h, len(A), self._ops(A), int(i_src), float(sigma), float(j_c),
                                       arr, _stream(stream)), "subspace_predict")
        return U

    def loss_grad(self, A, src, fields, want_grad=True, stream=None):
        torch = _torch()
        i_src, sigma, j_c = src
        loss = C.c_double()
        g = torch.empty(self.nparams, dtype=torch.float32, device="cuda") if want_grad else None
        arr = _ptr_array(fields, torch.complex128, "f", [a.D for a in A])
        _check(load().predictor_loss_grad(self._h, len(A), self._ops(A), int(i_src), float(sigma), float(j_c),
                                          arr, C.byref(loss), _vp(g.data_ptr()) if g is not None else None,
                                          _stream(stream)), "predictor_loss_grad")
        return loss.value, g

    def set_loss(self, kind: str):
        """'projection' (Eq. 5; train with solved fields) or 'residual' (Eq. 6; train with b)."""
        _check(load().predictor_set_loss(self._h, {"projection": 0, "residual": 1}[kind]), "predictor_set_loss")

    def adam_step(self, lr, stream=None):
        _check(load().predictor_adam_step(self._h, float(lr), _stream(stream)), "predictor_adam_step")

    def train_step(self, A, src, fields, lr, stream=None):
        torch = _torch()
        i_src, sigma, j_c = src
        loss = C.c_double()
        arr = _ptr_array(fields, torch.complex128, "f", [a.D for a in A])
        _check(load().predictor_train_step(self._h, len(A), self._ops(A), int(i_src), float(sigma), float(j_c),
                                           arr, float(lr), C.byref(loss), _stream(stream)), "predictor_train_step")
        return loss.value

    def save(self, path):
        _check(load().predictor_save(self._h, str(path).encode()), "predictor_save")

    def load_file(self, path):
        _check(load().predictor_load(self._h, str(path).encode()), "predictor_load")

    def close(self):
        if getattr(self, "_h", None):
            load().predictor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def predictor_create(k=8, channels=(32, 48, 64, 96, 128, 128)) -> Predictor:
    return Predictor(k, channels)
