"""The C-ABI library builds, loads and exports every entry point of include/*.h (no GPU needed)."""
import ctypes
import glob
import os
import re

import pytest

from paper_1902_00090_gb300 import _build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             txt, flags=re.M):
            names.add(m.group(1))
    names.discard("if")
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return ctypes.CDLL(_build.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fdfd_operator", "fdfd_apply", "gmres_solve", "augmented_gmres_solve",
                     "gmres_solve_batched", "augmented_gmres_solve_batched"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol_and_status_strings(lib):
    for n in declared_functions():
        assert n in binding._SIGS, n
    L = binding.load()
    assert L.ddg_version() >= 100
    assert L.ddg_status_str(0) == b"ok"
    assert L.ddg_status_str(4).startswith(b"not converged")


def test_host_side_argument_checks_need_no_gpu(lib):
    # NULL handles are rejected on the host before any CUDA call.
    L = binding.load()
    assert L.fdfd_apply(None, None, None, None) == 1
    assert L.gmres_solve(None, None, None, None, 1e-6, 10, 10, 0, None, None) == 1
    assert b"NULL" in L.ddg_last_error()
    g = binding.ddg_grid(2, 2, 1e-8, 1.55e-6, 0, 0, 3.0, 1e-8)
    h = ctypes.c_void_p()
    assert L.fdfd_operator(ctypes.byref(g), ctypes.c_void_p(16), ctypes.byref(h), None) == 1
    # grids of 2^31 cells or more are refused before any allocation (the
    # kernels find a cell's row and column by 32-bit division)
    g = binding.ddg_grid(65536, 32768, 1e-8, 1.55e-6, 0, 0, 3.0, 1e-8)
    assert L.fdfd_operator(ctypes.byref(g), ctypes.c_void_p(16), ctypes.byref(h), None) == 1
    assert b"2^31" in L.ddg_last_error()


def test_context_setters_reject_null_and_bad_kinds(lib):
    # the context options added for the data-free baseline and the basis storage
    L = binding.load()
    assert L.ddg_context_set_preconditioner(None, 1) == 1
    assert b"ddg_context_set_preconditioner" in L.ddg_last_error()
    assert L.ddg_context_set_basis_storage(None, 1) == 1
    assert L.ddg_context_set_graphs(None, 1) == 1
    with pytest.raises(KeyError):
        binding.Context.set_preconditioner(object.__new__(binding.Context), "ilu")


def test_queue_rejects_bad_lanes_before_any_cuda_call(lib):
    L = binding.load()
    assert L.gmres_solve_queue(None, None, 1, 8, 1, None, None, None, 0, None, 1e-6, 10, 10, 1, None) == 1
    assert b"gmres_solve_queue" in L.ddg_last_error()
    two = (ctypes.c_void_p * 2)(16, 16)   # the same context twice
    A = (ctypes.c_void_p * 1)(16)
    assert L.gmres_solve_queue(two, None, 2, 8, 1, A, A, None, 0, A, 1e-6, 10, 10, 1, None) == 1
    assert b"share a context" in L.ddg_last_error()
    assert L.gmres_solve_queue(two, None, 9, 8, 1, A, A, None, 0, A, 1e-6, 10, 10, 1, None) == 1
