"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every function declared in include/grf.h, and rejects bad arguments
with status codes before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1105_2737_gb300 import build
    build()
    from paper_1105_2737_gb300 import _lib
    return _lib


def declared_functions():
    src = open(os.path.join(ROOT, "include", "grf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(grf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["grf_plan_create", "grf_sample", "grf_backward", "grf_rfft_forward", "grf_batch_plan_create",
                 "grf_batch_sample", "grf_status_word", "grf_plan_destroy", "grf_status_string"]:
        assert want in names


def test_library_exports_every_declared_symbol(L):
    lib = L.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(L):
    lib = L.lib()
    for s in range(7):
        assert lib.grf_status_string(s)
    assert lib.grf_status_string(99) == b"unknown status"


def _create(L, d, n, Ls, spec=None, alg=2, prec=0, max_batch=1):
    h = C.c_void_p()
    nn = (C.c_int64 * max(d, 1))(*n) if n is not None else None
    LL = (C.c_double * max(d, 1))(*Ls) if Ls is not None else None
    sp = spec if spec is not None else L.make_spectrum()
    return L.lib().grf_plan_create(C.byref(h), d, nn, LL, C.byref(sp), alg, prec, max_batch), h


@pytest.mark.parametrize("d,n,Ls,status", [
    (0, [4], [1.0], 1),            # bad dimension
    (4, [4, 4, 4, 4], [1.0] * 4, 1),
    (2, [5, 4], [1.0, 1.0], 1),    # odd N
    (2, [4, 0], [1.0, 1.0], 1),
    (2, [4, 4], [1.0, -1.0], 1),   # non-positive L
    (2, [22, 4], [1.0, 1.0], 2),   # even, with a prime factor above 7
    (2, [8192, 4], [1.0, 1.0], 2), # axis 1 above 4096
    (1, [2 ** 23], [1.0], 2),
])
def test_invalid_geometry(L, d, n, Ls, status):
    st, h = _create(L, d, n, Ls)
    assert st == status
    assert not h.value


@pytest.mark.parametrize("n", [[22, 4], [4, 26], [2 * 3 * 11]])
def test_fp64_rejects_prime_factors_above_7(L, n):
    st, h = _create(L, len(n), n, [1.0] * len(n), prec=1)
    assert st == 2 and not h.value


def test_invalid_parameters(L):
    for kw in [dict(sigma=0.0), dict(ell=-1.0), dict(nu=0.0), dict(family=7)]:
        st, _ = _create(L, 2, [8, 8], [1.0, 1.0], spec=L.make_spectrum(**kw))
        assert st == 1, kw
    st, _ = _create(L, 2, [8, 8], [1.0, 1.0], alg=3)
    assert st == 1
    st, _ = _create(L, 2, [8, 8], [1.0, 1.0], prec=5)
    assert st == 1
    st, _ = _create(L, 2, [8, 8], [1.0, 1.0], max_batch=0)
    assert st == 1
    assert L.lib().grf_plan_create(None, 2, None, None, None, 2, 0, 1) == 1
    assert L.lib().grf_sample(None, 0, 1, None, None) == 1
    assert L.lib().grf_cov_origin(None, 0, 1, None, None) == 1
    assert L.lib().grf_plan_destroy(None) == 0
    assert L.lib().grf_plan_query(None, 0) == -1


def test_no_device_is_reported_not_crashed(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    st, h = _create(L, 2, [8, 8], [1.0, 1.0])
    assert st in (3, 4)  # CUDA error, reported as a status
    assert L.lib().grf_last_error()


def _create_bc(L, d, n, Ls, bc=1, spec=None, max_batch=1):
    h = C.c_void_p()
    nn = (C.c_int64 * max(d, 1))(*n) if n is not None else None
    LL = (C.c_double * max(d, 1))(*Ls) if Ls is not None else None
    sp = spec if spec is not None else L.make_spectrum()
    return L.lib().grf_bc_plan_create(C.byref(h), d, nn, LL, C.byref(sp), bc, max_batch), h


@pytest.mark.parametrize("d,n,Ls,bc,status", [
    (0, [4], [1.0], 1, 1),
    (2, [4, 1], [1.0, 1.0], 1, 1),      # fewer than 2 intervals
    (2, [4, 4], [1.0, 0.0], 2, 1),      # non-positive L
    (2, [4, 4], [1.0, 1.0], 3, 1),      # unknown boundary condition
    (2, [6, 4], [1.0, 1.0], 1, 2),      # not a power of two
    (1, [8192], [1.0], 2, 2),           # above 4096 intervals
])
def test_boundary_plan_rejects_bad_arguments(L, d, n, Ls, bc, status):
    st, h = _create_bc(L, d, n, Ls, bc=bc)
    assert st == status
    assert not h.value


def test_boundary_plan_rejects_discrete_normalisation(L):
    st, h = _create_bc(L, 2, [8, 8], [1.0, 1.0], spec=L.make_spectrum(normalize_discrete=1))
    assert st == 2 and not h.value
    assert L.lib().grf_bc_plan_create(None, 1, None, None, None, 1, 1) == 1


def test_alu_peak_rejects_bad_arguments(L):
    v = C.c_double()
    assert L.lib().grf_alu_peak(3, C.byref(v), None) == 1
    assert L.lib().grf_alu_peak(-1, C.byref(v), None) == 1
    assert L.lib().grf_alu_peak(0, None, None) == 1
