"""ctypes binding of libgrf.so: the C ABI of include/grf.h, one Python function
per C function with the same name.  Argument marshalling only; every step of
the sampling path runs in the library's CUDA kernels.  Loading fails loudly if
the library has not been built: there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

GRF_OK = 0
GRF_ERR_INVALID_ARG = 1
GRF_ERR_UNSUPPORTED = 2
GRF_ERR_OOM = 3
GRF_ERR_CUDA = 4
GRF_ERR_TIMEOUT = 5
GRF_ERR_NOT_HERMITIAN = 6

GRF_MATERN = 0
GRF_GAUSSIAN = 1
GRF_PAPER_POLY = 2
GRF_ALG_TWO_FFT = 1
GRF_ALG_ONE_FFT = 2
GRF_FP32 = 0
GRF_FP64 = 1
GRF_BC_NEUMANN = 1
GRF_BC_DIRICHLET = 2


class grf_spectrum(C.Structure):
    _fields_ = [("family", C.c_int), ("sigma", C.c_double), ("ell", C.c_double), ("nu", C.c_double),
                ("m", C.c_double), ("k", C.c_int), ("l", C.c_int), ("n", C.c_int),
                ("normalize_discrete", C.c_int)]


class GRFError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, _status_text(status), detail))


_lib = None


def lib():
    """The loaded library (raises if libgrf.so is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError("libgrf.so is not built (run __graft_entry__.build()); "
                               "the GRF path has no CPU fallback")
        L = C.CDLL(LIB)
        P, I64, U64, VP, D = C.c_void_p, C.c_int64, C.c_uint64, C.c_void_p, C.c_double
        sig = {
            "grf_plan_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(I64), C.POINTER(D),
                                          C.POINTER(grf_spectrum), C.c_int, C.c_int, I64]),
            "grf_bc_plan_create": (C.c_int, [C.POINTER(P), C.c_int, C.POINTER(I64), C.POINTER(D),
                                             C.POINTER(grf_spectrum), C.c_int, I64]),
            "grf_plan_set_spectrum": (C.c_int, [P, C.POINTER(grf_spectrum), VP]),
            "grf_plan_tune": (C.c_int, [P, VP]),
            "grf_sample": (C.c_int, [P, U64, I64, VP, VP]),
            "grf_sample_host": (C.c_int, [P, U64, I64, VP, VP]),
            "grf_backward": (C.c_int, [P, U64, I64, VP, VP, VP]),
            "grf_rfft_forward": (C.c_int, [P, I64, VP, VP, VP]),
            "grf_batch_plan_create": (C.c_int, [C.POINTER(P), I64, C.POINTER(C.c_int), C.POINTER(I64),
                                                C.POINTER(D), C.POINTER(grf_spectrum), C.c_int]),
            "grf_batch_sample": (C.c_int, [P, U64, C.POINTER(VP), VP]),
            "grf_batch_graph_launch": (C.c_int, [P, U64, C.POINTER(VP), VP]),
            "grf_status_word": (C.c_int, [P, VP]),
            "grf_batch_set_debug": (C.c_int, [P, C.c_int, C.c_double]),
            "grf_batch_set_mode": (C.c_int, [P, C.c_int]),
            "grf_philox_words": (C.c_int, [U64, C.c_uint32, U64, I64, VP, VP]),
            "grf_cov_origin": (C.c_int, [P, U64, I64, VP, VP]),
            "grf_sample_2d_static": (C.c_int, [C.POINTER(I64), C.POINTER(D), C.POINTER(grf_spectrum), U64, I64,
                                               VP, VP]),
            "grf_alu_peak": (C.c_int, [C.c_int, C.POINTER(D), VP]),
            "grf_plan_query": (I64, [P, C.c_int]),
            "grf_plan_timing": (C.c_int, [P, I64]),
            "grf_plan_timing_read": (I64, [P, C.POINTER(C.c_int), C.POINTER(C.c_float), I64]),
            "grf_plan_destroy": (C.c_int, [P]),
            "grf_status_string": (C.c_char_p, [C.c_int]),
            "grf_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _status_text(s: int) -> str:
    try:
        return lib().grf_status_string(s).decode()
    except Exception:
        return str(s)


def check(status: int, where: str):
    if status != GRF_OK:
        raise GRFError(status, where, lib().grf_last_error().decode())


def make_spectrum(family=GRF_MATERN, sigma=1.0, ell=0.1, nu=1.5, m=1.0, k=1, l=1, n=1, normalize_discrete=0):
    return grf_spectrum(int(family), float(sigma), float(ell), float(nu), float(m), int(k), int(l), int(n),
                        int(normalize_discrete))


def grf_plan_create(d, n, L, spec, alg=GRF_ALG_ONE_FFT, prec=GRF_FP32, max_batch=1):
    h = C.c_void_p()
    nn = (C.c_int64 * d)(*[int(x) for x in n])
    LL = (C.c_double * d)(*[float(x) for x in L])
    check(lib().grf_plan_create(C.byref(h), int(d), nn, LL, C.byref(spec), int(alg), int(prec), int(max_batch)),
          "grf_plan_create")
    return h


def grf_bc_plan_create(d, n, L, spec, bc, max_batch=1):
    h = C.c_void_p()
    nn = (C.c_int64 * d)(*[int(x) for x in n])
    LL = (C.c_double * d)(*[float(x) for x in L])
    check(lib().grf_bc_plan_create(C.byref(h), int(d), nn, LL, C.byref(spec), int(bc), int(max_batch)),
          "grf_bc_plan_create")
    return h


def grf_plan_set_spectrum(plan, spec, stream=0):
    check(lib().grf_plan_set_spectrum(plan, C.byref(spec), C.c_void_p(stream)), "grf_plan_set_spectrum")


def grf_plan_tune(plan, stream=0):
    check(lib().grf_plan_tune(plan, C.c_void_p(stream)), "grf_plan_tune")


SCHEDULE_KEYS = {"T": 7, "colA_P": 8, "colA_C": 9, "row_P": 10, "row_C": 11, "pipe": 12, "colB_P": 13, "colB_C": 14,
                 "row_tma": 15}


def grf_plan_schedule(plan):
    return {k: grf_plan_query(plan, v) for k, v in SCHEDULE_KEYS.items()}


def grf_sample(plan, seed, batch, out_ptr, stream=0):
    check(lib().grf_sample(plan, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(batch), C.c_void_p(out_ptr),
                           C.c_void_p(stream)), "grf_sample")


def grf_sample_host(plan, seed, batch, host_ptr, stream=0):
    check(lib().grf_sample_host(plan, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(batch), C.c_void_p(host_ptr),
                                C.c_void_p(stream)), "grf_sample_host")


def grf_backward(plan, seed, batch, grad_out_ptr, grad_params_ptr, stream=0):
    check(lib().grf_backward(plan, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(batch), C.c_void_p(grad_out_ptr),
                             C.c_void_p(grad_params_ptr), C.c_void_p(stream)), "grf_backward")


def grf_rfft_forward(plan, batch, in_ptr, out_ptr, stream=0):
    check(lib().grf_rfft_forward(plan, int(batch), C.c_void_p(in_ptr), C.c_void_p(out_ptr), C.c_void_p(stream)),
          "grf_rfft_forward")


def grf_batch_plan_create(dims, shapes, lengths, specs):
    count = len(dims)
    h = C.c_void_p()
    d = (C.c_int * count)(*[int(x) for x in dims])
    n = (C.c_int64 * (3 * count))()
    L = (C.c_double * (3 * count))()
    for i, (shp, ln) in enumerate(zip(shapes, lengths)):
        for j in range(3):
            n[3 * i + j] = int(shp[j]) if j < len(shp) else 1
            L[3 * i + j] = float(ln[j]) if j < len(ln) else 1.0
    sp = (grf_spectrum * count)(*specs)
    check(lib().grf_batch_plan_create(C.byref(h), count, d, n, L, sp, GRF_FP32), "grf_batch_plan_create")
    return h


def _ptr_array(ptrs):
    return (C.c_void_p * len(ptrs))(*[C.c_void_p(int(p)) for p in ptrs])


def grf_batch_sample(plan, seed, out_ptrs, stream=0):
    arr = _ptr_array(out_ptrs)
    check(lib().grf_batch_sample(plan, C.c_uint64(seed), arr, C.c_void_p(stream)), "grf_batch_sample")


def grf_batch_graph_launch(plan, seed, out_ptrs, stream=0):
    arr = _ptr_array(out_ptrs)
    check(lib().grf_batch_graph_launch(plan, C.c_uint64(seed), arr, C.c_void_p(stream)), "grf_batch_graph_launch")


def grf_batch_set_debug(plan, withhold_field=-1, timeout_ms=0.0):
    check(lib().grf_batch_set_debug(plan, int(withhold_field), float(timeout_ms)), "grf_batch_set_debug")


def grf_batch_set_mode(plan, mode):
    check(lib().grf_batch_set_mode(plan, int(mode)), "grf_batch_set_mode")


def grf_status_word(plan, stream=0) -> int:
    return int(lib().grf_status_word(plan, C.c_void_p(stream)))


def grf_philox_words(key, tag, q0, count, out_ptr, stream=0):
    check(lib().grf_philox_words(C.c_uint64(key & 0xFFFFFFFFFFFFFFFF), C.c_uint32(tag), C.c_uint64(q0), int(count),
                                 C.c_void_p(out_ptr), C.c_void_p(stream)), "grf_philox_words")


def grf_cov_origin(plan, seed, count, sums_ptr, stream=0):
    check(lib().grf_cov_origin(plan, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(count), C.c_void_p(sums_ptr),
                               C.c_void_p(stream)), "grf_cov_origin")


def grf_sample_2d_static(n, L, spec, seed, batch, out_ptr, stream=0):
    """2-D FP32 Algorithm 2 sampling that allocates no device memory (see grf.h)."""
    nn = (C.c_int64 * 2)(*[int(x) for x in n])
    LL = (C.c_double * 2)(*[float(x) for x in L])
    check(lib().grf_sample_2d_static(nn, LL, C.byref(spec), C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(batch),
                                     C.c_void_p(out_ptr), C.c_void_p(stream)), "grf_sample_2d_static")


ALU_PEAK_KINDS = {"fma": 0, "philox": 1, "mufu": 2}


def grf_alu_peak(kind: str, stream=0) -> float:
    """Measured operations per second of one microbenchmark kind (see grf.h)."""
    v = C.c_double()
    check(lib().grf_alu_peak(ALU_PEAK_KINDS[kind], C.byref(v), C.c_void_p(stream)), "grf_alu_peak")
    return float(v.value)


def grf_plan_query(plan, key: int) -> int:
    return int(lib().grf_plan_query(plan, int(key)))


KERNEL_KINDS = {0: "noise_columns", 1: "columns", 2: "rows_c2r", 3: "rows_r2c", 4: "rows_1d", 5: "plain64",
                6: "reduce", 7: "r2r_noise_rows", 8: "r2r_columns"}


def grf_plan_timing(plan, cap):
    check(lib().grf_plan_timing(plan, int(cap)), "grf_plan_timing")


def grf_plan_timing_read(plan, cap_out=1 << 16):
    kinds = (C.c_int * cap_out)()
    ms = (C.c_float * cap_out)()
    n = int(lib().grf_plan_timing_read(plan, kinds, ms, cap_out))
    m = min(n, cap_out)
    return n, [(KERNEL_KINDS.get(kinds[i], str(kinds[i])), float(ms[i])) for i in range(m)]


def grf_plan_destroy(plan):
    check(lib().grf_plan_destroy(plan), "grf_plan_destroy")
