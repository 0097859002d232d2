"""ctypes binding of libuw (include/uw.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  The CUDA
library must be built (``paper_2106_00554_gb300.build.build()``); there is no
CPU fallback: if libuw.so is missing the first call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libuw.so")

UW_BOUNDARY_PERIODIC, UW_BOUNDARY_VMP = 0, 1
UW_FILTER_SYMLET = 0x100
UW_F64, UW_F32, UW_F32_SPLIT_BF16 = 0, 1, 2
STATUS = {0: "UW_OK", 1: "UW_ERR_INVALID_ARG", 2: "UW_ERR_UNSUPPORTED", 3: "UW_ERR_OOM",
          4: "UW_ERR_CUDA", 5: "UW_ERR_TIMEOUT", 6: "UW_ERR_INTERNAL"}

_c_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)

# name -> (restype, argtypes)
SIGNATURES = {
    "uw_plan_create": (_c_p, [_int, _int, _int, _int, _int]),
    "uw_plan_set_coarsest": (_int, [_c_p, _int]),
    "uw_plan_set_mask": (_int, [_c_p, _i64p, _i64]),
    "uw_plan_reserve": (_int, [_c_p, _int]),
    "uw_plan_num_samples": (_i64, [_c_p]),
    "uw_plan_num_coeffs": (_i64, [_c_p]),
    "uw_plan_coarsest": (_int, [_c_p]),
    "uw_plan_n": (_i64, [_c_p]),
    "uw_forward": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_adjoint": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_forward_noalloc": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_forward_host": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_adjoint_host": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_forward_host_async": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_adjoint_host_async": (_int, [_c_p, _int, _c_p, _c_p, _int, _c_p]),
    "uw_host_wait": (_int, [_c_p]),
    "uw_group_create": (_c_p, [ctypes.POINTER(_c_p), _int, _int]),
    "uw_group_forward": (_int, [_c_p, _int, ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), _c_p]),
    "uw_group_adjoint": (_int, [_c_p, _int, ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), _c_p]),
    "uw_group_tune": (_int, [_c_p, _int, ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), _int, _c_p]),
    "uw_group_tune_cached": (_int, [_c_p, _int, ctypes.POINTER(_c_p), ctypes.POINTER(_c_p), _int, ctypes.c_char_p,
                                    _c_p]),
    "uw_group_params": (_int, [_c_p, ctypes.POINTER(_int)]),
    "uw_group_device_status": (_int, [_c_p]),
    "uw_group_destroy": (None, [_c_p]),
    "uw_plan_destroy": (None, [_c_p]),
    "uw_plan_table": (_i64, [_c_p, _int, _dp, _i64]),
    "uw_host_table": (_i64, [_int, _int, _int, _dp, _i64]),
    "uw_plan_last_launches": (_int, [_c_p]),
    "uw_plan_device_status": (_int, [_c_p]),
    "uw_plan_profile": (_int, [_c_p, _int]),
    "uw_plan_profile_read": (_int, [_c_p, _int, ctypes.c_char_p, _int, _dp, _i64p, _dp]),
    "uw_fista_step": (_int, [_int, _i64, _c_p, _c_p, _c_p, _c_p, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, _c_p, _c_p, _c_p]),
    "uw_fista_step_backward": (_int, [_int, _i64, _c_p, _c_p, _c_p, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p]),
    "uw_dot": (_int, [_int, _i64, _c_p, _c_p, _c_p, _c_p]),
    "uw_axpby": (_int, [_int, _i64, ctypes.c_double, _c_p, ctypes.c_double, _c_p, _c_p, _c_p]),
    "uw_last_error": (_int, []),
    "uw_last_message": (ctypes.c_char_p, []),
    "uw_status_string": (ctypes.c_char_p, [_int]),
}

_LIB = None


def lib():
    """Load libuw.so (built in-tree).  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIBPATH):
            raise RuntimeError("libuw.so is not built: run paper_2106_00554_gb300.build.build() "
                               "(the CUDA library is required; there is no CPU path)")
        L = ctypes.CDLL(LIBPATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class UWError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().uw_last_message().decode(errors="replace")
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


def _chk(st, where):
    if st != 0:
        raise UWError(st, where)


# --- thin wrappers with the C names -----------------------------------------
def uw_plan_create(d, R, q, p, boundary):
    h = lib().uw_plan_create(d, R, q, p, boundary)
    if not h:
        raise UWError(lib().uw_last_error(), "uw_plan_create")
    return h


def uw_plan_set_coarsest(h, J0):
    _chk(lib().uw_plan_set_coarsest(h, J0), "uw_plan_set_coarsest")


def uw_plan_set_mask(h, omega):
    import numpy as np
    if omega is None:
        _chk(lib().uw_plan_set_mask(h, None, -1), "uw_plan_set_mask")
        return
    om = np.ascontiguousarray(omega, dtype=np.int64)
    _chk(lib().uw_plan_set_mask(h, om.ctypes.data_as(_i64p), om.size), "uw_plan_set_mask")


def uw_plan_reserve(h, max_batch):
    _chk(lib().uw_plan_reserve(h, max_batch), "uw_plan_reserve")


def uw_forward(h, precision, x_ptr, y_ptr, batch, stream):
    _chk(lib().uw_forward(h, precision, x_ptr, y_ptr, batch, stream), "uw_forward")


def uw_adjoint(h, precision, y_ptr, x_ptr, batch, stream):
    _chk(lib().uw_adjoint(h, precision, y_ptr, x_ptr, batch, stream), "uw_adjoint")


def uw_forward_noalloc(h, precision, x_ptr, y_ptr, batch, stream):
    _chk(lib().uw_forward_noalloc(h, precision, x_ptr, y_ptr, batch, stream), "uw_forward_noalloc")


def uw_forward_host(h, precision, x_ptr, y_ptr, batch, stream):
    _chk(lib().uw_forward_host(h, precision, x_ptr, y_ptr, batch, stream), "uw_forward_host")


def uw_adjoint_host(h, precision, y_ptr, x_ptr, batch, stream):
    _chk(lib().uw_adjoint_host(h, precision, y_ptr, x_ptr, batch, stream), "uw_adjoint_host")


def uw_forward_host_async(h, precision, x_ptr, y_ptr, batch, stream):
    _chk(lib().uw_forward_host_async(h, precision, x_ptr, y_ptr, batch, stream), "uw_forward_host_async")


def uw_adjoint_host_async(h, precision, y_ptr, x_ptr, batch, stream):
    _chk(lib().uw_adjoint_host_async(h, precision, y_ptr, x_ptr, batch, stream), "uw_adjoint_host_async")


def uw_host_wait(h):
    _chk(lib().uw_host_wait(h), "uw_host_wait")


def _ptrs(ptrs):
    return (_c_p * len(ptrs))(*ptrs)


def uw_group_create(plan_handles, nstreams):
    g = lib().uw_group_create(_ptrs(plan_handles), len(plan_handles), nstreams)
    if not g:
        raise UWError(lib().uw_last_error(), "uw_group_create")
    return g


def uw_group_forward(g, precision, x_ptrs, y_ptrs, stream):
    _chk(lib().uw_group_forward(g, precision, _ptrs(x_ptrs), _ptrs(y_ptrs), stream), "uw_group_forward")


def uw_group_adjoint(g, precision, y_ptrs, x_ptrs, stream):
    _chk(lib().uw_group_adjoint(g, precision, _ptrs(y_ptrs), _ptrs(x_ptrs), stream), "uw_group_adjoint")


def uw_group_tune(g, precision, x_ptrs, y_ptrs, reps, stream):
    _chk(lib().uw_group_tune(g, precision, _ptrs(x_ptrs), _ptrs(y_ptrs), reps, stream), "uw_group_tune")


def uw_group_tune_cached(g, precision, x_ptrs, y_ptrs, reps, cache_path, stream):
    path = cache_path.encode() if cache_path else None
    _chk(lib().uw_group_tune_cached(g, precision, _ptrs(x_ptrs), _ptrs(y_ptrs), reps, path, stream),
         "uw_group_tune_cached")


def uw_group_params(g):
    out = (_int * 7)()
    _chk(lib().uw_group_params(g, out), "uw_group_params")
    return list(out)


def uw_group_device_status(g):
    return lib().uw_group_device_status(g)


def uw_group_destroy(g):
    lib().uw_group_destroy(g)


def uw_fista_step(precision, n, z, G, B, x0, tau, lam, beta, x1, z1, stream):
    _chk(lib().uw_fista_step(precision, n, z, G, B, x0, tau, lam, beta, x1, z1, stream), "uw_fista_step")


def uw_fista_step_backward(precision, n, z, G, B, tau, lam, beta, gx1, gz1, gz, gG, gB, gx0, glam, stream):
    _chk(lib().uw_fista_step_backward(precision, n, z, G, B, tau, lam, beta, gx1, gz1, gz, gG, gB, gx0, glam,
                                      stream), "uw_fista_step_backward")


def uw_dot(precision, n, a, b, out, stream):
    _chk(lib().uw_dot(precision, n, a, b, out, stream), "uw_dot")


def uw_axpby(precision, n, alpha, a, beta, b, out, stream):
    _chk(lib().uw_axpby(precision, n, alpha, a, beta, b, out, stream), "uw_axpby")


def uw_plan_device_status(h):
    """UW_OK, or UW_ERR_TIMEOUT if a bounded device wait gave up since the
    last query (synchronises the device); returns the status, does not raise."""
    return lib().uw_plan_device_status(h)


def uw_plan_destroy(h):
    lib().uw_plan_destroy(h)


def uw_host_table(p, q, which):
    import numpy as np
    n = lib().uw_host_table(p, q, which, None, 0)
    if n < 0:
        raise ValueError("invalid p or q")
    out = np.zeros(n)
    lib().uw_host_table(p, q, which, out.ctypes.data_as(_dp), n)
    return out


def uw_plan_table(h, which):
    import numpy as np
    n = lib().uw_plan_table(h, which, None, 0)
    out = np.zeros(n)
    lib().uw_plan_table(h, which, out.ctypes.data_as(_dp), n)
    return out


def uw_plan_profile(h, enable):
    _chk(lib().uw_plan_profile(h, 1 if enable else 0), "uw_plan_profile")


def uw_plan_profile_read(h):
    """list of dicts {name, total_ms, launches, bytes_per_launch}"""
    L = lib()
    n = L.uw_plan_profile_read(h, -1, None, 0, None, None, None)
    out = []
    for i in range(n):
        buf = ctypes.create_string_buffer(128)
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        by = ctypes.c_double()
        L.uw_plan_profile_read(h, i, buf, 128, ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(by))
        out.append({"name": buf.value.decode(), "total_ms": ms.value, "launches": cnt.value,
                    "bytes_per_launch": by.value})
    return out
