"""ctypes declarations of the C ABI in include/lhe_lbm.h (argument marshalling only).

Every function of the header is available here under the same name; a non-zero status raises
LHEError carrying the library's message. The library is the in-tree liblhe_lbm.so built by
``paper_2410_13165_gb300.build``; there is no fallback when it is missing.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "liblhe_lbm.so")

MAX_DIM, MAX_Q, MAX_MODES = 5, 51, 16
ABI_VERSION = 1

OK, ERR_ARG, ERR_UNSTABLE, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_STATE = range(7)
STATUS_NAMES = ["LHE_OK", "LHE_ERR_ARG", "LHE_ERR_UNSTABLE", "LHE_ERR_CUDA", "LHE_ERR_OOM", "LHE_ERR_NONFINITE",
                "LHE_ERR_STATE"]
BC_PERIODIC, BC_FULLWAY, BC_HALFWAY = 0, 1, 2
FP64, FP32_DEV = 0, 1
M4_RULE, M4_EXPLICIT = 0, 1
FLAG_NO_STAGING = 1
FLAG_NO_PDL = 2
FLAG_TEST_EXPIRE_WAIT = 4  # test hook: the first staged launch of a handle takes its wait-timeout path
FLAG_NODE_BOUNDARY = 8

# every entry point declared in include/lhe_lbm.h
EXPORTS = [
    "lhe_lbm_abi_version", "lhe_lbm_params_size", "lhe_lbm_default_params", "lhe_lbm_model", "lhe_lbm_create",
    "lhe_lbm_destroy", "lhe_lbm_last_error", "lhe_lbm_info", "lhe_lbm_set_stream", "lhe_lbm_init",
    "lhe_lbm_set_boundary_wave", "lhe_lbm_step", "lhe_lbm_macro", "lhe_lbm_diagnostics", "lhe_lbm_get_state",
    "lhe_lbm_set_state", "lhe_lbm_adjoint_seed", "lhe_lbm_adjoint_step", "lhe_lbm_adjoint_grads",
    "lhe_lbm_diagnostics_noalloc", "lhe_lbm_stability_map", "lhe_lbm_boundary_points", "lhe_lbm_set_boundary_jet",
    "lhe_lbm_adjoint_jet_grad", "lhe_lbm_set_source", "lhe_lbm_set_boundary_sine_product",
]


class lhe_lbm_params(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32), ("bc", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("init_order", ctypes.c_int32), ("bc_order", ctypes.c_int32), ("m4_mode", ctypes.c_int32),
        ("allow_unstable", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("n", ctypes.c_int64 * MAX_DIM), ("lo", ctypes.c_double * MAX_DIM), ("hi", ctypes.c_double * MAX_DIM),
        ("c", ctypes.c_double), ("u", ctypes.c_double * MAX_DIM), ("R", ctypes.c_double),
        ("tau", ctypes.c_double), ("g", ctypes.c_double), ("m4", ctypes.c_double * 10),
        ("stream", ctypes.c_void_p),
    ]


class lhe_lbm_info_t(ctypes.Structure):
    _fields_ = [
        ("d", ctypes.c_int32), ("Q", ctypes.c_int32), ("S", ctypes.c_int64), ("n_boundary", ctypes.c_int64),
        ("step", ctypes.c_int64), ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("s", ctypes.c_double),
        ("m4", ctypes.c_double * 10), ("omega", ctypes.c_double * MAX_Q),
        ("e", ctypes.c_int32 * (MAX_Q * MAX_DIM)), ("state_bytes", ctypes.c_uint64),
    ]


class lhe_wave(ctypes.Structure):
    _fields_ = [
        ("nmodes", ctypes.c_int32), ("reserved0", ctypes.c_int32), ("b", ctypes.c_double),
        ("g", ctypes.c_double * MAX_DIM), ("a", ctypes.c_double * MAX_MODES),
        ("kappa", ctypes.c_double * (MAX_MODES * MAX_DIM)), ("theta", ctypes.c_double * MAX_MODES),
    ]


class lhe_sine_product(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_double), ("lam", ctypes.c_double), ("kappa", ctypes.c_double * MAX_DIM),
        ("theta", ctypes.c_double * MAX_DIM),
    ]


class LHEError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


_lib = None
_H = ctypes.c_void_p
_D = ctypes.c_void_p  # device or host pointer (int address)


def load(path: str | None = None):
    """Load liblhe_lbm.so; raises when it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIBPATH
    if not os.path.exists(path):
        raise RuntimeError("liblhe_lbm.so is missing: build it with `python -m paper_2410_13165_gb300.build` "
                           "(or __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    sig = {
        "lhe_lbm_abi_version": (ctypes.c_int32, []),
        "lhe_lbm_params_size": (ctypes.c_uint64, []),
        "lhe_lbm_default_params": (st, [ctypes.POINTER(lhe_lbm_params)]),
        "lhe_lbm_model": (st, [ctypes.POINTER(lhe_lbm_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.POINTER(ctypes.c_int32)]),
        "lhe_lbm_create": (st, [ctypes.POINTER(lhe_lbm_params), ctypes.POINTER(_H)]),
        "lhe_lbm_destroy": (st, [_H]),
        "lhe_lbm_last_error": (ctypes.c_char_p, [_H]),
        "lhe_lbm_info": (st, [_H, ctypes.POINTER(lhe_lbm_info_t)]),
        "lhe_lbm_set_stream": (st, [_H, ctypes.c_void_p]),
        "lhe_lbm_set_source": (st, [_H, _D]),
        "lhe_lbm_init": (st, [_H, _D, _D, _D]),
        "lhe_lbm_set_boundary_wave": (st, [_H, ctypes.POINTER(lhe_wave)]),
        "lhe_lbm_set_boundary_sine_product": (st, [_H, ctypes.POINTER(lhe_sine_product)]),
        "lhe_lbm_boundary_points": (st, [_H, _D, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
        "lhe_lbm_set_boundary_jet": (st, [_H, _D]),
        "lhe_lbm_step": (st, [_H, ctypes.c_int64]),
        "lhe_lbm_macro": (st, [_H, _D]),
        "lhe_lbm_diagnostics": (st, [_H, ctypes.POINTER(ctypes.c_double)]),
        "lhe_lbm_get_state": (st, [_H, _D]),
        "lhe_lbm_set_state": (st, [_H, _D, ctypes.c_int64]),
        "lhe_lbm_adjoint_seed": (st, [_H, _D]),
        "lhe_lbm_adjoint_step": (st, [_H, ctypes.c_int64]),
        "lhe_lbm_adjoint_grads": (st, [_H, _D, _D, _D]),
        "lhe_lbm_adjoint_jet_grad": (st, [_H, _D]),
        "lhe_lbm_diagnostics_noalloc": (st, [ctypes.POINTER(lhe_lbm_params), _D, _D, _D]),
        "lhe_lbm_stability_map": (st, [ctypes.POINTER(lhe_lbm_params), _D, ctypes.c_int64, ctypes.c_int32, _D, _D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype, fn.argtypes = res, args
    if L.lhe_lbm_abi_version() != ABI_VERSION:
        raise RuntimeError("liblhe_lbm.so ABI version mismatch")
    if L.lhe_lbm_params_size() != ctypes.sizeof(lhe_lbm_params):
        raise RuntimeError("lhe_lbm_params layout mismatch between the binding and the library")
    _lib = L
    return L


def check(status: int, handle=None) -> None:
    if status != OK:
        msg = load().lhe_lbm_last_error(handle)
        raise LHEError(status, msg.decode() if msg else "")


# ---- thin wrappers with the C names (raise on error) ----

def lhe_lbm_default_params() -> lhe_lbm_params:
    p = lhe_lbm_params()
    check(load().lhe_lbm_default_params(ctypes.byref(p)))
    return p


def lhe_lbm_model(p: lhe_lbm_params, allow_unstable: bool = False):
    """Returns (omega[Q], m4[npairs], e[Q][d]) computed by the library."""
    L = load()
    om = (ctypes.c_double * MAX_Q)()
    m4 = (ctypes.c_double * 10)()
    e = (ctypes.c_int32 * (MAX_Q * MAX_DIM))()
    Q = ctypes.c_int32()
    st = L.lhe_lbm_model(ctypes.byref(p), ctypes.addressof(om), ctypes.addressof(m4), ctypes.addressof(e),
                         ctypes.byref(Q))
    if not (st == OK or (allow_unstable and st == ERR_UNSTABLE)):
        check(st)
    d = p.d
    return (list(om[: Q.value]), list(m4[: d * (d - 1) // 2]),
            [list(e[k * d:(k + 1) * d]) for k in range(Q.value)])


def lhe_lbm_create(p: lhe_lbm_params):
    h = _H()
    check(load().lhe_lbm_create(ctypes.byref(p), ctypes.byref(h)))
    return h


def lhe_lbm_destroy(h) -> None:
    check(load().lhe_lbm_destroy(h), h)


def lhe_lbm_info(h) -> lhe_lbm_info_t:
    info = lhe_lbm_info_t()
    check(load().lhe_lbm_info(h, ctypes.byref(info)), h)
    return info


def lhe_lbm_set_stream(h, stream: int) -> None:
    check(load().lhe_lbm_set_stream(h, stream), h)


def lhe_lbm_init(h, phi0_ptr: int, grad_ptr: int | None, R_ptr: int | None) -> None:
    check(load().lhe_lbm_init(h, phi0_ptr, grad_ptr, R_ptr), h)


def lhe_lbm_set_boundary_wave(h, w: lhe_wave) -> None:
    check(load().lhe_lbm_set_boundary_wave(h, ctypes.byref(w)), h)


def lhe_lbm_set_boundary_sine_product(h, sp: lhe_sine_product) -> None:
    check(load().lhe_lbm_set_boundary_sine_product(h, ctypes.byref(sp)), h)


def lhe_lbm_boundary_points(h, d: int):
    """(points[P][d], t_offset): where the Dirichlet jets of the next step are needed and the time of
    the data relative to the current step's time."""
    import numpy as np

    L = load()
    P = ctypes.c_int64(0)
    toff = ctypes.c_double(0.0)
    check(L.lhe_lbm_boundary_points(h, None, ctypes.byref(P), ctypes.byref(toff)), h)
    pts = np.zeros((P.value, d), dtype=np.float64)
    if P.value:
        check(L.lhe_lbm_boundary_points(h, pts.ctypes.data, ctypes.byref(P), ctypes.byref(toff)), h)
    return pts, toff.value


def lhe_lbm_set_boundary_jet(h, jet_ptr: int) -> None:
    check(load().lhe_lbm_set_boundary_jet(h, jet_ptr), h)


def lhe_lbm_set_source(h, R_ptr) -> None:
    check(load().lhe_lbm_set_source(h, R_ptr), h)


def lhe_lbm_step(h, n: int) -> None:
    check(load().lhe_lbm_step(h, int(n)), h)


def lhe_lbm_macro(h, phi_ptr: int) -> None:
    check(load().lhe_lbm_macro(h, phi_ptr), h)


def lhe_lbm_diagnostics(h):
    out = (ctypes.c_double * 4)()
    st = load().lhe_lbm_diagnostics(h, out)
    if st not in (OK, ERR_NONFINITE):
        check(st, h)
    return list(out), st


def lhe_lbm_get_state(h, buf_ptr: int) -> None:
    check(load().lhe_lbm_get_state(h, buf_ptr), h)


def lhe_lbm_set_state(h, buf_ptr: int, step: int) -> None:
    check(load().lhe_lbm_set_state(h, buf_ptr, int(step)), h)


def lhe_lbm_adjoint_seed(h, seed_ptr: int) -> None:
    check(load().lhe_lbm_adjoint_seed(h, seed_ptr), h)


def lhe_lbm_adjoint_step(h, n: int) -> None:
    check(load().lhe_lbm_adjoint_step(h, int(n)), h)


def lhe_lbm_adjoint_grads(h, gphi0_ptr: int, ggrad_ptr: int | None, gR_ptr: int | None) -> None:
    check(load().lhe_lbm_adjoint_grads(h, gphi0_ptr, ggrad_ptr, gR_ptr), h)


def lhe_lbm_adjoint_jet_grad(h, out_ptr: int) -> None:
    check(load().lhe_lbm_adjoint_jet_grad(h, out_ptr), h)


def lhe_lbm_diagnostics_noalloc(p: lhe_lbm_params, pop_ptr: int, R_ptr: int | None, out_ptr: int) -> None:
    """Diagnostics of a caller-owned FP64 state into 4 device doubles, with no device allocation."""
    check(load().lhe_lbm_diagnostics_noalloc(ctypes.byref(p), pop_ptr, R_ptr, out_ptr))


def lhe_lbm_stability_map(p: lhe_lbm_params, sigma_ptr: int, npoints: int, nxi: int, rho_ptr: int, omin_ptr: int) -> None:
    """Stability map of host arrays (see the header): rho_max and omega_min per velocity."""
    check(load().lhe_lbm_stability_map(ctypes.byref(p), sigma_ptr, int(npoints), int(nxi), rho_ptr, omin_ptr))
