"""The C-ABI library builds, loads and exports every entry point include/lhe_lbm.h declares; its
host-side model agrees with the independent oracle. No GPU compute is run here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "lhe_lbm.h")).read()
    return sorted(set(re.findall(r"^LHE_API[^(]*?\b(lhe_lbm_\w+)\s*\(", src, flags=re.M)))


def test_header_and_binding_agree():
    assert _declared() == sorted(_abi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_struct_layout_and_version(lib):
    assert lib.lhe_lbm_abi_version() == _abi.ABI_VERSION
    assert lib.lhe_lbm_params_size() == ctypes.sizeof(_abi.lhe_lbm_params)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_library_model_matches_the_oracle(lib, d):
    rng = np.random.default_rng(123 + d)
    for _ in range(5):
        u = rng.uniform(-0.15, 0.15, d)
        p = _abi.lhe_lbm_default_params()
        p.d = d
        for i in range(d):
            p.u[i] = u[i]
        omega, m4, e = _abi.lhe_lbm_model(p, allow_unstable=True)
        assert np.array_equal(np.array(e), O.velocities(d))
        want_m4 = O.m4_rule(d, u, 0.5)
        assert np.allclose(m4, want_m4, rtol=0, atol=1e-16)
        assert np.max(np.abs(np.array(omega) - O.weights_closed(d, u, want_m4))) < 1e-15


def test_library_model_with_c_and_explicit_m4(lib):
    p = _abi.lhe_lbm_default_params()
    p.d, p.c, p.m4_mode = 3, 2.0, _abi.M4_EXPLICIT
    for i, v in enumerate((0.1, -0.2, 0.3)):
        p.u[i] = v
    for q, v in enumerate((0.08, 0.09, 0.1)):
        p.m4[q] = v
    omega, m4, _ = _abi.lhe_lbm_model(p, allow_unstable=True)
    sigma = np.array([0.1, -0.2, 0.3]) / 2.0
    assert np.max(np.abs(np.array(omega) - O.weights_closed(3, sigma, [0.08, 0.09, 0.1]))) < 1e-15


def test_model_reports_instability_and_bad_arguments(lib):
    p = _abi.lhe_lbm_default_params()
    p.d = 4
    for i in range(4):
        p.u[i] = 0.4  # Example 3: not entropy stable
    with pytest.raises(_abi.LHEError) as ei:
        _abi.lhe_lbm_model(p)
    assert ei.value.status == _abi.ERR_UNSTABLE
    for field, value in (("d", 6), ("tau", 0.0), ("c", -1.0), ("init_order", 2), ("g", 1.5)):
        q = _abi.lhe_lbm_default_params()
        setattr(q, field, value)
        with pytest.raises(_abi.LHEError) as ei:
            _abi.lhe_lbm_model(q)
        assert ei.value.status == _abi.ERR_ARG
        assert lib.lhe_lbm_last_error(None)
    q = _abi.lhe_lbm_default_params()
    q.bc, q.bc_order = _abi.BC_FULLWAY, 2
    with pytest.raises(_abi.LHEError):
        _abi.lhe_lbm_model(q)
    q = _abi.lhe_lbm_default_params()
    q.n[1] = 17  # not a square lattice on [0,1]^3
    with pytest.raises(_abi.LHEError):
        _abi.lhe_lbm_model(q)


def test_binding_refuses_a_missing_library(tmp_path):
    with pytest.raises(RuntimeError):
        _abi._lib = None
        _abi.load(str(tmp_path / "nope.so"))
    _abi._lib = None


def test_create_rejects_oversized_and_unknown_flag_arguments_before_touching_the_device(lib):
    """Size and argument checks of lhe_lbm_create run before any CUDA call, so they hold on a machine
    without a GPU: a lattice above 2^31 - 1 nodes (32-bit node indices), unknown flag bits."""
    p = _abi.lhe_lbm_default_params()
    p.d = 3
    for i, n in enumerate((2048, 2048, 1024)):   # 2^32 nodes on a square lattice
        p.n[i], p.lo[i], p.hi[i] = n, 0.0, float(n)
    with pytest.raises(_abi.LHEError) as ei:
        _abi.lhe_lbm_create(p)
    assert ei.value.status == _abi.ERR_ARG
    assert b"2^31" in lib.lhe_lbm_last_error(None)
    q = _abi.lhe_lbm_default_params()
    q.flags = 0x10  # bits 1, 2, 4 and 8 are defined
    with pytest.raises(_abi.LHEError) as ei:
        _abi.lhe_lbm_create(q)
    assert ei.value.status == _abi.ERR_ARG


def test_stability_map_argument_checks_without_a_device(lib):
    """lhe_lbm_stability_map validates its arguments on the host (no device work for bad input or
    an empty batch)."""
    import ctypes

    p = _abi.lhe_lbm_default_params()
    p.d = 5
    sig = (ctypes.c_double * 5)()
    out = (ctypes.c_double * 1)()
    st = lib.lhe_lbm_stability_map(ctypes.byref(p), ctypes.addressof(sig), 1, 4, ctypes.addressof(out),
                                   ctypes.addressof(out))
    assert st == _abi.ERR_ARG
    p.d = 2
    assert lib.lhe_lbm_stability_map(ctypes.byref(p), ctypes.addressof(sig), 1, 0, ctypes.addressof(out),
                                     ctypes.addressof(out)) == _abi.ERR_ARG
    assert lib.lhe_lbm_stability_map(ctypes.byref(p), None, 0, 8, None, None) == _abi.OK
