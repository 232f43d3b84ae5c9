"""GB300 (sm_103a) implementation of the unified fourth-order BGK lattice Boltzmann model for the
d-dimensional linear hyperbolic equation d_t phi + u . grad phi = R (arXiv:2410.13165).

The compute path is the CUDA library liblhe_lbm.so behind the C ABI of include/lhe_lbm.h; this
package only marshals arguments to it. PyTorch provides device memory and streams.

    >>> import torch, paper_2410_13165_gb300 as lhe
    >>> sim = lhe.LBM(d=3, n=64, u=(0.1, 0.1, 0.1))           # D3Q19, periodic, FP64, tau = 1/2
    >>> sim.init(phi0)                                        # phi0: float64 CUDA tensor, shape (S,)
    >>> sim.step(100); phi = sim.macro()
"""
from __future__ import annotations

import ctypes

from . import _abi
from ._abi import LHEError  # noqa: F401

__all__ = ["LBM", "LHEError", "model"]

_BC = {"periodic": _abi.BC_PERIODIC, "fullway": _abi.BC_FULLWAY, "halfway": _abi.BC_HALFWAY}
_PREC = {"fp64": _abi.FP64, "fp32dev": _abi.FP32_DEV}


def _params(d, n, lo=0.0, hi=1.0, u=None, R=0.0, tau=0.5, c=1.0, bc="periodic", bc_order=4, init_order=3,
            precision="fp64", g=0.5, m4=None, allow_unstable=False, stream=0, staged=True,
            pdl=True, flags=0) -> _abi.lhe_lbm_params:
    p = _abi.lhe_lbm_default_params()
    p.d = int(d)
    p.bc = _BC[bc]
    p.precision = _PREC[precision]
    p.init_order = int(init_order)
    p.bc_order = int(bc_order)
    p.allow_unstable = int(bool(allow_unstable))
    p.flags = (0 if staged else _abi.FLAG_NO_STAGING) | (0 if pdl else _abi.FLAG_NO_PDL) | int(flags)
    ns = list(n) if hasattr(n, "__len__") else [n] * d
    los = list(lo) if hasattr(lo, "__len__") else [lo] * d
    his = list(hi) if hasattr(hi, "__len__") else [hi] * d
    us = [0.0] * d if u is None else list(u)
    for i in range(d):
        p.n[i], p.lo[i], p.hi[i], p.u[i] = int(ns[i]), float(los[i]), float(his[i]), float(us[i])
    p.c, p.R, p.tau, p.g = float(c), float(R), float(tau), float(g)
    if m4 is not None:
        p.m4_mode = _abi.M4_EXPLICIT
        vals = list(m4) if hasattr(m4, "__len__") else [m4] * (d * (d - 1) // 2)
        for q, v in enumerate(vals):
            p.m4[q] = float(v)
    p.stream = stream
    return p


def jet_len(d: int) -> int:
    """Number of derivatives in a boundary jet: orders 0..3 in the d + 1 variables (t, x_1..x_d)."""
    return (d + 4) * (d + 3) * (d + 2) // 6


def jet_index(d: int):
    """The derivatives of a boundary jet, in order: tuples of variable indices (0: t, i: x_i),
    non-decreasing, of length 0..3, lexicographic within each length."""
    import itertools

    return [tup for q in range(4) for tup in itertools.combinations_with_replacement(range(d + 1), q)]


def model(d, u, c=1.0, g=0.5, m4=None, allow_unstable=False):
    """EDF weights omega_k, fourth moments and lattice vectors as computed by the library."""
    p = _params(d, 4, u=u, c=c, g=g, m4=m4)
    return _abi.lhe_lbm_model(p, allow_unstable=allow_unstable)


def stability_map(d, sigmas, nxi, tau=0.5, g=0.5, m4=None):
    """Per velocity sigma (rows of sigmas): (rho_max, omega_min) -- the largest spectral radius of the
    amplification matrix over the xi grid and the smallest EDF weight (lhe_lbm_stability_map)."""
    import numpy as np

    sig = np.ascontiguousarray(np.atleast_2d(np.asarray(sigmas, dtype=np.float64)))
    if sig.shape[1] != d:
        raise ValueError("sigmas must have d columns")
    p = _params(d, 4, tau=tau, g=g, m4=m4)
    rho = np.empty(sig.shape[0])
    omin = np.empty(sig.shape[0])
    _abi.lhe_lbm_stability_map(p, sig.ctypes.data, sig.shape[0], nxi, rho.ctypes.data, omin.ctypes.data)
    return rho, omin


class LBM:
    """One lattice-Boltzmann problem on the current CUDA device (owns its population buffers)."""

    def __init__(self, d, n, lo=0.0, hi=1.0, u=None, R=0.0, tau=0.5, c=1.0, bc="periodic", bc_order=4,
                 init_order=3, precision="fp64", g=0.5, m4=None, allow_unstable=False, staged=True, pdl=True,
                 flags=0):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (no CPU fallback)")
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._torch = torch
        self.params = _params(d, n, lo, hi, u, R, tau, c, bc, bc_order, init_order, precision, g, m4,
                              allow_unstable, stream=torch.cuda.current_stream().cuda_stream, staged=staged,
                              pdl=pdl, flags=flags)
        self.h = _abi.lhe_lbm_create(self.params)
        info = _abi.lhe_lbm_info(self.h)
        self.d, self.Q, self.S = info.d, info.Q, info.S
        self.n = [int(self.params.n[i]) for i in range(d)]
        self.dx, self.dt, self.s = info.dx, info.dt, info.s
        self.omega = list(info.omega[: self.Q])
        self.m4 = list(info.m4[: d * (d - 1) // 2])
        self.e = [list(info.e[k * d:(k + 1) * d]) for k in range(self.Q)]
        self.n_boundary = info.n_boundary
        self.state_bytes = int(info.state_bytes)
        self.precision = precision
        self.bc = bc

    # -- helpers
    def _stream(self):
        _abi.lhe_lbm_set_stream(self.h, self._torch.cuda.current_stream(self.device).cuda_stream)

    def _ptr(self, t, numel, name):
        if t is None:
            return None
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous() or t.device != self.device:
            raise TypeError("%s must be a contiguous float64 tensor on %s" % (name, self.device))
        if t.numel() != numel:
            raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
        return t.data_ptr()

    @property
    def step_index(self) -> int:
        return int(_abi.lhe_lbm_info(self.h).step)

    # -- forward
    def init(self, phi0, grad=None, R=None):
        self._stream()
        _abi.lhe_lbm_init(self.h, self._ptr(phi0, self.S, "phi0"), self._ptr(grad, self.d * self.S, "grad"),
                          self._ptr(R, self.S, "R"))

    def set_boundary_wave(self, a=(), kappa=(), theta=(), b=0.0, g=None):
        w = _abi.lhe_wave()
        w.nmodes = len(a)
        w.b = float(b)
        for i in range(self.d):
            w.g[i] = 0.0 if g is None else float(g[i])
        for m in range(len(a)):
            w.a[m] = float(a[m])
            w.theta[m] = float(theta[m]) if len(theta) else 0.0
            for i in range(self.d):
                w.kappa[m * _abi.MAX_DIM + i] = float(kappa[m][i])
        self._stream()
        _abi.lhe_lbm_set_boundary_wave(self.h, w)

    def set_source(self, R=None):
        """Per-site source R(x) (float64 tensor of S values) for the steps from the next one on, or
        None for the constant R (lhe_lbm_set_source)."""
        self._stream()
        _abi.lhe_lbm_set_source(self.h, self._ptr(R, self.S, "R"))

    def set_boundary_sine_product(self, A=1.0, lam=1.0, kappa=None, theta=None):
        """Boundary data and source of phi* = A exp(-lam t) prod_i sin(kappa_i x_i + theta_i) (default
        kappa_i = pi, theta_i = 0), formed on the device for every following step; initialise with
        R(x, 0) of the same solution (lhe_lbm_set_boundary_sine_product)."""
        import math

        sp = _abi.lhe_sine_product()
        sp.A, sp.lam = float(A), float(lam)
        for i in range(self.d):
            sp.kappa[i] = math.pi if kappa is None else float(kappa[i])
            sp.theta[i] = 0.0 if theta is None else float(theta[i])
        self._stream()
        _abi.lhe_lbm_set_boundary_sine_product(self.h, sp)

    def boundary_points(self):
        """(points[P][d] as a numpy array, t_offset): the points where the Dirichlet jets of the next
        step are needed (full-way: the boundary nodes; half-way: the mid-link points of the unknown
        populations) and the time of those data relative to the current time step_index * dt."""
        return _abi.lhe_lbm_boundary_points(self.h, self.d)

    def set_boundary_jet(self, jet):
        """Jets of phi at boundary_points() for the next step: a float64 tensor of P * jet_len(d)
        values (every derivative of order 0..3 in (t, x_1..x_d), in the order of jet_index(d))."""
        P = len(self.boundary_points()[0])
        self._stream()
        _abi.lhe_lbm_set_boundary_jet(self.h, self._ptr(jet, P * jet_len(self.d), "jet"))

    def step(self, n: int = 1):
        self._stream()
        _abi.lhe_lbm_step(self.h, n)

    def macro(self, out=None):
        if out is None:
            out = self._torch.empty(self.S, dtype=self._torch.float64, device=self.device)
        self._stream()
        _abi.lhe_lbm_macro(self.h, self._ptr(out, self.S, "out"))
        return out

    def diagnostics(self) -> dict:
        self._stream()
        v, st = _abi.lhe_lbm_diagnostics(self.h)
        return {"mass": v[0], "entropy": v[1], "max_abs": v[2], "nonfinite": int(v[3]), "ok": st == _abi.OK}

    def get_state(self, out=None):
        if out is None:
            out = self._torch.empty(self.state_bytes, dtype=self._torch.uint8, device=self.device)
        self._stream()
        _abi.lhe_lbm_get_state(self.h, out.data_ptr())
        return out

    def set_state(self, buf, step: int):
        self._stream()
        _abi.lhe_lbm_set_state(self.h, buf.data_ptr(), step)

    # -- adjoint
    def adjoint_seed(self, dL_dphiT):
        self._stream()
        _abi.lhe_lbm_adjoint_seed(self.h, self._ptr(dL_dphiT, self.S, "dL_dphiT"))

    def adjoint_step(self, n: int = 1):
        self._stream()
        _abi.lhe_lbm_adjoint_step(self.h, n)

    def adjoint_grads(self, want_grad=False, want_R=True):
        torch = self._torch
        gphi = torch.empty(self.S, dtype=torch.float64, device=self.device)
        ggrad = torch.empty(self.d * self.S, dtype=torch.float64, device=self.device) if want_grad else None
        gR = torch.empty(self.S, dtype=torch.float64, device=self.device) if want_R else None
        self._stream()
        _abi.lhe_lbm_adjoint_grads(self.h, gphi.data_ptr(), None if ggrad is None else ggrad.data_ptr(),
                                   None if gR is None else gR.data_ptr())
        return gphi, ggrad, gR

    def adjoint_jet_grad(self, out=None):
        """dL/d(jet) of the Dirichlet data of the step that the next adjoint_step(1) reverses, as a
        (P, jet_len(d)) float64 tensor at boundary_points() (lhe_lbm_adjoint_jet_grad)."""
        P = len(self.boundary_points()[0])
        JL = jet_len(self.d)
        if out is None:
            out = self._torch.empty((P, JL), dtype=self._torch.float64, device=self.device)
        self._stream()
        _abi.lhe_lbm_adjoint_jet_grad(self.h, self._ptr(out, P * JL, "out"))
        return out

    def close(self):
        if getattr(self, "h", None):
            _abi.lhe_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
