"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle, element by element.

Tolerances (relative max-norm of phi): FP64 path 1e-13; FP32-deviation path 1e-5. The norm is
taken relative to the larger of the final and the initial field: with tau != 1/2 the scheme is
dissipative and under-resolved modes decay by many orders of magnitude, after which a norm relative
to the final field alone would compare rounding noise.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import LBM, LHEError, build, workloads as W
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13
DEV_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def relerr(a, b, scale=0.0):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), scale, 1e-300))


def run_pair(d, n, u, steps, lo=0.0, hi=1.0, tau=0.5, R=0.0, bc="periodic", bc_order=4, init_order=3,
             precision="fp64", nmodes=4, seed=0, lin=None, explicit_grad=True, Rfield=None, return_models=False):
    n = list(n) if hasattr(n, "__len__") else [n] * d
    m = O.Model(d, n, lo, hi, u, tau=tau, R=R, bc=bc, bc_order=bc_order)
    X = W.node_coords(d, n, lo, m.dx, halfway=(bc == "halfway"))
    assert np.allclose(X, m.coords(), atol=1e-14, rtol=0)
    F = W.fourier_field(d, nmodes, seed, lo, hi)
    b, g = (0.0, None) if lin is None else lin
    phi0 = F.value(X) + b + (0.0 if g is None else np.asarray(g) @ X)
    grad = F.grad(X) + (0.0 if g is None else np.asarray(g)[:, None])
    a, kap, th = F.wave_params()
    wave = m.wave(a=a, kappa=kap, theta=th, b=b, g=g)
    f = m.init(phi0, grad if explicit_grad else None, init_order)
    f = m.step(f, 0, steps, wave=wave, Rfield=Rfield)
    phi_o = m.phi(f)
    sim = LBM(d, n, lo, hi, u=u, R=R, tau=tau, bc=bc, bc_order=bc_order, init_order=init_order, precision=precision)
    sim.init(_t(phi0), _t(grad) if explicit_grad else None, None if Rfield is None else _t(Rfield))
    if bc != "periodic":
        sim.set_boundary_wave(a, kap, th, b, g)
    sim.step(steps)
    phi_g = sim.macro().cpu().numpy()
    run_pair.scale = float(np.max(np.abs(phi0)))
    if return_models:
        return phi_g, phi_o, sim, m, f
    sim.close()
    return phi_g, phi_o


def rel(g, o):
    """Relative max-norm against the larger of the final and the initial field of the last run_pair."""
    return relerr(g, o, run_pair.scale)


# ------------------------------------------------------------------------------ FP64, periodic

@pytest.mark.parametrize("tau", [0.5, 0.8])
def test_fp64_d2q9_64_periodic_200_steps(tau):
    """D2Q9 64x64, 4 seeded Fourier modes, u inside the stability region, 200 steps."""
    g, o = run_pair(2, 64, (0.1, 0.2), 200, tau=tau, nmodes=4, seed=1)
    assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("d,n", [(1, (37,)), (2, (33, 29)), (3, (19, 17, 13)), (4, (7, 6, 5, 9)), (5, (5, 4, 6, 5, 3))])
def test_fp64_periodic_ragged_extents_all_dimensions(d, n):
    u = [0.1, -0.05, 0.08, 0.03, -0.02][:d]
    hi = [ni / 32.0 for ni in n]
    g, o = run_pair(d, n, u, 30, hi=hi, tau=0.5, nmodes=3, seed=d)
    assert relerr(g, o) < FP64_TOL
    g, o = run_pair(d, n, u, 8, hi=hi, tau=0.8, nmodes=3, seed=d)
    assert rel(g, o) < FP64_TOL


@pytest.mark.parametrize("tau", [0.5, 0.8, 1.2])
def test_fp64_d5q51_source_field(tau):
    """D5Q51 (two lanes per node on the GPU) with a per-site source field, each collision form."""
    n = (6, 5, 4, 5, 6)
    S = int(np.prod(n))
    Rf = 0.4 * np.random.default_rng(15).normal(size=S)
    g, o = run_pair(5, n, (0.02, 0.04, 0.06, 0.08, 0.1), 12, hi=[ni / 16.0 for ni in n], tau=tau, Rfield=Rf,
                    nmodes=3, seed=16)
    assert rel(g, o) < FP64_TOL


def test_fp64_d3q19_64cubed_1000_steps():
    """D3Q19 64^3, 8 modes, 1000 steps (the parity case of the 256^3 workload's family)."""
    g, o = run_pair(3, 64, (0.1, 0.1, 0.1), 1000, tau=0.5, nmodes=8, seed=2)
    assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2])
def test_fp64_d3q19_tau_sweep(tau):
    g, o = run_pair(3, 24, (0.1, 0.1, 0.1), 100, tau=tau, nmodes=8, seed=3)
    assert rel(g, o) < FP64_TOL


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2, 0.5])
def test_fp64_d3q19_256cubed_full_size(tau):
    """The benchmark's workload (D3Q19 256^3, 8 modes, tau in {0.6, 0.8, 1.2}, plus tau = 1/2) and
    launch configuration (scaled collision for tau != 1/2), a few steps, every node compared."""
    g, o = run_pair(3, 256, (0.1, 0.1, 0.1), 4, tau=tau, nmodes=8, seed=2)
    assert rel(g, o) < FP64_TOL


def test_fp32dev_d3q19_256cubed_full_size():
    """The benchmark's FP32-deviation form (D3Q19 256^3, tau = 0.8), every node compared."""
    g, o = run_pair(3, 256, (0.1, 0.1, 0.1), 4, tau=0.8, nmodes=8, seed=2, precision="fp32dev")
    assert rel(g, o) < DEV_TOL


def test_fp64_source_field_and_fd_gradient():
    d, n = 2, 24
    rng = np.random.default_rng(5)
    Rf = 0.5 * rng.normal(size=n * n)
    g, o = run_pair(d, n, (0.1, 0.2), 40, R=0.0, Rfield=Rf, explicit_grad=False, seed=4)
    assert relerr(g, o) < FP64_TOL
    g, o = run_pair(d, n, (0.1, 0.2), 40, R=3.0, explicit_grad=False, init_order=1, seed=4)
    assert relerr(g, o) < FP64_TOL


def test_fp64_minimal_grid_and_zero_steps():
    g, o = run_pair(2, 3, (0.1, 0.2), 5, seed=6)
    assert relerr(g, o) < FP64_TOL
    g, o = run_pair(3, 5, (0.1, 0.0, -0.1), 0, seed=6)
    assert relerr(g, o) < FP64_TOL


# ------------------------------------------------------------------------------ FP64, Dirichlet

@pytest.mark.parametrize("bc,u", [("fullway", (0.1, 0.1)), ("fullway", (0.4, 0.4)), ("halfway", (0.01, 0.01))])
def test_fp64_dirichlet_d2q9(bc, u):
    n = 21 if bc == "fullway" else 20
    g, o = run_pair(2, n, u, 60, R=5.0, bc=bc, nmodes=2, seed=7, lin=(0.2, (0.3, -0.4)))
    assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("bc,order", [("fullway", 1), ("fullway", 3), ("halfway", 1), ("halfway", 2), ("halfway", 3)])
def test_fp64_dirichlet_lower_orders(bc, order):
    g, o = run_pair(2, 17, (0.1, -0.05), 30, R=1.0, bc=bc, bc_order=order, nmodes=2, seed=8)
    assert relerr(g, o) < FP64_TOL


def test_fp64_dirichlet_d3q19():
    for bc in ("fullway", "halfway"):
        g, o = run_pair(3, (13, 11, 12) if bc == "halfway" else (13, 11, 12), (0.1, 0.05, -0.08), 30,
                        hi=[13 / 12, 11 / 12, 1.0] if bc == "halfway" else [1.0, 10 / 12, 11 / 12], R=2.0, bc=bc,
                        nmodes=3, seed=9)
        assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("bc,u", [("fullway", (0.05, 0.2, 0.08, 0.1)), ("halfway", (1e-3, 1e-3, 1e-3, 1e-3))])
def test_fp64_dirichlet_d4q33_12(bc, u):
    """Example 3's 4D Dirichlet box on [-1, 1]^4 with phi = sin(pi sum_i (x_i - u_i t)) data, 12^4 nodes."""
    n = 12
    m = O.Model(4, n, -1.0, 1.0, u, bc=bc)
    w = m.wave(a=[1.0], kappa=[[np.pi] * 4], theta=[0.0])
    X = m.coords()
    phi0 = np.sin(np.pi * X.sum(axis=0))
    grad = np.repeat((np.pi * np.cos(np.pi * X.sum(axis=0)))[None, :], 4, axis=0)
    steps = 24
    f = m.step(m.init(phi0, grad, 3), 0, steps, wave=w)
    o = m.phi(f)
    sim = LBM(4, n, -1.0, 1.0, u=u, bc=bc)
    sim.init(_t(phi0), _t(grad))
    sim.set_boundary_wave([1.0], [[np.pi] * 4], [0.0])
    sim.step(steps)
    g = sim.macro().cpu().numpy()
    assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("bc,u", [("fullway", (0.05, 0.2, 0.08, 0.1)), ("halfway", (1e-3, 1e-3, 1e-3, 1e-3))])
def test_fp64_dirichlet_d4q33_64_full_size(bc, u):
    """Example 3's 4D box at the benchmark's size, 64^4 = 16.8 M nodes (2.0 M boundary nodes), in its
    launch configuration (the row kernel with the x_1-face nodes, then the boundary-node kernel), 3
    steps, every node against the oracle (about 18 GB of host memory for the oracle's buffers)."""
    n, steps = 64, 3
    m = O.Model(4, n, -1.0, 1.0, u, bc=bc)
    ssum = np.pi * m.coords().sum(axis=0)
    phi0 = np.sin(ssum)
    grad = np.repeat((np.pi * np.cos(ssum))[None, :], 4, axis=0)
    del ssum
    o = m.phi(m.step(m.init(phi0, grad, 3), 0, steps, wave=m.wave(a=[1.0], kappa=[[np.pi] * 4], theta=[0.0])))
    sim = LBM(4, n, -1.0, 1.0, u=u, bc=bc)
    sim.init(_t(phi0), _t(grad))
    sim.set_boundary_wave([1.0], [[np.pi] * 4], [0.0])
    sim.step(steps)
    g = sim.macro().cpu().numpy()
    sim.close()
    assert relerr(g, o) < FP64_TOL


@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_d5q51_24_full_size(precision):
    """The precision workload's D5Q51 box at its size, 24^5 = 8.0 M nodes, u = (0.02, .., 0.1),
    tau = 1/2, seeded modes, 3 steps, every node against the oracle."""
    g, o = run_pair(5, 24, (0.02, 0.04, 0.06, 0.08, 0.1), 3, tau=0.5, nmodes=8, seed=5, precision=precision)
    assert rel(g, o) < (FP64_TOL if precision == "fp64" else DEV_TOL)


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
@pytest.mark.parametrize("d,n,u,tau", [
    (1, (23,), (0.3,), 0.5), (1, (16,), (0.1,), 0.8),
    (2, (3, 17), (0.1, 0.05), 0.8), (3, (9, 6, 7), (0.1, -0.05, 0.08), 1.2),
    (5, (5, 4, 6, 5, 4), (0.02, 0.04, 0.06, 0.08, 0.1), 0.5), (5, (4, 5, 4, 4, 5), (0.01,) * 5, 0.8)])
def test_fp64_dirichlet_all_dimensions(bc, d, n, u, tau):
    """Both Dirichlet schemes in d = 1..5 on ragged boxes (including rows of 3 nodes), with the
    s = 2 and the general collision: the x_1-face nodes go through the interior-row kernel, the
    other boundary nodes through the boundary-node kernel."""
    h = 1.0 / 16
    hi = [(ni - 1) * h if bc == "fullway" else ni * h for ni in n]
    g, o = run_pair(d, n, u, 20, hi=hi, tau=tau, R=0.6, bc=bc, nmodes=2, seed=31 + d)
    assert rel(g, o) < FP64_TOL


@pytest.mark.parametrize("precision,tol", [("fp64", FP64_TOL), ("fp32dev", DEV_TOL)])
@pytest.mark.parametrize("bc", ["periodic", "fullway", "halfway"])
@pytest.mark.parametrize("tau,u,R", [(1.0, (0.1, -0.05, 0.08), 0.0), (1.0, (0.1, -0.05, 0.08), 0.7),
                                     (0.5, (0.0, 0.0, 0.0), 0.7), (1.0, (0.0, 0.0, 0.0), 0.0),
                                     (1.7, (0.05, 0.02, -0.03), 0.3)])
def test_degenerate_relaxation_and_velocity(precision, tol, bc, tau, u, R):
    """The method's degenerate cases on a ragged D3Q19 box: tau = 1 (s = 1: the collision keeps
    nothing of the pre-collision populations, f* = omega phi + dt omega R; the scaled FP64 state,
    which stores (1 - s)^-j f*, does not apply), u = 0 (no transport: with the s = 2 collision phi
    changes by the source alone), and tau > 1 (s < 1), each with and without a source."""
    n = (9, 8, 7)
    h = 1.0 / 16
    hi = [(ni - 1) * h if bc == "fullway" else ni * h for ni in n]
    g, o = run_pair(3, n, u, 25, hi=hi, tau=tau, R=R, bc=bc, precision=precision, nmodes=3, seed=41)
    assert rel(g, o) < tol


# ------------------------------------------------------------------------------ FP32 deviations

def test_fp32dev_d3q19_periodic():
    g, o = run_pair(3, 32, (0.1, 0.1, 0.1), 300, precision="fp32dev", nmodes=8, seed=10)
    assert relerr(g, o) < DEV_TOL


@pytest.mark.parametrize("tau", [0.5, 0.8])
def test_fp32dev_all_dimensions(tau):
    for d, n in ((1, (40,)), (2, (24, 20)), (4, (8, 7, 6, 5)), (5, (6, 5, 4, 5, 6))):
        u = [0.02, 0.04, 0.06, 0.08, 0.1][:d]
        g, o = run_pair(d, n, u, 60 if tau == 0.5 else 12, hi=[ni / 16.0 for ni in n], tau=tau,
                        precision="fp32dev", nmodes=3, seed=11)
        assert rel(g, o) < DEV_TOL, d


def test_fp32dev_source_field():
    rng = np.random.default_rng(12)
    Rf = 0.3 * rng.normal(size=32 * 32)
    g, o = run_pair(2, 32, (0.1, 0.2), 80, Rfield=Rf, precision="fp32dev", explicit_grad=False, seed=12)
    assert relerr(g, o) < DEV_TOL


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
def test_fp32dev_dirichlet(bc):
    n = 21 if bc == "fullway" else 20
    g, o = run_pair(2, n, (0.1, 0.1) if bc == "fullway" else (0.01, 0.01), 60, R=5.0, bc=bc, precision="fp32dev",
                    nmodes=2, seed=13)
    assert relerr(g, o) < DEV_TOL


# ------------------------------------------------------------------------------ diagnostics / state

@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
@pytest.mark.parametrize("tau", [0.5, 0.8])
def test_diagnostics_match_the_oracle(precision, tau):
    g, o, sim, m, f = run_pair(2, 16, (0.1, 0.2), 25, tau=tau, R=0.7, precision=precision, seed=14,
                               return_models=True)
    dg = sim.diagnostics()
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert dg["ok"] and dg["nonfinite"] == 0
    assert abs(dg["mass"] - o.sum()) < tol * max(1.0, np.abs(o).sum())
    assert abs(dg["entropy"] - m.entropy(f)) < tol * m.entropy(f)
    assert abs(dg["max_abs"] - np.max(np.abs(o))) < tol * np.max(np.abs(o))
    sim.close()


def test_state_roundtrip_and_restart():
    _, _, sim, m, f = run_pair(3, 12, (0.1, 0.0, 0.05), 7, seed=15, return_models=True)
    buf = sim.get_state()
    sim.step(5)
    a = sim.macro().cpu().numpy()
    sim.set_state(buf, 7)
    assert sim.step_index == 7
    sim.step(5)
    b = sim.macro().cpu().numpy()
    assert np.array_equal(a, b)
    sim.close()


def test_error_paths():
    import torch

    sim = LBM(2, 8, u=(0.1, 0.1))
    with pytest.raises(LHEError) as ei:
        sim.step(1)
    assert ei.value.status == _abi.ERR_STATE
    phi = torch.zeros(64, dtype=torch.float64, device="cuda")
    phi[3] = float("nan")
    sim.init(phi, torch.zeros(128, dtype=torch.float64, device="cuda"))
    sim.step(2)
    dg = sim.diagnostics()
    assert not dg["ok"] and dg["nonfinite"] > 0
    sim.close()
    with pytest.raises(LHEError) as ei:
        LBM(4, 6, u=(0.4, 0.4, 0.4, 0.4))
    assert ei.value.status == _abi.ERR_UNSTABLE
    dsim = LBM(2, 9, u=(0.1, 0.1), bc="fullway")
    with pytest.raises(LHEError) as ei:
        dsim.init(torch.zeros(81, dtype=torch.float64, device="cuda"), None)
    assert ei.value.status == _abi.ERR_ARG
    dsim.init(torch.zeros(81, dtype=torch.float64, device="cuda"), torch.zeros(162, dtype=torch.float64, device="cuda"))
    with pytest.raises(LHEError) as ei:
        dsim.step(1)  # no boundary data
    assert ei.value.status == _abi.ERR_STATE
    dsim.close()
