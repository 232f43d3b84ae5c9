"""GPU: Dirichlet data given as jets of phi (lhe_lbm_boundary_points, lhe_lbm_set_boundary_jet).

The library forms the unknown populations of Eq. (bun1) / the B_k of Eq. (bun2) from the caller's
jets; the oracle forms them from the same jets with its own directional derivatives
(Model.step_jets). Data: a Gaussian pulse, an exact solution of Eq. (HE) that the sine family of
lhe_lbm_set_boundary_wave cannot express, and the jets of that family, which must reproduce the
library's wave path. FP64 1e-13, FP32-deviation 1e-5 (relative max-norm)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import LBM, LHEError, build, jet_len, workloads as W
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _pulse(d):
    return dict(A=1.0, xc=[0.45, 0.55, 0.5, 0.48, 0.52][:d], sigma=0.2)


def _run_jets(sim, steps, jet_fn):
    pts, toff = sim.boundary_points()
    for _ in range(steps):
        t = sim.step_index * sim.dt + toff
        sim.set_boundary_jet(_t(jet_fn(pts, t)))
        sim.step(1)


@pytest.mark.parametrize("d,n,bc,order,tau", [
    (2, 17, "fullway", 4, 0.5), (2, 17, "fullway", 3, 0.8), (2, 17, "fullway", 1, 0.5),
    (2, 16, "halfway", 4, 0.5), (2, 16, "halfway", 3, 0.8), (2, 16, "halfway", 2, 0.5), (2, 16, "halfway", 1, 1.2),
    (3, 9, "fullway", 4, 0.5), (3, 8, "halfway", 4, 0.8), (4, 6, "fullway", 4, 0.5), (4, 6, "halfway", 4, 0.5)])
@pytest.mark.parametrize("precision", ["fp64", "fp32dev"])
def test_pulse_jets_match_the_oracle(d, n, bc, order, tau, precision):
    u = [0.1, 0.05, -0.08, 0.06][:d] if bc == "fullway" else [0.01, 0.02, -0.01, 0.015][:d]
    R, steps = 0.5, 12
    pk = _pulse(d)
    hi = 1.0
    m = O.Model(d, n, 0.0, hi, u, tau=tau, R=R, bc=bc, bc_order=order)
    X = m.coords()
    phi0 = W.gaussian_value(X, 0.0, u, R, **pk)
    grad = W.gaussian_grad(X, 0.0, u, **pk)
    jets = lambda P, t: W.gaussian_jets(P, t, u, R, **pk)
    ref = m.phi(m.step_jets(m.init(phi0, grad, 3), 0, steps, jets))
    sim = LBM(d, n, 0.0, hi, u=u, tau=tau, R=R, bc=bc, bc_order=order, precision=precision)
    sim.init(_t(phi0), _t(grad))
    _run_jets(sim, steps, jets)
    got = sim.macro().cpu().numpy()
    sim.close()
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("bc,order", [("fullway", 4), ("fullway", 3), ("halfway", 4), ("halfway", 2)])
@pytest.mark.parametrize("d", [2, 3, 5])
def test_jets_of_the_wave_family_match_the_wave_path(d, bc, order):
    n = {2: 14, 3: 8, 5: 5}[d] + (1 if bc == "fullway" else 0)
    u = [0.02, 0.04, 0.06, 0.08, 0.1][:d] if bc == "fullway" else [0.01, 0.02, 0.01, 0.02, 0.01][:d]
    R = 0.4
    F = W.fourier_field(d, 2, 60 + d, 0.0, 1.0)
    a, kap, th = F.wave_params()
    res = []
    for mode in ("wave", "jets"):
        sim = LBM(d, n, 0.0, 1.0, u=u, R=R, bc=bc, bc_order=order)
        X = W.node_coords(d, [n] * d, 0.0, sim.dx, halfway=(bc == "halfway"))
        sim.init(_t(F.value(X)), _t(F.grad(X)))
        if mode == "wave":
            sim.set_boundary_wave(a, kap, th)
            for _ in range(9):
                sim.step(1)
        else:
            _run_jets(sim, 9, lambda P, t: W.wave_jets(P, t, u, R, a, kap, th))
        res.append(sim.macro().cpu().numpy())
        sim.close()
    assert np.max(np.abs(res[0] - res[1])) < 1e-13 * np.max(np.abs(res[0]))


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
def test_boundary_points(bc):
    d, n = 3, (7, 5, 6)
    h = 1.0 / 8
    hi = [(ni - 1) * h if bc == "fullway" else ni * h for ni in n]
    sim = LBM(d, list(n), 0.0, hi, u=(0.01, 0.02, 0.01), bc=bc)
    pts, toff = sim.boundary_points()
    X = W.node_coords(d, list(n), 0.0, sim.dx, halfway=(bc == "halfway"))
    idx = np.stack(np.unravel_index(np.arange(int(np.prod(n))), n[::-1])[::-1])
    expect = []
    for site in range(X.shape[1]):
        for k, e in enumerate(sim.e):
            src = idx[:, site] - np.asarray(e)
            if np.any(src < 0) or np.any(src >= np.asarray(n)):
                expect.append(tuple(np.round(X[:, site] if bc == "fullway" else X[:, site] - 0.5 * sim.dx * np.asarray(e), 12)))
    if bc == "fullway":
        expect = sorted(set(expect))
        assert toff == sim.dt and len(pts) == sim.n_boundary
    else:
        expect = sorted(expect)
        assert toff == 0.0
    assert sorted(tuple(np.round(p, 12)) for p in pts) == expect
    sim.close()


def test_jet_error_paths():
    d, n = 2, 9
    sim = LBM(d, n, 0.0, 1.0, u=(0.1, 0.05), bc="fullway")
    X = W.node_coords(d, [n] * d, 0.0, sim.dx)
    pk = _pulse(d)
    sim.init(_t(W.gaussian_value(X, 0.0, (0.1, 0.05), 0.0, **pk)), _t(W.gaussian_grad(X, 0.0, (0.1, 0.05), **pk)))
    pts, toff = sim.boundary_points()
    jet = _t(W.gaussian_jets(pts, toff, (0.1, 0.05), 0.0, **pk))
    sim.set_boundary_jet(jet)
    with pytest.raises(LHEError) as ei:
        sim.step(2)
    assert ei.value.status == _abi.ERR_STATE
    sim.step(1)
    with pytest.raises(LHEError) as ei:
        sim.step(1)  # the jets served the previous step
    assert ei.value.status == _abi.ERR_STATE
    sim.set_boundary_wave([1.0], [[1.0, 2.0]], [0.0])  # back to the exact-solution family
    sim.step(3)
    with pytest.raises(ValueError):
        sim.set_boundary_jet(_t(np.zeros(3)))
    assert jet_len(2) == 20
    sim.close()
    per = LBM(d, n, u=(0.1, 0.05))
    with pytest.raises(LHEError) as ei:
        per.boundary_points()
    assert ei.value.status == _abi.ERR_STATE
    per.close()
