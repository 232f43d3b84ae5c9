"""GPU adjoint: gradients of L = 1/2 |phi(T) - target|^2 w.r.t. phi0 and R(x) from the CUDA adjoint
kernels, against the oracle's discrete adjoint and against central finite differences (exact up to
rounding: L is quadratic in (phi0, R))."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import LBM, build, workloads as W
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


def gpu_gradient(sim, phi0, R, target, T, grad=None):
    sim.init(_t(phi0), None if grad is None else _t(grad), _t(R))
    sim.step(T)
    r = sim.macro() - _t(target)
    loss = 0.5 * float((r * r).sum())
    sim.adjoint_seed(r.contiguous())
    sim.adjoint_step(T)
    gphi, ggrad, gR = sim.adjoint_grads(want_grad=grad is not None, want_R=True)
    return loss, gphi.cpu().numpy(), None if ggrad is None else ggrad.cpu().numpy().reshape(-1), gR.cpu().numpy()


def _problem(d, n, seed):
    rng = np.random.default_rng(seed)
    S = n ** d
    return rng.normal(size=S), 0.3 * rng.normal(size=S), rng.normal(size=S)


@pytest.mark.parametrize("tau", [0.5, 0.8])
@pytest.mark.parametrize("d,n,u", [(2, 8, (0.1, -0.2)), (3, 6, (0.1, 0.05, -0.15)), (1, 12, (0.3,)),
                                   (4, 5, (0.05, 0.1, 0.08, 0.1)), (5, 4, (0.02, 0.04, 0.06, 0.08, 0.1))])
@pytest.mark.parametrize("order,explicit", [(3, False), (3, True), (1, False)])
def test_fp64_adjoint_matches_the_oracle(d, n, u, tau, order, explicit):
    phi0, R, target = _problem(d, n, 40 + d)
    T = 9
    m = O.Model(d, n, 0.0, 1.0, u, tau=tau)
    grad = np.random.default_rng(7).normal(size=(d, n ** d)) if explicit else None
    loss_o, gphi_o, gR_o, ggrad_o = m.gradient(phi0, R, target, T, order=order, grad=grad)
    sim = LBM(d, n, u=u, tau=tau, init_order=order)
    loss_g, gphi_g, ggrad_g, gR_g = gpu_gradient(sim, phi0, R, target, T, grad)
    sim.close()
    assert abs(loss_g - loss_o) < 1e-12 * loss_o
    assert np.max(np.abs(gphi_g - gphi_o)) < 1e-12 * np.max(np.abs(gphi_o))
    assert np.max(np.abs(gR_g - gR_o)) < 1e-12 * np.max(np.abs(gR_o))
    if explicit and order == 3:
        assert np.max(np.abs(ggrad_g - ggrad_o.ravel())) < 1e-12 * np.max(np.abs(ggrad_o))


@pytest.mark.parametrize("d,n", [(2, 16), (3, 8), (5, 4)])
def test_fp32dev_adjoint_matches_the_oracle(d, n):
    rng = np.random.default_rng(50 + d)
    u = [0.1, -0.05, 0.08, 0.03, -0.02][:d]
    m = O.Model(d, n, 0.0, 1.0, u)
    F = W.fourier_field(d, 3, 60 + d)
    X = m.coords()
    phi0 = F.value(X)
    R = 0.1 * W.fourier_field(d, 2, 70 + d).value(X)
    target = W.fourier_field(d, 4, 80 + d).value(X)
    T = 12
    loss_o, gphi_o, gR_o, _ = m.gradient(phi0, R, target, T)
    sim = LBM(d, n, u=u, precision="fp32dev")
    loss_g, gphi_g, _, gR_g = gpu_gradient(sim, phi0, R, target, T)
    sim.close()
    assert abs(loss_g - loss_o) < 1e-5 * loss_o
    assert np.max(np.abs(gphi_g - gphi_o)) < 1e-5 * np.max(np.abs(gphi_o))
    assert np.max(np.abs(gR_g - gR_o)) < 1e-5 * np.max(np.abs(gR_o))


def test_fp64_adjoint_central_differences_16cubed():
    """The differentiation workload's FD check on its 16^3 copy: 16 seeded directions in FP64."""
    d, n, T = 3, 16, 64
    u = (0.1, 0.1, 0.1)
    X = W.node_coords(d, n, 0.0, 1.0 / n)
    phi0 = W.fourier_field(d, 8, 90).value(X)
    R = 0.1 * W.fourier_field(d, 4, 91).value(X)
    target = W.fourier_field(d, 8, 92).value(X)
    sim = LBM(d, n, u=u)
    loss, gphi, _, gR = gpu_gradient(sim, phi0, R, target, T)

    def L(p, r):
        sim.init(_t(p), None, _t(r))
        sim.step(T)
        res = sim.macro() - _t(target)
        return 0.5 * float((res * res).sum())

    rng = np.random.default_rng(93)
    for j in range(16):
        vp, vR = rng.normal(size=n ** d), rng.normal(size=n ** d)
        h = 1e-3
        fd = (L(phi0 + h * vp, R + h * vR) - L(phi0 - h * vp, R - h * vR)) / (2 * h)
        an = gphi @ vp + gR @ vR
        assert abs(fd - an) <= 1e-6 * abs(an), (j, fd, an)
    sim.close()


def test_autograd_function():
    import torch

    from paper_2410_13165_gb300.autograd import lbm_loss

    d, n, T = 2, 10, 15
    rng = np.random.default_rng(100)
    phi0 = _t(rng.normal(size=n * n)).requires_grad_(True)
    R = _t(0.2 * rng.normal(size=n * n)).requires_grad_(True)
    target = _t(rng.normal(size=n * n))
    sim = LBM(d, n, u=(0.1, 0.2))
    loss = lbm_loss(phi0, R, sim, T, target)
    loss.backward()
    m = O.Model(d, n, 0.0, 1.0, (0.1, 0.2))
    lo, gphi_o, gR_o, _ = m.gradient(phi0.detach().cpu().numpy(), R.detach().cpu().numpy(),
                                     target.cpu().numpy(), T)
    assert abs(float(loss.detach()) - lo) < 1e-12 * lo
    assert np.max(np.abs(phi0.grad.cpu().numpy() - gphi_o)) < 1e-12 * np.max(np.abs(gphi_o))
    assert np.max(np.abs(R.grad.cpu().numpy() - gR_o)) < 1e-12 * np.max(np.abs(gR_o))
    sim.close()


# ------------------------------------------------------------------ Dirichlet boxes (FP64)

def _dirichlet_case(d, bc):
    n = {2: 8, 3: 6}[d]
    u = {2: (0.1, -0.2), 3: (0.1, 0.05, -0.15)}[d]
    wave = (dict(a=[1.0, 0.5], kappa=[(np.pi, np.pi), (2.0, -1.0)], theta=[0.3, 1.1], b=0.2) if d == 2 else
            dict(a=[0.8], kappa=[(np.pi, 1.0, -2.0)], theta=[0.4], b=-0.1))
    return n, u, wave


def _dirichlet_gpu(d, n, u, tau, bc, wave, phi0, grad, target, T, R=0.7, precision="fp64"):
    sim = LBM(d, n, u=u, tau=tau, R=R, bc=bc, precision=precision)
    sim.init(_t(phi0), _t(grad))
    sim.set_boundary_wave(wave["a"], wave["kappa"], wave["theta"], wave["b"])
    sim.step(T)
    r = sim.macro() - _t(target)
    loss = 0.5 * float((r * r).sum())
    sim.adjoint_seed(r.contiguous())
    sim.adjoint_step(T)
    gphi, ggrad, _ = sim.adjoint_grads(want_grad=True, want_R=False)
    sim.close()
    return loss, gphi.cpu().numpy(), ggrad.cpu().numpy().reshape(-1)


@pytest.mark.parametrize("tau", [0.5, 0.8])
@pytest.mark.parametrize("bc", ["fullway", "halfway"])
@pytest.mark.parametrize("d", [2, 3])
def test_fp64_dirichlet_adjoint_matches_the_oracle(d, bc, tau):
    n, u, wave = _dirichlet_case(d, bc)
    rng = np.random.default_rng(80 + d)
    S = n ** d
    phi0, grad, target = rng.normal(size=S), rng.normal(size=(d, S)), rng.normal(size=S)
    T = 9
    m = O.Model(d, n, 0.0, 1.0, u, tau=tau, R=0.7, bc=bc)
    w = m.wave(**wave)
    loss_o, gphi_o, _, ggrad_o = m.gradient(phi0, None, target, T, order=3, grad=grad, wave=w)
    loss_g, gphi_g, ggrad_g = _dirichlet_gpu(d, n, u, tau, bc, wave, phi0, grad, target, T)
    assert abs(loss_g - loss_o) < 1e-12 * loss_o
    assert np.max(np.abs(gphi_g - gphi_o)) < 1e-12 * np.max(np.abs(gphi_o))
    assert np.max(np.abs(ggrad_g - ggrad_o.ravel())) < 1e-12 * np.max(np.abs(ggrad_o))


@pytest.mark.parametrize("tau", [0.5, 0.8])
@pytest.mark.parametrize("bc", ["fullway", "halfway"])
@pytest.mark.parametrize("d", [2, 3])
def test_fp32dev_dirichlet_adjoint_matches_the_oracle(d, bc, tau):
    """The FP32-deviation forward and adjoint of a Dirichlet box (boundary adjoint in the deviation
    form) against the oracle's FP64 discrete adjoint: loss and gradients within 1e-5."""
    n, u, wave = _dirichlet_case(d, bc)
    rng = np.random.default_rng(180 + d)
    S = n ** d
    phi0, grad, target = rng.normal(size=S), rng.normal(size=(d, S)), rng.normal(size=S)
    T = 9
    m = O.Model(d, n, 0.0, 1.0, u, tau=tau, R=0.7, bc=bc)
    loss_o, gphi_o, _, ggrad_o = m.gradient(phi0, None, target, T, order=3, grad=grad, wave=m.wave(**wave))
    loss_g, gphi_g, ggrad_g = _dirichlet_gpu(d, n, u, tau, bc, wave, phi0, grad, target, T, precision="fp32dev")
    assert abs(loss_g - loss_o) < 1e-5 * loss_o
    assert np.max(np.abs(gphi_g - gphi_o)) < 1e-5 * np.max(np.abs(gphi_o))
    assert np.max(np.abs(ggrad_g - ggrad_o.ravel())) < 1e-5 * np.max(np.abs(ggrad_o))


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
def test_fp64_dirichlet_gradient_central_differences(bc):
    """The loss is quadratic in (phi0, grad phi0): central differences of the library's own forward
    runs equal the adjoint gradient up to rounding (16x16 box, 40 steps, 8 random directions)."""
    d, n, T = 2, 16, 40
    u = (0.1, -0.2) if bc == "fullway" else (0.01, 0.02)
    wave = dict(a=[1.0, 0.5], kappa=[(np.pi, np.pi), (2.0, -1.0)], theta=[0.3, 1.1], b=0.2)
    rng = np.random.default_rng(90)
    S = n * n
    phi0, grad, target = rng.normal(size=S), rng.normal(size=(d, S)), rng.normal(size=S)
    _, gphi, ggrad = _dirichlet_gpu(d, n, u, 0.5, bc, wave, phi0, grad, target, T)

    def loss(p, g):
        sim = LBM(d, n, u=u, R=0.7, bc=bc)
        sim.init(_t(p), _t(g))
        sim.set_boundary_wave(wave["a"], wave["kappa"], wave["theta"], wave["b"])
        sim.step(T)
        r = sim.macro().cpu().numpy() - target
        sim.close()
        return 0.5 * float(r @ r)

    for trial in range(8):
        vp, vg = rng.normal(size=S), rng.normal(size=(d, S))
        h = 1e-3
        fd = (loss(phi0 + h * vp, grad + h * vg) - loss(phi0 - h * vp, grad - h * vg)) / (2 * h)
        an = gphi @ vp + float(ggrad @ vg.ravel())
        assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_dirichlet_adjoint_error_paths():
    from paper_2410_13165_gb300 import LHEError

    n, u, wave = _dirichlet_case(2, "fullway")
    sim = LBM(2, n, u=u, bc="fullway")
    sim.init(_t(np.zeros(n * n)), _t(np.zeros((2, n * n))))
    sim.adjoint_seed(_t(np.ones(n * n)))
    sim.adjoint_step(2)
    with pytest.raises(LHEError) as ei:
        sim.adjoint_grads(want_R=True)
    assert ei.value.status == _abi.ERR_ARG
    sim.close()
