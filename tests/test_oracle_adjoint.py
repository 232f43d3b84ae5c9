"""Pins of the oracle's discrete adjoint (periodic box): transpose identities and finite differences.

The forward map (phi0, R) -> phi(T) is affine, so L = 1/2 |phi(T) - target|^2 is quadratic and a
central difference is exact up to rounding for any step size."""
import numpy as np
import pytest

from oracle import oracle as O


def _model(d=2, n=5, tau=0.5):
    u = {1: (0.2,), 2: (0.1, -0.2), 3: (0.1, 0.05, -0.15)}[d]
    return O.Model(d, n, 0.0, 1.0, u, tau=tau)


@pytest.mark.parametrize("tau", [0.5, 0.8])
@pytest.mark.parametrize("d", [1, 2, 3])
def test_adjoint_step_is_the_transpose_of_the_step(d, tau):
    m = _model(d, 4 if d == 3 else 5, tau)
    rng = np.random.default_rng(20 + d)
    x = rng.normal(size=(m.Q, m.S))
    y = rng.normal(size=(m.Q, m.S))
    lhs = np.vdot(m.step(x), y)               # R = 0: the step is linear
    rhs = np.vdot(x, m.adjoint_step(y))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_dense_step_matrix_transpose():
    m = _model(2, 3)
    N = m.Q * m.S
    A = np.zeros((N, N))
    B = np.zeros((N, N))
    for j in range(N):
        v = np.zeros(N)
        v[j] = 1.0
        A[:, j] = m.step(v.reshape(m.Q, m.S)).ravel()
        B[:, j] = m.adjoint_step(v.reshape(m.Q, m.S)).ravel()
    assert np.max(np.abs(A.T - B)) < 1e-15
    # the step is a permutation composed with a per-site collision: exactly Q nonzeros per site column
    assert np.count_nonzero(np.abs(A) > 0) <= N * m.Q


def _loss(m, phi0, R, target, T, order=3, grad=None):
    f = m.init(phi0, grad, order)
    for n in range(T):
        f = m.step(f, n0=n, nsteps=1, Rfield=R)
    r = m.phi(f) - target
    return 0.5 * float(r @ r)


@pytest.mark.parametrize("order,explicit_grad", [(3, False), (3, True), (1, False)])
def test_gradient_matches_central_differences(order, explicit_grad):
    m = _model(2, 6)
    rng = np.random.default_rng(31)
    phi0 = rng.normal(size=m.S)
    R = 0.3 * rng.normal(size=m.S)
    target = rng.normal(size=m.S)
    grad = rng.normal(size=(2, m.S)) if explicit_grad else None
    T = 7
    loss, gphi0, gR, ggrad = m.gradient(phi0, R, target, T, order=order, grad=grad)
    assert abs(loss - _loss(m, phi0, R, target, T, order, grad)) < 1e-12 * loss
    for trial in range(4):
        vp, vR = rng.normal(size=m.S), rng.normal(size=m.S)
        vg = rng.normal(size=(2, m.S)) if explicit_grad else None
        h = 10.0 ** (-1 - trial)
        gp = None if grad is None else grad + h * vg
        gm = None if grad is None else grad - h * vg
        fd = (_loss(m, phi0 + h * vp, R + h * vR, target, T, order, gp) -
              _loss(m, phi0 - h * vp, R - h * vR, target, T, order, gm)) / (2 * h)
        an = gphi0 @ vp + gR @ vR + (0.0 if vg is None else float(np.sum(ggrad * vg)))
        assert abs(fd - an) < 1e-9 * max(1.0, abs(an)), (fd, an, h)


def test_gradient_dense_jacobian_on_a_tiny_grid():
    """d phi(T)/d phi0 built column by column from the forward oracle, contracted with the residual."""
    m = _model(2, 3)
    rng = np.random.default_rng(41)
    phi0 = rng.normal(size=m.S)
    R = rng.normal(size=m.S)
    target = rng.normal(size=m.S)
    T = 4

    def phiT(p, r):
        f = m.init(p, None, 3)
        for n in range(T):
            f = m.step(f, n0=n, nsteps=1, Rfield=r)
        return m.phi(f)

    base = phiT(np.zeros(m.S), np.zeros(m.S))
    J0 = np.stack([phiT(np.eye(m.S)[j], np.zeros(m.S)) - base for j in range(m.S)], axis=1)
    JR = np.stack([phiT(np.zeros(m.S), np.eye(m.S)[j]) - base for j in range(m.S)], axis=1)
    res = J0 @ phi0 + JR @ R + base - target
    _, gphi0, gR, _ = m.gradient(phi0, R, target, T)
    assert np.max(np.abs(gphi0 - J0.T @ res)) < 1e-12
    assert np.max(np.abs(gR - JR.T @ res)) < 1e-12


# ---------------------------------------------------------------- Dirichlet boxes

def _dmodel(bc, d=2, n=5, tau=0.5, order=4):
    u = {2: (0.1, -0.2), 3: (0.1, 0.05, -0.15)}[d]
    return O.Model(d, n, 0.0, 1.0, u, tau=tau, R=0.7, bc=bc, bc_order=order)


def _dwave(m):
    if m.d == 2:
        return m.wave(a=[1.0, 0.5], kappa=[(np.pi, np.pi), (2.0, -1.0)], theta=[0.3, 1.1], b=0.2)
    return m.wave(a=[0.8], kappa=[(np.pi, 1.0, -2.0)], theta=[0.4], b=-0.1)


@pytest.mark.parametrize("tau", [0.5, 0.8])
@pytest.mark.parametrize("bc,d,n", [("fullway", 2, 5), ("halfway", 2, 5), ("fullway", 3, 4), ("halfway", 3, 4)])
def test_dirichlet_adjoint_step_is_the_transpose(bc, d, n, tau):
    """The Dirichlet step is affine in the state (the boundary data enter additively): its linear
    part step(x) - step(0) and the adjoint step are transposes."""
    m = _dmodel(bc, d, n, tau)
    w = _dwave(m)
    rng = np.random.default_rng(60 + d)
    x = rng.normal(size=(m.Q, m.S))
    y = rng.normal(size=(m.Q, m.S))
    zero = np.zeros_like(x)
    lin = m.step(x, 0, 1, wave=w) - m.step(zero, 0, 1, wave=w)
    lhs = np.vdot(lin, y)
    rhs = np.vdot(x, m.adjoint_step(y))
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
def test_dirichlet_dense_step_matrix_transpose(bc):
    m = _dmodel(bc, 2, 3)
    w = _dwave(m)
    N = m.Q * m.S
    base = m.step(np.zeros((m.Q, m.S)), 0, 1, wave=w).ravel()
    A = np.zeros((N, N))
    B = np.zeros((N, N))
    for j in range(N):
        v = np.zeros(N)
        v[j] = 1.0
        A[:, j] = m.step(v.reshape(m.Q, m.S), 0, 1, wave=w).ravel() - base
        B[:, j] = m.adjoint_step(v.reshape(m.Q, m.S)).ravel()
    assert np.max(np.abs(A.T - B)) < 1e-14
    if bc == "halfway":  # the -f*_kbar coupling makes some columns feed two entries at one node
        assert np.count_nonzero(np.abs(A) > 0) > 0


def _dloss(m, w, phi0, grad, target, T, order=3):
    f = m.init(phi0, grad, order)
    f = m.step(f, 0, T, wave=w)
    r = m.phi(f) - target
    return 0.5 * float(r @ r)


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
@pytest.mark.parametrize("tau", [0.5, 0.8])
def test_dirichlet_gradient_matches_central_differences(bc, tau):
    m = _dmodel(bc, 2, 6, tau)
    w = _dwave(m)
    rng = np.random.default_rng(71)
    phi0 = rng.normal(size=m.S)
    grad = rng.normal(size=(2, m.S))
    target = rng.normal(size=m.S)
    T = 9
    loss, gphi0, _, ggrad = m.gradient(phi0, None, target, T, order=3, grad=grad, wave=w)
    assert abs(loss - _dloss(m, w, phi0, grad, target, T)) < 1e-12 * loss
    for trial in range(4):
        vp, vg = rng.normal(size=m.S), rng.normal(size=(2, m.S))
        h = 10.0 ** (-1 - trial)
        fd = (_dloss(m, w, phi0 + h * vp, grad + h * vg, target, T) -
              _dloss(m, w, phi0 - h * vp, grad - h * vg, target, T)) / (2 * h)
        an = gphi0 @ vp + float(np.sum(ggrad * vg))
        assert abs(fd - an) < 1e-9 * max(1.0, abs(an)), (fd, an, h)
