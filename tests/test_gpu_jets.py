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


def _source_run(sim, m, X, u, steps, Rt):
    """Steps with the source R(x, t_{n+1}) of each step's collision set first, then the jets."""
    for n in range(steps):
        sim.set_source(_t(Rt(n + 1)))
        pts, toff = sim.boundary_points()
        sim.set_boundary_jet(_t(W.sine_product_jets(pts, sim.step_index * sim.dt + toff)))
        sim.step(1)


@pytest.mark.parametrize("d,n,bc,precision", [(2, 17, "fullway", "fp64"), (2, 16, "halfway", "fp64"),
                                              (3, 9, "fullway", "fp64"), (2, 17, "fullway", "fp32dev"),
                                              (3, 8, "halfway", "fp32dev")])
def test_time_varying_source_on_dirichlet_boxes(d, n, bc, precision):
    """The manufactured solution prod_i sin(pi x_i) exp(-t) with its source R(x, t) set before each
    step and boundary data as jets, against the oracle with the same sources and jets."""
    u = [0.1, 0.05, -0.08][:d] if bc == "fullway" else [0.01, 0.02, -0.01][:d]
    steps = 10
    m = O.Model(d, n, -1.0, 1.0, u, bc=bc)
    X = m.coords()
    phi0, grad = W.sine_product_value(X, 0.0), W.sine_product_grad(X, 0.0)
    Rt = lambda k: W.sine_product_source(X, k * m.dt, u)  # R(x, t_k), the source of the collision at t_k
    ref = m.phi(m.step_jets(m.init(phi0, grad, 3), 0, steps, lambda P, t: W.sine_product_jets(P, t), Rfield_fn=Rt))
    sim = LBM(d, n, -1.0, 1.0, u=u, bc=bc, precision=precision)
    sim.init(_t(phi0), _t(grad), _t(Rt(0)))
    _source_run(sim, m, X, u, steps, Rt)
    got = sim.macro().cpu().numpy()
    sim.close()
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("d,n,tau,precision", [(2, 24, 0.5, "fp64"), (2, 24, 0.8, "fp64"), (3, 16, 0.8, "fp32dev")])
def test_time_varying_source_on_periodic_boxes(d, n, tau, precision):
    """A source changed before every step (periodic: the FP64 kernel in both collision forms, the
    staged FP32-deviation kernel of D3Q19), against the oracle; macro between steps, after the next
    source is set, still reports phi of the last collision."""
    u = [0.1, 0.05, -0.08][:d]
    F = W.fourier_field(d, 3, 80 + d, 0.0, 1.0)
    m = O.Model(d, n, 0.0, 1.0, u, tau=tau)
    X = m.coords()
    src = lambda k: 0.3 * np.cos(np.pi * k * m.dt + X[0]) * np.sin(2 * np.pi * X[-1])
    f = m.init(F.value(X), F.grad(X), 3)
    sim = LBM(d, n, u=u, tau=tau, precision=precision)
    sim.init(_t(F.value(X)), _t(F.grad(X)), _t(src(0)))  # the source of the collision at t_0
    tol = 1e-13 if precision == "fp64" else 1e-5
    for k in range(8):
        f = m.step(f, k, 1, Rfield=src(k))  # the oracle collides at t_k, then streams
        sim.set_source(_t(src(k + 1)))      # the library streams, then collides at t_{k+1}
        sim.step(1)
        sim.set_source(_t(src(k + 2)))      # set ahead of the next step: macro must not use it
        ref = m.phi(f)
        assert np.max(np.abs(sim.macro().cpu().numpy() - ref)) < tol * np.max(np.abs(ref)), k
    sim.set_source(None)                    # the collisions at t_9, t_10 take the constant R (0)
    f = m.step(f, 8, 1, Rfield=src(8))      # oracle: collision at t_8 (the library's was at step 8)
    f = m.step(f, 9, 1)                     # and at t_9 with the constant source
    sim.step(2)
    ref = m.phi(f)
    assert np.max(np.abs(sim.macro().cpu().numpy() - ref)) < tol * np.max(np.abs(ref))
    sim.close()


def test_a_source_field_needs_jets_on_dirichlet_boxes():
    d, n = 2, 9
    sim = LBM(d, n, 0.0, 1.0, u=(0.1, 0.05), bc="fullway")
    X = W.node_coords(d, [n] * d, 0.0, sim.dx)
    sim.init(_t(W.sine_product_value(X, 0.0)), _t(W.sine_product_grad(X, 0.0)), _t(np.ones(n * n)))
    sim.set_boundary_wave([1.0], [[1.0, 2.0]], [0.0])
    with pytest.raises(LHEError) as ei:
        sim.step(1)
    assert ei.value.status == _abi.ERR_STATE
    sim.set_source(None)
    sim.step(1)  # constant R again: the wave data apply
    sim.close()


def _adjoint_jet_grads(sim, seed, steps):
    """dL/d(jet) of every step, newest first reversed to step order, from dL/dphi_T = seed."""
    sim.adjoint_seed(_t(seed))
    out = []
    for _ in range(steps):
        out.append(sim.adjoint_jet_grad().cpu().numpy())
        sim.adjoint_step(1)
    return out[::-1]


def _oracle_jet_grads(m, seed, steps):
    lam = np.ascontiguousarray(np.broadcast_to(np.asarray(seed).ravel(), (m.Q, m.S)).copy())
    out = []
    for _ in range(steps):
        pts, g = m.jet_grad(lam)
        out.append(g)
        lam = m.adjoint_step(lam)
    return pts, out[::-1]


def _by_point(pts, g, dx):
    """Rows summed per distinct point (half-way mid-link points of diagonal links of neighbouring
    nodes coincide), keyed by the point in units of dx / 2."""
    acc = {}
    for p, row in zip(pts, g):
        key = tuple(np.round(np.asarray(p) / dx * 2).astype(int))
        acc[key] = acc.get(key, 0.0) + row
    return acc


@pytest.mark.parametrize("d,n,bc,order,tau", [
    (2, 41, "fullway", 4, 0.5), (2, 40, "halfway", 4, 0.8), (2, 41, "fullway", 1, 0.8), (2, 20, "halfway", 2, 0.5),
    (3, 11, "fullway", 3, 1.2), (3, 10, "halfway", 4, 0.5), (4, 6, "fullway", 4, 0.5), (4, 6, "halfway", 3, 0.8)])
def test_adjoint_jet_grad_matches_the_oracle(d, n, bc, order, tau):
    """The cotangent of every step's jets from a seeded dL/dphi_T against the oracle's transpose
    (Model.jet_grad after Model.adjoint_step): full-way per boundary node, half-way per distinct
    mid-link point; several blocks of boundary nodes. FP64 1e-12 relative."""
    u = [0.1, 0.05, -0.08, 0.06][:d] if bc == "fullway" else [0.01, 0.02, -0.01, 0.015][:d]
    steps = 4
    rng = np.random.default_rng(17 + d + order)
    m = O.Model(d, n, 0.0, 1.0, u, tau=tau, R=0.3, bc=bc, bc_order=order)
    seed = rng.normal(size=m.S)
    opts, og = _oracle_jet_grads(m, seed, steps)
    sim = LBM(d, n, 0.0, 1.0, u=u, tau=tau, R=0.3, bc=bc, bc_order=order)
    sim.init(_t(np.zeros(m.S)), _t(np.zeros(d * m.S)))
    pts, _ = sim.boundary_points()
    gg = _adjoint_jet_grads(sim, seed, steps)
    sim.close()
    assert len(pts) > 128 and gg[0].shape == (len(pts), jet_len(d)) and len(pts) == len(opts)
    scale = max(np.max(np.abs(g)) for g in og)
    for a, b in zip(gg, og):
        A, B = _by_point(pts, a, m.dx), _by_point(opts, b, m.dx)
        assert A.keys() == B.keys()
        err = max(np.max(np.abs(A[k] - B[k])) for k in A)
        assert err <= 1e-12 * scale, err


@pytest.mark.parametrize("d,n,bc,order,precision", [
    (2, 19, "fullway", 4, "fp64"), (2, 18, "halfway", 4, "fp64"), (3, 9, "fullway", 3, "fp64"),
    (3, 8, "halfway", 3, "fp64"), (5, 5, "fullway", 4, "fp64"), (5, 4, "halfway", 4, "fp64"),
    (2, 19, "fullway", 4, "fp32dev"), (3, 8, "halfway", 3, "fp32dev")])
def test_adjoint_jet_grad_is_the_transpose_of_the_forward(d, n, bc, order, precision):
    """With phi0 = 0 and R = 0 the final field is linear in the jets V_n of the steps, so
    <seed, phi_T(V)> = sum_n <dL/djet_n, V_n> for L = <seed, phi_T>; random V per row (one jet per
    unknown population, coincident half-way points included)."""
    import torch

    u = [0.02, 0.04, 0.06, 0.08, 0.1][:d] if bc == "fullway" else [0.01, 0.02, 0.01, 0.02, 0.01][:d]
    steps = 3
    rng = np.random.default_rng(5 + d)
    sim = LBM(d, n, 0.0, 1.0, u=u, tau=0.8, R=0.0, bc=bc, bc_order=order, precision=precision)
    S = sim.S
    sim.init(_t(np.zeros(S)), _t(np.zeros(d * S)))
    P = len(sim.boundary_points()[0])
    V = rng.normal(size=(steps, P, jet_len(d)))
    for k in range(steps):
        sim.set_boundary_jet(_t(V[k]))
        sim.step(1)
    seed = rng.normal(size=S)
    lhs = float(np.dot(seed, sim.macro().cpu().numpy()))
    G = _adjoint_jet_grads(sim, seed, steps)
    rhs = float(sum(np.sum(g * v) for g, v in zip(G, V)))
    sim.close()
    torch.cuda.synchronize()
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert abs(lhs - rhs) <= tol * max(1.0, abs(lhs), float(sum(np.sum(np.abs(g * v)) for g, v in zip(G, V))))


def test_adjoint_jet_grad_errors():
    import torch

    buf = torch.zeros(4096, dtype=torch.float64, device="cuda")
    sim = LBM(2, 8, 0.0, 1.0, u=(0.1, 0.05), bc="fullway", bc_order=4)
    sim.init(_t(np.zeros(64)), _t(np.zeros(128)))
    with pytest.raises(LHEError):
        _abi.lhe_lbm_adjoint_jet_grad(sim.h, buf.data_ptr())  # before adjoint_seed
    sim.adjoint_seed(_t(np.ones(64)))
    with pytest.raises(LHEError):
        _abi.lhe_lbm_adjoint_jet_grad(sim.h, None)
    g = sim.adjoint_jet_grad()
    assert g.shape == (28, jet_len(2)) and bool(torch.isfinite(g).all())
    sim.close()
    per = LBM(2, 8, u=(0.1, 0.05))
    per.init(_t(np.zeros(64)))
    per.adjoint_seed(_t(np.zeros(64)))
    with pytest.raises(LHEError):
        _abi.lhe_lbm_adjoint_jet_grad(per.h, buf.data_ptr())  # periodic box
    per.close()


@pytest.mark.parametrize("d,n,bc,order", [(2, 17, "fullway", 4), (2, 16, "halfway", 4), (3, 8, "halfway", 2)])
def test_box_autograd_matches_central_differences(d, n, bc, order):
    """LBMBoxFunction: phi_T of a Dirichlet box as a function of phi0, grad phi0 and every step's
    jets; torch.autograd's gradients against central differences of the loss 1/2 |phi_T - target|^2
    along random directions (exact up to rounding: the loss is quadratic in all three)."""
    import torch
    from paper_2410_13165_gb300.autograd import LBMBoxFunction

    u = [0.1, 0.05, -0.08][:d] if bc == "fullway" else [0.01, 0.02, -0.01][:d]
    T = 5
    sim = LBM(d, n, 0.0, 1.0, u=u, tau=0.8, R=0.3, bc=bc, bc_order=order)
    S, P, JL = sim.S, len(sim.boundary_points()[0]), jet_len(d)
    rng = np.random.default_rng(31 + d)
    cuda = lambda a, g=False: torch.tensor(a, dtype=torch.float64, device="cuda", requires_grad=g)  # noqa: E731
    phi0, grad, jets = cuda(rng.normal(size=S), True), cuda(rng.normal(size=(d, S)), True), cuda(rng.normal(size=(T, P, JL)), True)
    target = cuda(rng.normal(size=S))

    def loss(a, b, c):
        r = LBMBoxFunction.apply(a, b, c, sim) - target
        return 0.5 * torch.dot(r, r)

    loss(phi0, grad, jets).backward()
    assert phi0.grad.shape == phi0.shape and grad.grad.shape == grad.shape and jets.grad.shape == jets.shape
    with torch.no_grad():
        for _ in range(3):
            v = [cuda(rng.normal(size=tuple(x.shape))) for x in (phi0, grad, jets)]
            lp = float(loss(phi0 + v[0], grad + v[1], jets + v[2]))
            lm = float(loss(phi0 - v[0], grad - v[1], jets - v[2]))
            an = float(sum(torch.sum(x.grad * w) for x, w in zip((phi0, grad, jets), v)))
            assert abs((lp - lm) / 2.0 - an) <= 1e-11 * max(lp, lm, 1.0), ((lp - lm) / 2.0, an)
    sim.close()


_SP = dict(A=0.8, lam=1.3, kappa=[np.pi, 2.0, 1.5, 2.5, 1.2], theta=[0.3, -0.2, 0.1, 0.4, -0.3])


def _sp(d):
    return dict(A=_SP["A"], lam=_SP["lam"], kappa=_SP["kappa"][:d], theta=_SP["theta"][:d])


@pytest.mark.parametrize("d,n,bc,precision,steps", [
    (2, 17, "fullway", "fp64", 12), (2, 16, "halfway", "fp64", 12), (3, 9, "fullway", "fp32dev", 10),
    (3, 8, "halfway", "fp64", 10), (3, 9, "fullway", "fp64", 10), (4, 12, "fullway", "fp64", 6),
    (4, 12, "halfway", "fp64", 6)])
def test_sine_product_provider_matches_the_oracle(d, n, bc, precision, steps):
    """lhe_lbm_set_boundary_sine_product: the manufactured solution A exp(-lam t) prod_i sin(kappa_i x_i +
    theta_i) with its source R = phi_t + u.grad phi, data and source formed on the device for several
    steps per call, against the oracle fed that solution's jets and sources step by step (D4Q33 on a
    12^4 box). FP64 1e-13, FP32 deviations 1e-5."""
    p = _sp(d)
    u = [0.1, 0.05, -0.08, 0.06][:d] if bc == "fullway" else [0.01, 0.02, -0.01, 0.015][:d]
    m = O.Model(d, n, -1.0, 1.0, u, bc=bc)
    X = m.coords()
    phi0, grad = W.sine_product_value(X, 0.0, **p), W.sine_product_grad(X, 0.0, **p)
    Rt = lambda k: W.sine_product_source(X, k * m.dt, u, **p)  # noqa: E731  R(x, t_k)
    ref = m.phi(m.step_jets(m.init(phi0, grad, 3), 0, steps, lambda P, t: W.sine_product_jets(P, t, **p), Rfield_fn=Rt))
    sim = LBM(d, n, -1.0, 1.0, u=u, bc=bc, precision=precision)
    sim.init(_t(phi0), _t(grad), _t(Rt(0)))
    sim.set_boundary_sine_product(**p)
    sim.step(steps // 2)
    sim.step(steps - steps // 2)
    got = sim.macro().cpu().numpy()
    sim.close()
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))


@pytest.mark.parametrize("bc", ["fullway", "halfway"])
def test_sine_product_provider_equals_the_jet_path(bc):
    """The provider against the library's own per-step path (lhe_lbm_set_source with R(x, t_{n+1}) and
    lhe_lbm_set_boundary_jet with the solution's jets) on a 3D box over 20 steps: the same scheme, the
    records formed once and scaled by exp(-lam t) instead of every step (rounding-level differences)."""
    d, n = 3, (13 if bc == "fullway" else 12)
    p = _sp(d)
    u = [0.1, 0.05, -0.08] if bc == "fullway" else [0.01, 0.02, -0.01]
    X = W.node_coords(d, [n] * d, -1.0, 2.0 / ((n - 1) if bc == "fullway" else n), halfway=(bc == "halfway"))
    out = []
    for mode in ("provider", "jets"):
        sim = LBM(d, n, -1.0, 1.0, u=u, bc=bc)
        dt = sim.dt
        sim.init(_t(W.sine_product_value(X, 0.0, **p)), _t(W.sine_product_grad(X, 0.0, **p)),
                 _t(W.sine_product_source(X, 0.0, u, **p)))
        if mode == "provider":
            sim.set_boundary_sine_product(**p)
            sim.step(20)
        else:
            pts, toff = sim.boundary_points()
            for k in range(20):
                sim.set_source(_t(W.sine_product_source(X, (k + 1) * dt, u, **p)))
                sim.set_boundary_jet(_t(W.sine_product_jets(pts, k * dt + toff, **p)))
                sim.step(1)
        out.append(sim.macro().cpu().numpy())
        sim.close()
    assert np.max(np.abs(out[0] - out[1])) < 1e-13 * np.max(np.abs(out[1]))


def test_sine_product_provider_errors():
    import math

    per = LBM(2, 8, u=(0.1, 0.05))
    with pytest.raises(LHEError) as ei:
        per.set_boundary_sine_product()
    assert ei.value.status == _abi.ERR_STATE
    per.close()
    box = LBM(2, 9, -1.0, 1.0, u=(0.1, 0.05), bc="fullway")
    with pytest.raises(LHEError) as ei:
        box.set_boundary_sine_product(lam=math.nan)
    assert ei.value.status == _abi.ERR_ARG
    box.close()


def test_sine_product_provider_restart_from_a_checkpoint():
    """get_state at step 5, five more steps; set_state back to step 5 (the provider re-forms the source
    of that state's last collision) and the same five steps again: identical fields, bit for bit."""
    import torch

    d, n, bc = 3, 10, "halfway"
    p = _sp(d)
    u = [0.01, 0.02, -0.01]
    X = W.node_coords(d, [n] * d, -1.0, 2.0 / n, halfway=True)
    sim = LBM(d, n, -1.0, 1.0, u=u, bc=bc)
    sim.init(_t(W.sine_product_value(X, 0.0, **p)), _t(W.sine_product_grad(X, 0.0, **p)),
             _t(W.sine_product_source(X, 0.0, u, **p)))
    sim.set_boundary_sine_product(**p)
    sim.step(5)
    ck = sim.get_state().clone()
    phi5 = sim.macro().clone()
    sim.step(5)
    a = sim.macro().clone()
    sim.step(3)  # move on, then restore
    sim.set_state(ck, 5)
    assert torch.equal(sim.macro(), phi5)
    sim.step(5)
    assert torch.equal(sim.macro(), a)
    sim.close()
