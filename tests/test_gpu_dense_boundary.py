"""GPU: the FP64 step of Dirichlet boxes runs the whole box as rows that take their unknown populations
from a dense array of the step's boundary data (default); LHE_FLAG_NODE_BOUNDARY selects the
boundary-node kernels instead. With boundary data given as records (jets each step, or the
manufactured solution's records formed on the device) both compute the same bits; with the
exact-solution family (its data separated in time in the dense form) they agree to rounding, and
both with the oracle. Both schemes, every boundary order, s = 2 and general s, d = 1..5 on ragged
boxes (edges and corners included)."""
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


U = (0.1, -0.05, 0.08, 0.03, -0.06)
U_HALF = (0.01, -0.02, 0.015, 0.01, -0.01)


def _wave(d):
    kap = [tuple(np.pi * np.array([1.0, -0.5, 0.7, 0.3, -0.4][:d])), tuple(np.array([2.0, 1.0, -1.5, 0.5, 1.0][:d]))]
    return dict(a=[1.0, 0.4], kappa=kap, theta=[0.3, 1.1], b=0.2, g=[0.5, -0.3, 0.2, 0.1, -0.2][:d])


def _box(d, n, bc):
    """A box with equal dx on [0, L_1] x ... (ragged extents): hi_i from n_i."""
    span = [(ni - 1) if bc == "fullway" else ni for ni in n]
    dx = 1.0 / span[0]
    return [0.0] * d, [s * dx for s in span], dx


@pytest.mark.parametrize("d,n,bc,P,tau", [
    (1, (11,), "fullway", 4, 0.5), (1, (10,), "halfway", 3, 0.8),
    (2, (9, 7), "fullway", 4, 0.5), (2, (8, 6), "halfway", 4, 0.8), (2, (33, 5), "fullway", 3, 0.5),
    (3, (9, 7, 6), "fullway", 4, 0.5), (3, (8, 6, 5), "halfway", 3, 0.5), (3, (5, 9, 4), "fullway", 1, 0.8),
    (3, (40, 3, 4), "halfway", 2, 0.6), (4, (7, 5, 4, 6), "fullway", 4, 0.5), (4, (6, 5, 4, 3), "halfway", 4, 1.2),
    (5, (5, 4, 4, 3, 4), "fullway", 4, 0.5), (5, (4, 4, 3, 4, 3), "halfway", 1, 0.5)])
def test_dense_boundary_with_the_family_equals_the_node_kernels_and_the_oracle(d, n, bc, P, tau):
    lo, hi, dx = _box(d, n, bc)
    u = (U if bc == "fullway" else U_HALF)[:d]
    wv = _wave(d)
    R = 0.7
    X = W.node_coords(d, list(n), 0.0, dx, halfway=(bc == "halfway"))
    phi0, grad = W.wave_solution(X, 0.0, u, R, **wv)
    steps = 12
    outs = []
    for flags in (0, _abi.FLAG_NODE_BOUNDARY):
        sim = LBM(d, list(n), lo, hi, u=u, R=R, tau=tau, bc=bc, bc_order=P, flags=flags)
        sim.init(_t(phi0), _t(grad))
        sim.set_boundary_wave(wv["a"], wv["kappa"], wv["theta"], wv["b"], wv["g"])
        sim.step(steps)
        outs.append(sim.get_state().view(__import__("torch").float64).cpu().numpy())
        phi = sim.macro().cpu().numpy()
        sim.close()
    scale = np.max(np.abs(outs[1]))
    assert np.max(np.abs(outs[0] - outs[1])) <= 1e-14 * scale
    m = O.Model(d, list(n), lo, hi, u, tau=tau, R=R, bc=bc, bc_order=P)
    w = m.wave(a=wv["a"], kappa=wv["kappa"], theta=wv["theta"], b=wv["b"], g=wv["g"])
    ref = m.phi(m.step(m.init(phi0, grad, 3), 0, steps, wave=w))
    assert np.max(np.abs(phi - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("d,n,bc,tau", [(1, (12,), "halfway", 0.5), (2, (9, 7), "fullway", 0.5), (2, (8, 6), "halfway", 0.8),
                                        (3, (9, 7, 6), "halfway", 0.5), (4, (7, 5, 4, 6), "fullway", 0.8),
                                        (5, (5, 4, 4, 3, 4), "halfway", 0.5)])
def test_dense_boundary_with_records_is_bitwise_the_node_kernels(d, n, bc, tau):
    """Records: the manufactured solution's (formed once, scaled every step) and jets set every step."""
    import torch

    lo, hi, dx = _box(d, n, bc)
    u = (U if bc == "fullway" else U_HALF)[:d]
    X = W.node_coords(d, list(n), 0.0, dx, halfway=(bc == "halfway"))
    kap, th = [np.pi] * d, [0.2 * (i + 1) for i in range(d)]
    states = {}
    for kind in ("sine_product", "jets"):
        for flags in (0, _abi.FLAG_NODE_BOUNDARY):
            sim = LBM(d, list(n), lo, hi, u=u, tau=tau, bc=bc, flags=flags)
            sim.init(_t(W.sine_product_value(X, 0.0, kappa=kap, theta=th)),
                     _t(W.sine_product_grad(X, 0.0, kappa=kap, theta=th)),
                     _t(W.sine_product_source(X, 0.0, u, kappa=kap, theta=th)))
            if kind == "sine_product":
                sim.set_boundary_sine_product(kappa=kap, theta=th)
                sim.step(9)
            else:
                for _ in range(9):
                    sim.set_source(_t(W.sine_product_source(X, (sim.step_index + 1) * sim.dt, u, kappa=kap, theta=th)))
                    pts, toff = sim.boundary_points()
                    sim.set_boundary_jet(_t(W.sine_product_jets(pts, sim.step_index * sim.dt + toff, kappa=kap, theta=th)))
                    sim.step(1)
            states[(kind, flags)] = sim.get_state().clone()
            sim.close()
        assert torch.equal(states[(kind, 0)], states[(kind, _abi.FLAG_NODE_BOUNDARY)]), kind
