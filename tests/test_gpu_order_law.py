"""GPU: the order law of Eq. (cr-estimation), Z = min(K + 1, P), for the CUDA path with Dirichlet
boundaries: full-way boundary orders P = 1, 3, 4 and half-way P = 1..4 against the initialisation
orders K = 1, 3 in 2D (Example 1's setting: R = 5, exact solutions of the family h = b + R t +
sum_m a_m sin(kappa_m.(x - u t) + theta_m)), the half-way P = 3 case that reaches fourth order at
small u (the O(u dt^3) argument after Eq. (cr-estimation)), and the 4D full-way box of Example 3.
Rates are measured on the last refinement of three grids."""
import numpy as np
import pytest

from paper_2410_13165_gb300 import LBM, build, workloads as W
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu

WAVE2 = dict(a=[1.0, 0.5], kappa=[(np.pi, np.pi), (2.0, -1.0)], theta=[0.3, 1.1], b=0.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def dirichlet_rmse(d, bc, P, K, N, u, T, R, wave, lo=0.0, hi=1.0):
    n = N + 1 if bc == "fullway" else N
    dx = (hi - lo) / N
    X = W.node_coords(d, n, lo, dx, halfway=(bc == "halfway"))
    phi0, grad = W.wave_solution(X, 0.0, u, R, **wave)
    sim = LBM(d, n, lo, hi, u=u, R=R, bc=bc, bc_order=P, init_order=K)
    sim.init(_t(phi0), _t(grad))
    sim.set_boundary_wave(wave["a"], wave["kappa"], wave["theta"], wave.get("b", 0.0), wave.get("g"))
    steps = int(round(T / sim.dt))
    sim.step(steps)
    exact, _ = W.wave_solution(X, steps * sim.dt, u, R, **wave)
    err = float(np.sqrt(np.mean((sim.macro().cpu().numpy() - exact) ** 2)))
    sim.close()
    return err


def rates(errs):
    return [float(np.log2(a / b)) for a, b in zip(errs, errs[1:])]


@pytest.mark.parametrize("P,K", [(1, 1), (1, 3), (3, 1), (3, 3), (4, 1), (4, 3)])
def test_fullway_order_law_2d(P, K):
    errs = [dirichlet_rmse(2, "fullway", P, K, N, (0.1, 0.1), 2.0, 5.0, WAVE2) for N in (20, 40, 80)]
    sl = rates(errs)
    assert abs(sl[-1] - min(K + 1, P)) < 0.45, (errs, sl)


@pytest.mark.parametrize("P,K,Z", [(1, 1, 1), (1, 3, 1), (2, 1, 2), (2, 3, 2), (3, 1, 2), (4, 1, 2), (4, 3, 4),
                                   (3, 3, 4)])
def test_halfway_order_law_2d_small_velocity(P, K, Z):
    """Half-way at u = (0.01, 0.01): Z = min(K + 1, P), except P = 3 with K = 3, which converges at
    fourth order because the order-dt^3 terms of Eq. (bun2) are O(u dt^3)."""
    errs = [dirichlet_rmse(2, "halfway", P, K, N, (0.01, 0.01), 2.0, 5.0, WAVE2) for N in (20, 40, 80)]
    sl = rates(errs)
    assert abs(sl[-1] - Z) < 0.5, (errs, sl)


@pytest.mark.parametrize("P,K", [(4, 3), (4, 1)])
def test_fullway_order_law_4d_example3(P, K):
    """Example 3's box [-1, 1]^4 with phi = sin(pi sum_i (x_i - u_i t)) and u = (0.05, 0.2, 0.08, 0.1)."""
    wave = dict(a=[1.0], kappa=[(np.pi,) * 4], theta=[0.0])
    u = (0.05, 0.2, 0.08, 0.1)
    errs = [dirichlet_rmse(4, "fullway", P, K, N, u, 0.5, 0.0, wave, lo=-1.0, hi=1.0) for N in (10, 20, 40)]
    sl = rates(errs)
    assert abs(sl[-1] - min(K + 1, P)) < 0.5, (errs, sl)
