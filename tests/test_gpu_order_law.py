"""GPU: the order law of Eq. (cr-estimation), Z = min(K + 1, P), for the CUDA path with Dirichlet
boundaries: full-way boundary orders P = 1, 3, 4 and half-way P = 1..4 against the initialisation
orders K = 1, 3 in 2D (Example 1's setting: R = 5, exact solutions of the family h = b + R t +
sum_m a_m sin(kappa_m.(x - u t) + theta_m)), the half-way P = 3 case that reaches fourth order at
small u (the O(u dt^3) argument after Eq. (cr-estimation)), and the 4D full-way box of Example 3.
Rates are measured on the last refinement of three grids. Table 1's stability pattern at T = 10: the
half-way scheme's error grows under refinement at u = (0.1, 0.1) while the full-way scheme converges
(also at u = (0.4, 0.4)). The RMSEs equal the oracle's on one grid of each scheme."""
import numpy as np
import pytest

from oracle import oracle as O
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


def oracle_rmse(bc, P, K, N, u, T, R, wave):
    """The same 2D problem on the oracle (Model.step with the exact-solution family as boundary data)."""
    n = N + 1 if bc == "fullway" else N
    m = O.Model(2, n, 0.0, 1.0, u, R=R, bc=bc, bc_order=P)
    w = m.wave(a=wave["a"], kappa=wave["kappa"], theta=wave["theta"], b=wave.get("b", 0.0))
    f = m.init(m.exact(w, 0.0), m.exact_grad(w, 0.0), order=K)
    steps = int(round(T / m.dt))
    f = m.step(f, 0, steps, wave=w)
    return O.rmse(m.phi(f), m.exact(w, steps * m.dt))


@pytest.mark.parametrize("bc,P,K,u", [("fullway", 4, 3, (0.1, 0.1)), ("fullway", 1, 1, (0.1, 0.1)),
                                      ("halfway", 4, 3, (0.01, 0.01)), ("halfway", 3, 1, (0.01, 0.01))])
def test_order_law_rmse_equals_the_oracles(bc, P, K, u):
    gpu = dirichlet_rmse(2, bc, P, K, 20, u, 2.0, 5.0, WAVE2)
    orc = oracle_rmse(bc, P, K, 20, u, 2.0, 5.0, WAVE2)
    assert abs(gpu - orc) <= 1e-9 * orc, (gpu, orc)


def test_halfway_diverges_where_fullway_converges_table1():
    """Table 1's pattern at T = 10 with R = 5 and order-4 boundaries (K = 3): at u = (0.1, 0.1), inside
    the bulk's entropy and L2 region, the half-way error grows under refinement (N = 10, 20, 40) and
    exceeds 1, while the full-way error falls by more than 12 per halving of dx; at u = (0.01, 0.01)
    the half-way scheme converges, and the full-way scheme converges even at u = (0.4, 0.4). Every run
    is bounded in steps; a diverging one is reported through its values (no fault is involved)."""
    def errs(bc, u):
        return [dirichlet_rmse(2, bc, 4, 3, N, u, 10.0, 5.0, WAVE2) for N in (10, 20, 40)]
    full = errs("fullway", (0.1, 0.1))
    half = errs("halfway", (0.1, 0.1))
    half_slow = errs("halfway", (0.01, 0.01))
    full_fast = errs("fullway", (0.4, 0.4))
    for e in (full, half_slow, full_fast):
        assert all(a / b > 12.0 for a, b in zip(e, e[1:])), e
    assert half[0] < half[1] < half[2] and half[2] > 1.0, half
    # the converging runs equal the oracle's on the coarsest grid
    assert abs(full[0] - oracle_rmse("fullway", 4, 3, 10, (0.1, 0.1), 10.0, 5.0, WAVE2)) <= 1e-9 * full[0]
    assert abs(half_slow[0] - oracle_rmse("halfway", 4, 3, 10, (0.01, 0.01), 10.0, 5.0, WAVE2)) <= 1e-9 * half_slow[0]
