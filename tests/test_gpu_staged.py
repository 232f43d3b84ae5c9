"""GPU: the staged FP32-deviation step (periodic D3Q19, rows brought into shared memory by bulk
asynchronous copies) against the register-pull kernel, bit for bit, and against the oracle.

Both kernels evaluate the same per-node arithmetic in the same order, so every population, phi and
dL/dR must agree exactly; the shapes cover tiles of one and several rows, wrap-around in y and z
on grids of 3 rows, the maximum row length and extents the staged kernel does not take. Rows of 128
and 256 nodes are run both where the kernel takes their length as a compile-time constant (tiles of
4 and 2 rows) and where it does not (n_2 without such a divisor)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import LBM, LHEError, build, workloads as W
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


def _problem(n, seed):
    m = O.Model(3, list(n), 0.0, [ni / 32.0 for ni in n], [0.0] * 3)
    X = m.coords()
    F = W.fourier_field(3, 4, seed, 0.0, [ni / 32.0 for ni in n])
    return F.value(X), F.grad(X)


def _pair(n, tau, steps, R=0.0, Rf=None, seed=0):
    import torch

    phi0, grad = _problem(n, seed)
    out = []
    for staged in (True, False):
        sim = LBM(3, list(n), 0.0, [ni / 32.0 for ni in n], u=(0.1, -0.05, 0.08), tau=tau, R=R,
                  precision="fp32dev", staged=staged)
        sim.init(_t(phi0), _t(grad), None if Rf is None else _t(Rf))
        sim.step(steps)
        out.append((sim.get_state().clone(), sim.macro().clone()))
        sim.close()
    torch.cuda.synchronize()
    return out, phi0, grad


SHAPES = [(16, 12, 8), (32, 6, 5), (12, 20, 7), (64, 8, 3), (8, 3, 4), (128, 4, 3), (512, 3, 3), (4, 5, 6),
          (20, 9, 5), (10, 6, 4), (576, 3, 3), (128, 8, 5), (128, 6, 4), (256, 6, 3), (256, 3, 4)]


@pytest.mark.parametrize("n", SHAPES)
@pytest.mark.parametrize("tau", [0.5, 0.8])
def test_staged_step_is_bitwise_the_register_kernel(n, tau):
    import torch

    (st_a, phi_a), (st_b, phi_b) = _pair(n, tau, 13, seed=sum(n))[0]
    assert torch.equal(st_a, st_b)
    assert torch.equal(phi_a, phi_b)


@pytest.mark.parametrize("n", [(32, 12, 6), (128, 8, 3), (256, 4, 3)])
def test_staged_step_with_sources_matches_the_oracle(n):
    import torch

    S = int(np.prod(n))
    Rf = 0.4 * np.sin(np.arange(S) * 0.013)
    (res, phi0, grad) = _pair(n, 0.8, 40, Rf=Rf, seed=3)
    (st_a, phi_a), (st_b, phi_b) = res
    assert torch.equal(st_a, st_b) and torch.equal(phi_a, phi_b)
    m = O.Model(3, list(n), 0.0, [ni / 32.0 for ni in n], (0.1, -0.05, 0.08), tau=0.8)
    o = m.phi(m.step(m.init(phi0, grad, 3), 0, 40, Rfield=Rf))
    g = phi_a.cpu().numpy()
    assert np.max(np.abs(g - o)) < 1e-5 * max(np.max(np.abs(o)), np.max(np.abs(phi0)))
    (res, _, _) = _pair(n, 0.5, 40, R=2.5, seed=4)
    assert torch.equal(res[0][0], res[1][0])


@pytest.mark.parametrize("n", [(32, 8, 6), (128, 8, 3), (256, 4, 3)])
@pytest.mark.parametrize("tau", [0.5, 1.2])
def test_staged_adjoint_is_bitwise_the_register_kernel(n, tau):
    import torch

    phi0, grad = _problem(n, 9)
    rng = np.random.default_rng(10)
    target = rng.normal(size=int(np.prod(n)))
    res = []
    for staged in (True, False):
        sim = LBM(3, list(n), 0.0, [ni / 32.0 for ni in n], u=(0.1, -0.05, 0.08), tau=tau, precision="fp32dev",
                  staged=staged)
        sim.init(_t(phi0), _t(grad), _t(0.1 * target))
        sim.step(20)
        r = sim.macro() - _t(target)
        sim.adjoint_seed(r.contiguous())
        sim.adjoint_step(20)
        gphi, ggrad, gR = sim.adjoint_grads(want_grad=True, want_R=True)
        res.append((gphi.clone(), ggrad.clone(), gR.clone()))
        sim.close()
    for a, b in zip(*res):
        assert torch.equal(a, b)


def test_staged_step_full_size_256():
    """The benchmark's FP32-deviation workload and launch configuration (D3Q19 256^3, tau = 0.8)."""
    import torch

    n = 256
    phi0, grad, _, _ = W.periodic_problem(3, n, 8, 2)
    res = []
    for staged in (True, False):
        sim = LBM(3, n, u=(0.1, 0.1, 0.1), tau=0.8, precision="fp32dev", staged=staged)
        sim.init(_t(phi0), _t(grad))
        sim.step(3)
        res.append(sim.get_state().clone())
        sim.close()
    assert torch.equal(res[0], res[1])


def _seq_states(n, tau, calls, staged, seed=0, adjoint_calls=(), pdl=True):
    """State and phi after a sequence of step(k) calls (then adjoint_step calls, if any)."""
    import torch

    phi0, grad = _problem(n, seed)
    sim = LBM(3, list(n), 0.0, [ni / 32.0 for ni in n], u=(0.1, -0.05, 0.08), tau=tau, precision="fp32dev",
              staged=staged, pdl=pdl)
    sim.init(_t(phi0), _t(grad))
    for k in calls:
        sim.step(k)
    out = [sim.get_state().clone(), sim.macro().clone()]
    if adjoint_calls:
        sim.adjoint_seed(sim.macro().contiguous())
        for k in adjoint_calls:
            sim.adjoint_step(k)
        gphi, _, gR = sim.adjoint_grads(want_grad=False, want_R=True)
        out += [gphi.clone(), gR.clone()]
    sim.close()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,calls", [((16, 12, 8), [5, 1, 2, 7, 1, 3]), ((8, 3, 4), [2, 2, 9]),
                                     ((32, 6, 5), [1, 1, 6, 11]), ((12, 20, 7), [17])])
def test_consecutive_launches_in_one_call_are_bitwise_single_calls(n, calls):
    """Within one step(k) / adjoint_step(k) call the step kernels after the first are launched with
    programmatic dependent launch; the result must equal k calls of one step, plain stream ordering
    (LHE_FLAG_NO_PDL) and the register kernel, over call sequences that mix both."""
    import torch

    ref = _seq_states(n, 0.8, [1] * sum(calls), True, seed=sum(n), adjoint_calls=[1] * 6)
    run = _seq_states(n, 0.8, calls, True, seed=sum(n), adjoint_calls=[2, 3, 1])
    plain = _seq_states(n, 0.8, calls, True, seed=sum(n), adjoint_calls=[2, 3, 1], pdl=False)
    reg = _seq_states(n, 0.8, calls, False, seed=sum(n), adjoint_calls=[6])
    for a, b, c, d in zip(ref, run, plain, reg):
        assert torch.equal(a, b) and torch.equal(a, c) and torch.equal(a, d)


def test_staged_step_128_matches_register_kernel():
    """The precision workload's grid (D3Q19 128^3, tau = 0.8), 12 steps in one call."""
    import torch

    n = 128
    phi0, grad, _, _ = W.periodic_problem(3, n, 8, 2)
    res = []
    for staged in (True, False):
        sim = LBM(3, n, u=(0.1, 0.1, 0.1), tau=0.8, precision="fp32dev", staged=staged)
        sim.init(_t(phi0), _t(grad))
        sim.step(12)
        res.append((sim.get_state().clone(), sim.macro().clone()))
        sim.close()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


@pytest.mark.parametrize("adjoint", [False, True])
def test_wait_expiry_is_reported_and_a_new_state_recovers(adjoint):
    """The failure path of the staged kernel, run without any fault: LHE_FLAG_TEST_EXPIRE_WAIT gives the
    compute warps of the handle's first staged launch a zero wait limit, so they give up on copies
    still in flight. The kernel must return (the producer warp waits, bounded, for the copies it
    issued), the next calls must report LHE_ERR_CUDA, and a new state (lhe_lbm_init) must clear the
    report and step exactly like a handle that never failed."""
    import torch

    n = (64, 64, 64)
    hi = [ni / 32.0 for ni in n]
    v, g = _problem(n, 70)
    kw = dict(u=(0.1, -0.05, 0.08), tau=0.8, precision="fp32dev")
    ref = LBM(3, n, 0.0, hi, **kw)
    sim = LBM(3, n, 0.0, hi, flags=_abi.FLAG_TEST_EXPIRE_WAIT, **kw)
    for s in (ref, sim):
        s.init(_t(v), _t(g))
    if adjoint:
        sim.adjoint_seed(sim.macro())
        sim.adjoint_step(1)          # the armed launch: the adjoint kernel gives up
    else:
        sim.step(1)                  # the armed launch: the forward kernel gives up
    torch.cuda.synchronize()         # the kernel returned
    for call in ((lambda: sim.adjoint_step(1)) if adjoint else (lambda: sim.step(1)), sim.macro, sim.diagnostics):
        with pytest.raises(LHEError) as ei:
            call()
        assert ei.value.status == _abi.ERR_CUDA and "timed out" in str(ei.value)
    # a new state clears the report; the hook was one launch only
    sim.init(_t(v), _t(g))
    for s in (ref, sim):
        s.step(5)
    assert torch.equal(sim.get_state(), ref.get_state())
    if adjoint:
        for s in (ref, sim):
            s.adjoint_seed(s.macro())
            s.adjoint_step(4)
        gs = [s.adjoint_grads(want_grad=True, want_R=True) for s in (ref, sim)]
        for a, b in zip(gs[0], gs[1]):
            assert torch.equal(a, b)
    assert sim.diagnostics()["ok"]
    ref.close()
    sim.close()
