"""The allocation-free diagnostics entry point against the handle-based one.

lhe_lbm_diagnostics_noalloc serves callers that cannot allocate device memory when they inspect a
state (framework-managed or budgeted device memory, or places where cudaMalloc is refused): it
takes a caller-owned FP64 state and writes four device doubles, using only a scratch array compiled
into the library. Each case calls it twice in a row, with steps in between, on the state of a handle
and compares with that handle's own diagnostics: periodic boxes and both Dirichlet schemes, tau = 1
(where the post-collision values are used as they are) and lattices of more than 65536 nodes, so that
many reduction blocks meet in the final pass. This file is collected last so that a run stopping at
its first failure has already run every other test."""
import numpy as np
import pytest

from paper_2410_13165_gb300 import LBM, LHEError, build, workloads as W
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu

U3 = (0.1, -0.05, 0.08)
WAVE3 = dict(a=[1.0, 0.4], kappa=[(np.pi, np.pi, 0.0), (2.0, -1.0, 1.5)], theta=[0.3, 1.1], b=0.2)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


def _close(a, b, rtol):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1e-300)


def _t(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def _handle(bc, tau, R, n, field):
    d = 3
    if bc == "periodic":
        phi0, grad, _, _ = W.periodic_problem(d, n, 6, 21)
        Rf = _t(0.2 * W.fourier_field(d, 3, 22).value(W.node_coords(d, n, 0.0, 1.0 / n))) if field else None
        sim = LBM(d, n, u=U3, tau=tau, R=R)
        sim.init(_t(phi0), _t(grad), Rf)
        return sim, Rf
    N = n - 1 if bc == "fullway" else n
    X = W.node_coords(d, n, 0.0, 1.0 / N, halfway=(bc == "halfway"))
    phi0, grad = W.wave_solution(X, 0.0, U3, R, **WAVE3)
    sim = LBM(d, n, 0.0, 1.0, u=U3, tau=tau, R=R, bc=bc)
    sim.init(_t(phi0), _t(grad))
    sim.set_boundary_wave(WAVE3["a"], WAVE3["kappa"], WAVE3["theta"], WAVE3["b"], None)
    return sim, None


@pytest.mark.parametrize("bc,tau,R,n,field", [
    ("periodic", 0.5, 0.0, 40, False),
    ("periodic", 0.8, 1.5, 48, False),
    ("periodic", 1.0, 0.7, 40, False),
    ("periodic", 0.5, 0.0, 48, True),
    ("fullway", 0.8, 1.5, 41, False),
    ("fullway", 1.0, 0.7, 49, False),
    ("halfway", 0.5, 0.7, 40, False),
    ("halfway", 1.0, 1.5, 48, False),
])
def test_noalloc_matches_the_handle_diagnostics_twice(bc, tau, R, n, field):
    import torch

    sim, Rf = _handle(bc, tau, R, n, field)
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(3 + call)
        want = sim.diagnostics()
        state = sim.get_state().view(torch.float64)
        p = sim.params
        p.stream = torch.cuda.current_stream().cuda_stream
        _abi.lhe_lbm_diagnostics_noalloc(p, state.data_ptr(), None if Rf is None else Rf.data_ptr(), out.data_ptr())
        got = out.cpu().numpy()
        assert _close(got[0], want["mass"], 1e-12) or abs(got[0] - want["mass"]) < 1e-10, (got, want)
        assert _close(got[1], want["entropy"], 1e-12), (got, want)
        assert got[2] == want["max_abs"], (got, want)
        assert got[3] == want["nonfinite"] == 0
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_maximum_other_precisions_and_unstable_weights():
    import torch

    p = _abi.lhe_lbm_default_params()
    p.d = 3
    for i in range(3):
        p.n[i] = 1024  # 2^30 nodes > 2^28: rejected on the host before any launch
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(LHEError) as ei:
        _abi.lhe_lbm_diagnostics_noalloc(p, out.data_ptr(), None, out.data_ptr())
    assert ei.value.status == _abi.ERR_ARG and "268435456" in str(ei.value)
    q = _abi.lhe_lbm_default_params()
    q.precision = _abi.FP32_DEV
    with pytest.raises(LHEError) as ei:
        _abi.lhe_lbm_diagnostics_noalloc(q, out.data_ptr(), None, out.data_ptr())
    assert ei.value.status == _abi.ERR_ARG
    # Example 3's u = 0.4 (1, 1, 1, 1) has some omega_k < 0: rejected as by lhe_lbm_create ...
    r = _abi.lhe_lbm_default_params()
    r.d = 4
    for i in range(4):
        r.n[i] = 4
        r.u[i] = 0.4
    pop = torch.zeros(33 * 4 ** 4, dtype=torch.float64, device="cuda")
    with pytest.raises(LHEError) as ei:
        _abi.lhe_lbm_diagnostics_noalloc(r, pop.data_ptr(), None, out.data_ptr())
    assert ei.value.status == _abi.ERR_UNSTABLE
    # ... and accepted with allow_unstable (a zero state has zero mass and entropy)
    r.allow_unstable = 1
    r.stream = torch.cuda.current_stream().cuda_stream
    _abi.lhe_lbm_diagnostics_noalloc(r, pop.data_ptr(), None, out.data_ptr())
    assert out.cpu().numpy().tolist() == [0.0, 0.0, 0.0, 0.0]
