"""The allocation-free diagnostics entry point against the handle-based one.

lhe_lbm_diagnostics_noalloc serves callers that cannot allocate device memory when they inspect a
state (framework-managed or budgeted device memory, or places where cudaMalloc is refused): it
takes a caller-owned FP64 state and writes four device doubles, using only a scratch array compiled
into the library. This file is collected last so that a run stopping at its first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2410_13165_gb300 import LBM, LHEError, build, workloads as W
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


def _close(a, b, rtol):
    return abs(a - b) <= rtol * max(abs(a), abs(b), 1e-300)


@pytest.mark.parametrize("tau,R,field", [(0.5, 0.0, False), (0.8, 1.5, False), (0.5, 0.0, True)])
def test_noalloc_matches_the_handle_diagnostics_twice(tau, R, field):
    import torch

    d, n = 3, 40
    phi0, grad, _, _ = W.periodic_problem(d, n, 6, 21)
    Rf = torch.from_numpy(0.2 * W.fourier_field(d, 3, 22).value(W.node_coords(d, n, 0.0, 1.0 / n))).cuda() if field else None
    sim = LBM(d, n, u=(0.1, -0.05, 0.08), tau=tau, R=R)
    sim.init(torch.from_numpy(phi0).cuda(), torch.from_numpy(np.ascontiguousarray(grad).ravel()).cuda(), Rf)
    out = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        sim.step(3 + call)
        want = sim.diagnostics()
        state = sim.get_state().view(torch.float64)
        p = sim.params
        p.stream = torch.cuda.current_stream().cuda_stream
        _abi.lhe_lbm_diagnostics_noalloc(p, state.data_ptr(), None if Rf is None else Rf.data_ptr(), out.data_ptr())
        got = out.cpu().numpy()
        assert _close(got[0], want["mass"], 1e-12) or abs(got[0] - want["mass"]) < 1e-10
        assert _close(got[1], want["entropy"], 1e-12)
        assert got[2] == want["max_abs"]
        assert got[3] == want["nonfinite"] == 0
    sim.close()


def test_noalloc_rejects_lattices_beyond_its_scratch_and_other_precisions():
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
