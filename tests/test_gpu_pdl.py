"""GPU: programmatic dependent launch between the step kernels of one call changes no bit.

lhe_lbm_step(n) / lhe_lbm_adjoint_step(n) launch their second and later step kernels so that each
may be scheduled while the previous step finishes (it waits for that step before it touches global
memory). Every result must equal the same calls with plain stream ordering (LHE_FLAG_NO_PDL), for
the FP64 kernel (s = 2, general and scaled collisions), the register FP32-deviation kernel, and
Dirichlet boxes, where a boundary kernel sits between consecutive step kernels."""
import numpy as np
import pytest

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


def _run(d, n, u, tau, precision, bc, pdl, steps=23, adjoint=9):
    import torch

    halfway = bc == "halfway"
    sim = LBM(d, n, 0.0, 1.0, u=u, tau=tau, bc=bc, precision=precision, staged=False, pdl=pdl)
    X = W.node_coords(d, [n] * d, 0.0, sim.dx, halfway=halfway)
    F = W.fourier_field(d, 3, 7, 0.0, 1.0)
    sim.init(_t(F.value(X)), _t(F.grad(X)))
    if bc != "periodic":
        a, kap, th = F.wave_params()
        sim.set_boundary_wave(a, kap, th)
    sim.step(steps)
    out = [sim.get_state().clone(), sim.macro().clone()]
    sim.adjoint_seed(sim.macro().contiguous())
    sim.adjoint_step(adjoint)
    gphi, _, _ = sim.adjoint_grads(want_grad=False, want_R=False)
    out.append(gphi.clone())
    sim.close()
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("d,n,u,tau,precision,bc", [
    (3, 24, (0.1, 0.05, -0.1), 0.5, "fp64", "periodic"),
    (3, 24, (0.1, 0.05, -0.1), 0.8, "fp64", "periodic"),
    (2, 40, (0.1, 0.2), 1.2, "fp64", "periodic"),
    (4, 9, (0.05, 0.1, 0.08, 0.1), 0.5, "fp32dev", "periodic"),
    (2, 21, (0.1, 0.1), 0.5, "fp64", "fullway"),
    (3, 12, (0.01, 0.01, 0.01), 0.5, "fp64", "halfway"),
    (2, 20, (0.1, 0.1), 0.5, "fp32dev", "fullway"),
])
def test_pdl_is_bitwise_plain_ordering(d, n, u, tau, precision, bc):
    import torch

    if precision == "fp32dev" and bc != "periodic":
        # the FP32-deviation adjoint is not offered on Dirichlet boxes: compare the forward only
        sims = []
        for pdl in (True, False):
            sim = LBM(d, n, 0.0, 1.0, u=u, tau=tau, bc=bc, precision=precision, pdl=pdl)
            X = W.node_coords(d, [n] * d, 0.0, sim.dx, halfway=False)
            F = W.fourier_field(d, 3, 7, 0.0, 1.0)
            sim.init(_t(F.value(X)), _t(F.grad(X)))
            a, kap, th = F.wave_params()
            sim.set_boundary_wave(a, kap, th)
            sim.step(23)
            sims.append(sim.get_state().clone())
            sim.close()
        assert torch.equal(sims[0], sims[1])
        return
    a = _run(d, n, u, tau, precision, bc, True)
    b = _run(d, n, u, tau, precision, bc, False)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("precision,staged", [("fp64", False), ("fp32dev", True), ("fp32dev", False)])
def test_calls_of_one_step_chain_across_calls(precision, staged):
    """Consecutive calls of one handle chain their step kernels with programmatic dependent launch
    (the first kernel of a call too, when the library's last step kernels on the stream were this
    handle's). Calls of one step, interleaved with another handle's steps on the same stream, with
    macro and diagnostics reads and with an adjoint pass, must give the bits of the same calls with
    plain stream ordering."""
    import torch

    n = (32, 12, 10)
    X = W.node_coords(3, list(n), 0.0, 1.0 / 32)
    F = W.fourier_field(3, 3, 9, 0.0, [ni / 32.0 for ni in n])
    phi0, grad = _t(F.value(X)), _t(F.grad(X))

    def run(pdl):
        kw = dict(u=(0.1, -0.05, 0.08), tau=0.8, precision=precision, staged=staged, pdl=pdl)
        a = LBM(3, list(n), 0.0, [ni / 32.0 for ni in n], **kw)
        b = LBM(3, list(n), 0.0, [ni / 32.0 for ni in n], **kw)
        for s in (a, b):
            s.init(phi0, grad)
        reads = []
        for i in range(12):
            a.step(1)
            if i % 3 == 0:
                b.step(1)
            if i % 4 == 1:
                reads.append(a.macro().clone())
            if i == 7:
                reads.append(torch.tensor(a.diagnostics()["mass"]))
        a.adjoint_seed(a.macro().contiguous())
        for _ in range(5):
            a.adjoint_step(1)
        gphi, _, _ = a.adjoint_grads(want_grad=False, want_R=False)
        out = [a.get_state().clone(), b.get_state().clone(), gphi.clone()] + reads
        a.close()
        b.close()
        torch.cuda.synchronize()
        return out

    for x, y in zip(run(True), run(False)):
        assert torch.equal(x, y)
