"""GPU stability maps (Sec. 4, Eq. (G)): the CUDA eigenvalue kernel against the oracle (numpy
eigenvalues of the moment-space amplification matrix), and the paper's finding that the microscopic
entropy region (every omega_k > 0) is the von Neumann L2 region."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2410_13165_gb300 import LHEError, build, stability_map
from paper_2410_13165_gb300 import _abi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    _abi.load()


@pytest.mark.parametrize("d,nxi,tau", [(1, 16, 0.5), (2, 12, 0.5), (2, 10, 0.8), (3, 6, 0.5), (4, 4, 0.5)])
def test_stability_map_matches_the_oracle(d, nxi, tau):
    rng = np.random.default_rng(100 + d)
    S = rng.uniform(-0.7, 0.7, size=({1: 12, 2: 30, 3: 12, 4: 4}[d], d))
    S[0], S[1] = 0.0, 0.05  # points inside the region (small in 4D)
    rho_g, om_g = stability_map(d, S, nxi, tau=tau)
    rho_o, om_o = O.stability_map(d, S, nxi, tau=tau)
    assert np.max(np.abs(om_g - om_o)) < 1e-15
    assert np.max(np.abs(rho_g - rho_o)) < 1e-10, np.max(np.abs(rho_g - rho_o))
    assert np.any(om_g < 0) and np.any(om_g > 0)


@pytest.mark.parametrize("d", [2, 3])
def test_entropy_region_equals_l2_region_on_the_gpu(d):
    if d == 2:
        g = np.round(np.arange(-0.8, 0.81, 0.05), 10)
        S = np.array([(a, b) for a in g for b in g])
        nxi = 24
    else:
        g = np.round(np.arange(-0.6, 0.61, 0.1), 10)
        S = np.array([(a, b, c) for a in g for b in g for c in (0.0, 0.2, 0.4)])
        nxi = 10
    rho, omin = stability_map(d, S, nxi)
    away = np.abs(omin) > 1e-12
    assert np.count_nonzero(away & (omin < 0)) > 20 and np.count_nonzero(away & (omin > 0)) > 20
    assert np.all((omin[away] > 0) == (rho[away] <= 1.0 + 1e-9))


def test_stability_map_error_paths():
    with pytest.raises(LHEError) as ei:
        stability_map(5, np.zeros((1, 5)), 4)
    assert ei.value.status == _abi.ERR_ARG
    with pytest.raises(LHEError) as ei:
        stability_map(2, np.zeros((1, 2)), 0)
    assert ei.value.status == _abi.ERR_ARG
    rho, omin = stability_map(2, np.zeros((0, 2)), 8)
    assert rho.shape == (0,)
