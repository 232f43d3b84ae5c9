"""Pins of the oracle's lattice and equilibrium against what the paper prints and what the
mathematics fixes (Sec. 2.3, Sec. 3.1, Sec. 4.1 of arXiv:2410.13165)."""
import itertools
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_velocities_match_the_printed_d2q9_d3q19():
    rows = {}
    with open(os.path.join(GOLDEN, "velocities_d2q9_d3q19.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                lat, comp, *vals = line.split()
                rows[(lat, comp)] = [int(v) for v in vals]
    e2 = O.velocities(2)
    assert e2[:, 0].tolist() == rows[("D2Q9", "x1")]
    assert e2[:, 1].tolist() == rows[("D2Q9", "x2")]
    e3 = O.velocities(3)
    for i, c in enumerate(("x1", "x2", "x3")):
        assert e3[:, i].tolist() == rows[("D3Q19", c)]


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_velocity_set_structure(d):
    e = O.velocities(d)
    Q = e.shape[0]
    assert Q == 2 * d * d + 1
    assert len({tuple(r) for r in e}) == Q                       # distinct
    assert all(tuple(-r) in {tuple(x) for x in e} for r in e)    # closed under c -> -c
    assert np.all(np.abs(e).sum(axis=1) <= 2)                    # rest, axis, 2-axis diagonals
    # every velocity with at most two unit components, and no other: the DdQ(2d^2+1) set
    want = {tuple([0] * d)}
    for i in range(d):
        for s in (1, -1):
            v = [0] * d
            v[i] = s
            want.add(tuple(v))
    for i, j in itertools.combinations(range(d), 2):
        for si, sj in itertools.product((1, -1), repeat=2):
            v = [0] * d
            v[i], v[j] = si, sj
            want.add(tuple(v))
    assert {tuple(r) for r in e} == want


def _stable_sigmas(d, rng, n=6):
    out = []
    while len(out) < n:
        s = rng.uniform(-0.3, 0.3, d) * (1.0 if d <= 3 else 0.5)
        if O.weights_closed(d, s, O.m4_rule(d, s)).min() > 0:
            out.append(s)
    return out


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5])
def test_closed_form_weights_equal_the_moment_solve(d):
    """Eq. (omega_k-2) against omega = M^{-1} eps with M the natural-moment matrix."""
    rng = np.random.default_rng(2410 + d)
    for s in _stable_sigmas(d, rng) + [np.zeros(d)]:
        m4 = O.m4_rule(d, s, 0.5)
        wc = O.weights_closed(d, s, m4)
        ws = O.weights_solve(d, s, m4)
        assert np.max(np.abs(wc - ws)) < 5e-15


@pytest.mark.parametrize("d", [2, 3, 4, 5])
def test_closed_form_weights_have_the_prescribed_moments(d):
    """Sum omega = 1, sum omega c = sigma, second/third/fourth moments = Eq. (third-condition-2),
    evaluated directly on the velocity set (independent of the moment-matrix ordering)."""
    rng = np.random.default_rng(7 + d)
    e = O.velocities(d).astype(float)
    for s in _stable_sigmas(d, rng, 3):
        npairs = d * (d - 1) // 2
        m4 = rng.uniform(0.05, 0.1, npairs)          # arbitrary per-pair fourth moments
        w = O.weights_closed(d, s, m4)
        assert abs(w.sum() - 1.0) < 1e-15
        assert np.allclose(w @ e, s, atol=1e-15, rtol=0)
        for i in range(d):
            assert abs(w @ e[:, i] ** 2 - (1 + 2 * s[i] ** 2) / 3) < 1e-15
            assert abs(w @ e[:, i] ** 3 - s[i]) < 1e-15
        p = 0
        for i in range(d):
            for j in range(d):
                if i != j:
                    assert abs(w @ (e[:, i] ** 2 * e[:, j]) - s[j] / 3) < 1e-15
                if j > i:
                    assert abs(w @ (e[:, i] * e[:, j]) - 2 * s[i] * s[j] / 3) < 1e-15
        for i, j in itertools.combinations(range(d), 2):
            assert abs(w @ (e[:, i] ** 2 * e[:, j] ** 2) - m4[p]) < 1e-15
            p += 1
        for i, j, l in itertools.combinations(range(d), 3):
            assert abs(w @ (e[:, i] * e[:, j] * e[:, l])) < 1e-15


def test_d1q3_weights_match_remark_4():
    for s in np.linspace(-0.49, 0.49, 11):
        w = O.weights_closed(1, [s], 0.0)
        assert np.allclose(w, [(2 - 2 * s * s) / 3, s / 2 + (2 * s * s + 1) / 6, -s / 2 + (2 * s * s + 1) / 6],
                           atol=1e-15)


def test_2d_entropy_region_is_the_square_of_half_width():
    """Remark 4: in 2D the model is entropy stable (all omega_k > 0 for some m4) iff |sigma_i| < 1/2;
    with the g = 1/2 rule of Eq. (meq-4rd) the weights are positive exactly there."""
    grid = np.linspace(-0.7, 0.7, 57)
    for s1 in grid:
        for s2 in grid:
            if min(abs(abs(s1) - 0.5), abs(abs(s2) - 0.5)) < 0.02:
                continue
            s = np.array([s1, s2])
            inside = max(abs(s1), abs(s2)) < 0.5
            assert (O.weights_closed(2, s, O.m4_rule(2, s)).min() > 0) == inside, (s1, s2)


@pytest.mark.parametrize("d", [3, 4, 5])
def test_entropy_region_matches_the_m4_bounds(d):
    """Eq. (region-d>=3): positivity of every omega_k under the g-rule iff max(lower) < min(upper);
    the bounds are evaluated from Eq. (entropy-stable-condition) with equal fourth moments."""
    rng = np.random.default_rng(99 + d)
    for _ in range(400):
        s = rng.uniform(-0.5, 0.5, d)
        m4lo, m4hi = O.m4_rule(d, s, 1.0), O.m4_rule(d, s, 0.0)
        if abs(m4hi - m4lo) < 1e-9:
            continue
        pos = O.weights_closed(d, s, O.m4_rule(d, s, 0.5)).min() > 0
        assert pos == (m4lo < m4hi)


def test_4d_velocity_04_is_not_entropy_stable():
    """Example 3: u = 0.4 (1,1,1,1) violates the entropy-stability conditions."""
    s = np.full(4, 0.4)
    assert O.m4_rule(4, s, 1.0) > O.m4_rule(4, s, 0.0)
    assert O.weights_closed(4, s, O.m4_rule(4, s)).min() < 0
    for u in (0.2, 0.1, 0.05):
        s = np.full(4, u)
        assert O.weights_closed(4, s, O.m4_rule(4, s)).min() > 0


def test_at_rest_the_admissible_m4_interval_shrinks_with_d():
    """Eq. (sigma=0): at sigma = 0 the fourth-moment interval is ((d-3)/(3 d(d-1)/2), 1/(3(d-1)))
    and it is non-empty for d < 6; its width decreases with d."""
    widths = []
    for d in range(2, 6):
        lo, hi = O.m4_rule(d, np.zeros(d), 1.0), O.m4_rule(d, np.zeros(d), 0.0)
        assert lo < hi
        widths.append(hi - lo)
    assert all(a > b for a, b in zip(widths, widths[1:]))
    # d = 6 (outside the oracle's range) would give 2(6-3)/(3*30) = 1/15 = 1/(3*5): empty.
    assert abs(2 * (6 - 3) / (3 * 6 * 5) - 1 / (3 * 5)) < 1e-15
