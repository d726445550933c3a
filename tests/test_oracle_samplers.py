"""Pins of the oracle's random numbers, lobe samplers and lobe masses against
sources other than the oracle itself: published Philox known-answer vectors,
an independent Lambert W (scipy), the CDF landmarks the paper states,
numerical quadrature of the kernels, and goodness-of-fit of drawn samples."""
import math

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle as O
from conftest import read_golden


def test_philox_known_answers():
    for row in read_golden("philox4x32_10_kat.txt"):
        vals = [int(x, 16) for x in row]
        out = O.philox(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_u01_open_interval_and_midpoints():
    assert O.u01(0) == 0.5 * 2.0 ** -32
    assert O.u01(0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -32
    assert O.u01(0x80000000) == 0.5 + 0.5 * 2.0 ** -32


@pytest.mark.parametrize("branch", [0, -1])
def test_lambertw_matches_scipy_away_from_branch_point(branch):
    zs = -np.exp(-1) * (1 - np.logspace(-6, 0, 60, endpoint=False))
    zs = np.concatenate([zs, -np.logspace(-30, -1, 40)])
    for z in zs:
        p = math.sqrt(max(0.0, 2 * (1 + math.e * z)))
        w = O.lambertw(z, branch)
        ref = special.lambertw(z, branch).real
        if p > 1e-3:
            assert abs(w - ref) <= 1e-13 * max(1.0, abs(ref)), (z, branch, w, ref)
        # defining equation everywhere, including next to the branch point
        assert abs(w * math.exp(w) - z) <= 1e-15 + 1e-13 * abs(z)
        assert (w >= -1.0) if branch == 0 else (w <= -1.0)


def test_diag_cdf_landmarks():
    # CDF values 1/4, 1/2, 3/4 at -sigma, 0, +sigma (Suppl. "Sampling diagonal
    # of Hessian": scaled so that the CDF is 1/4 at -sigma)
    assert O.diag_cdf(-1.0) == pytest.approx(0.25, abs=1e-15)
    assert O.diag_cdf(0.0) == 0.5
    assert O.diag_cdf(1.0) == pytest.approx(0.75, abs=1e-15)
    assert O.diag_cdf(-40.0) == pytest.approx(0.0, abs=1e-300)
    assert O.diag_cdf(40.0) == pytest.approx(1.0, abs=1e-15)
    # continuity at +-1 and monotonicity
    for t0 in (-1.0, 1.0):
        assert abs(O.diag_cdf(t0 - 1e-9) - O.diag_cdf(t0 + 1e-9)) < 1e-8
    ts = np.linspace(-8, 8, 4001)
    c = np.array([O.diag_cdf(t) for t in ts])
    assert np.all(np.diff(c) >= 0)


def test_diag_cdf_is_integral_of_normalised_abs_second_derivative():
    # d/dt of the CDF equals |phi''(t)| / Z_d with sigma = 1, Z_d = 4 phi(1)
    phi = lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)
    Zd = 4 * phi(1.0)
    for t in (-3.0, -1.5, -0.5, 0.2, 0.9, 1.3, 2.5):
        lhs = (O.diag_cdf(t + 1e-6) - O.diag_cdf(t - 1e-6)) / 2e-6
        rhs = abs(t * t - 1) * phi(t) / Zd
        assert lhs == pytest.approx(rhs, rel=1e-6, abs=1e-12)
    # and the quadrature of that density reproduces the CDF
    for t in (-2.0, -1.0, 0.3, 1.7):
        pts = [x for x in (-1.0, 1.0) if -40.0 < x < t]
        val, _ = integrate.quad(lambda x: abs(x * x - 1) * phi(x) / Zd, -40.0, t, points=pts or None, limit=200)
        assert val == pytest.approx(O.diag_cdf(t), abs=1e-10)


def test_diag_inverse_cdf_round_trip():
    cs = np.concatenate([np.linspace(1e-12, 1 - 1e-12, 2001), [0.25, 0.75, 0.5, 0.25 - 1e-12, 0.75 + 1e-12]])
    for c in cs:
        t = O.diag_inv_cdf(c)
        assert abs(O.diag_cdf(t) - c) <= 2e-14, (c, t)
    assert O.diag_inv_cdf(0.25) == pytest.approx(-1.0, abs=1e-7)
    assert O.diag_inv_cdf(0.75) == pytest.approx(1.0, abs=1e-7)


@pytest.mark.parametrize("sigma", [0.05, 0.1, 1.0, 2.5])
def test_lobe_masses_by_quadrature(sigma):
    n1 = lambda x: math.exp(-0.5 * x * x / sigma ** 2) / (sigma * math.sqrt(2 * math.pi))
    L = 40 * sigma
    zg, _ = integrate.quad(lambda x: abs(x) / sigma ** 2 * n1(x), -L, L, points=[0.0], epsabs=0, epsrel=1e-13)
    zd, _ = integrate.quad(lambda x: abs(x * x - sigma ** 2) / sigma ** 4 * n1(x), -L, L,
                           points=[-sigma, sigma], limit=200, epsabs=0, epsrel=1e-13)
    assert O.Zg(sigma) == pytest.approx(zg, rel=1e-10)
    assert O.Zd(sigma) == pytest.approx(zd, rel=1e-10)
    assert O.Zo(sigma) == pytest.approx(zg * zg, rel=1e-10)
    # closed forms: sqrt(2/pi)/sigma, 4 e^-1/2 / (sqrt(2 pi) sigma^2)
    assert O.Zg(sigma) == pytest.approx(math.sqrt(2 / math.pi) / sigma, rel=1e-14)
    assert O.Zd(sigma) == pytest.approx(4 * math.exp(-0.5) / (math.sqrt(2 * math.pi) * sigma ** 2), rel=1e-14)


def _ks(samples, cdf):
    return stats.kstest(samples, cdf).pvalue


def test_diagonal_lobe_samples_follow_their_lobes():
    sigma, P = 0.7, 20000
    tau, comp = O.draw(1, 3, sigma, P, seed=11, request=5, sub=0, comp_i=1, comp_j=1)
    tp, tm = tau[0::2, 1] / sigma, tau[1::2, 1] / sigma
    # + lobe: tails |t| > 1, CDF restricted to (0,1/4) u (3/4,1) renormalised
    assert np.all(np.abs(tp) > 1 - 1e-6) and np.all(np.abs(tm) < 1 + 1e-6)
    cdf_p = lambda t: np.where(t < 0, 2 * np.vectorize(O.diag_cdf)(t),
                               2 * (np.vectorize(O.diag_cdf)(t) - 0.5))
    cdf_m = lambda t: 2 * (np.vectorize(O.diag_cdf)(t) - 0.25)
    assert _ks(tp, cdf_p) > 1e-3
    assert _ks(tm, cdf_m) > 1e-3
    # other dims: N(0, sigma^2), shared by both legs
    assert np.array_equal(tau[0::2, 0], tau[1::2, 0])
    assert _ks(tau[0::2, 0] / sigma, stats.norm.cdf) > 1e-3
    assert _ks(tau[0::2, 2] / sigma, stats.norm.cdf) > 1e-3


def test_gradient_and_offdiagonal_lobes():
    sigma, P = 0.3, 20000
    tau, _ = O.draw(0, 2, sigma, P, seed=3, request=1, sub=7, comp_i=0)
    r = tau[0::2, 0] / sigma
    assert np.all(r > 0) and np.array_equal(tau[1::2, 0], -tau[0::2, 0])
    assert _ks(r, stats.rayleigh.cdf) > 1e-3           # half-Rayleigh = |N'| lobe
    tau, _ = O.draw(1, 2, sigma, P, seed=3, request=1, sub=8, comp_i=0, comp_j=1)
    a, b = tau[0::2] / sigma, tau[1::2] / sigma
    assert np.all(np.sign(a[:, 0]) == np.sign(a[:, 1]))     # + lobe of tau_i tau_j
    assert np.all(np.sign(b[:, 0]) == -np.sign(b[:, 1]))    # - lobe
    assert np.array_equal(a[:, 0], b[:, 0])
    assert _ks(np.abs(a[:, 0]), stats.rayleigh.cdf) > 1e-3
    assert _ks(np.abs(a[:, 1]), stats.rayleigh.cdf) > 1e-3
    assert abs(np.mean(a[:, 0] > 0) - 0.5) < 0.02


def test_aggregate_component_choice_is_uniform_over_ordered_elements():
    n, P = 3, 36000
    _, comp = O.draw(1, n, 0.1, P, seed=9, request=2, sub=0)
    counts = np.bincount(comp, minlength=n * n)
    assert stats.chisquare(counts).pvalue > 1e-3
    _, comp = O.draw(0, 5, 0.1, P, seed=9, request=2, sub=0)
    assert stats.chisquare(np.bincount(comp, minlength=5)).pvalue > 1e-3


def test_counter_layout_separates_streams():
    a, _ = O.draw(1, 4, 0.1, 64, seed=1, request=1, sub=0)
    for kw in (dict(seed=2, request=1, sub=0), dict(seed=1, request=2, sub=0), dict(seed=1, request=1, sub=1)):
        b, _ = O.draw(1, 4, 0.1, 64, **kw)
        assert not np.any(np.all(a == b, axis=1))
    c, _ = O.draw(1, 4, 0.1, 64, seed=1, request=1, sub=0)
    assert np.array_equal(a, c)
