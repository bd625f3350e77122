"""Pins of the oracle's bounding functions and priors (App. C), and of the
host-side prior set-up helpers (CPU only)."""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, stats

from oracle import hmc as H
from oracle import sps as O
from paper_2506_19919_gb300 import priors as P

LO = np.array([-1.5, 0.5, 0.1, 0.1, 0.0, 6.0, 0.05, -2.0, 0.05, 0.0, -1.0, 0.0])
HI = np.array([2.5, 12.0, 5.0, 5.0, 0.2, 8.5, 1.5, 0.2, 0.5, 3.0, 0.4, 0.5])


def _lp1(x, **kw):
    """Oracle log prior of one parameter at the points x."""
    return O.log_prior_unbounded(torch.as_tensor(np.asarray(x, np.float64))[:, None], **kw).numpy()


@pytest.mark.parametrize("xi,om,s", [(0.3, 1.7, 4.0), (-1.0, 0.4, -2.5), (2.0, 3.0, 0.0)])
def test_skew_normal_density_is_scipys(xi, om, s):
    x = np.concatenate([np.linspace(xi - 12 * om, xi + 12 * om, 401), [xi - 40 * om]])
    lp = _lp1(x, skew=([xi], [om], [s]))
    ref = stats.skewnorm.logpdf(x, s, loc=xi, scale=om)
    fin = np.isfinite(ref)
    np.testing.assert_allclose(lp[fin], ref[fin], rtol=1e-10, atol=1e-10)
    assert np.isfinite(lp).all()                       # far tail stays finite (log Phi)
    if s == 0.0:
        np.testing.assert_allclose(lp, stats.norm.logpdf(x, xi, om), rtol=1e-12)
    tot, _ = integrate.quad(lambda v: math.exp(_lp1([v], skew=([xi], [om], [s]))[0]), -np.inf, np.inf)
    assert abs(tot - 1.0) < 1e-8


@pytest.mark.parametrize("k,x0", [(1.0, 0.0), (2.5, -0.7), (0.3, 1.5)])
def test_tuned_bounding_map(k, x0):
    lo, hi = 6.0, 8.5
    x = torch.linspace(-6.0, 6.0, 97, dtype=torch.float64)
    th = O.bound(x, lo, hi, k, x0).numpy()
    assert np.all(np.diff(th) > 0) and th.min() > lo and th.max() < hi
    assert float(O.bound(torch.tensor(x0, dtype=torch.float64), lo, hi, k, x0)) == pytest.approx(7.25, abs=1e-14)
    h = 1e-6
    slope = float(O.bound(torch.tensor(x0 + h, dtype=torch.float64), lo, hi, k, x0)
                  - O.bound(torch.tensor(x0 - h, dtype=torch.float64), lo, hi, k, x0)) / (2 * h)
    assert slope == pytest.approx((hi - lo) * k / 4.0, rel=1e-8)
    # the uniform prior's log density is the logistic density up to log k
    tot, _ = integrate.quad(lambda v: math.exp(_lp1([v], k=k, x0=x0)[0]), -np.inf, np.inf)
    assert tot == pytest.approx(1.0 / k, rel=1e-8)
    # theta uniform => x = F_B^-1(theta) has CDF sigma(k (x - x0))
    u = np.random.default_rng(1).uniform(size=20000)
    xs = x0 + np.log(u / (1 - u)) / k
    assert stats.kstest(xs, lambda v: 1.0 / (1.0 + np.exp(-k * (v - x0)))).pvalue > 1e-3


class _SkewPrior:
    """The skew-normal prior alone, as the HMC target (no band observed)."""

    def __init__(self, xi, om, s):
        self.skew = (xi, om, s)
        self.lo = torch.as_tensor(LO)
        self.hi = torch.as_tensor(HI)

    def __call__(self, x, rows):
        xt = torch.as_tensor(np.asarray(x)).clone().requires_grad_(True)
        lp = O.log_prior_unbounded(xt, skew=self.skew)
        (g,) = torch.autograd.grad(lp.sum(), xt)
        return lp.detach().numpy(), g.numpy()


def test_hmc_samples_the_skew_normal_prior():
    """With no data the sampler draws the skew-normal prior itself: pins the
    prior's log density and its gradient inside the sampler."""
    rng = np.random.default_rng(2)
    xi, om, s = rng.normal(0, 1, 12), rng.uniform(0.5, 2.0, 12), rng.uniform(-5, 5, 12)
    C = 32
    out = H.run_hmc(_SkewPrior(xi, om, s), rng.normal(size=(C, 12)), np.zeros(C, int), seed=3, n_warm=100,
                    n_samp=200, L_min=4, L_max=12)
    th = out["samples"].reshape(-1, 12)
    x = np.log((th - LO) / (HI - th))                  # back to unbounded space (k = 1, x0 = 0)
    for k in range(12):
        assert stats.kstest(x[::5, k], stats.skewnorm(s[k], loc=xi[k], scale=om[k]).cdf).pvalue > 1e-4


def test_tune_sigmoid_maps_the_unit_interval_onto_the_expected_range():
    a = LO + 0.3 * (HI - LO)
    b = LO + 0.6 * (HI - LO)
    k, x0 = P.tune_sigmoid(LO, HI, a, b)
    np.testing.assert_allclose(O.bound(torch.full((12,), -1.0, dtype=torch.float64), LO, HI, k, x0).numpy(), a,
                               rtol=1e-12)
    np.testing.assert_allclose(O.bound(torch.full((12,), 1.0, dtype=torch.float64), LO, HI, k, x0).numpy(), b,
                               rtol=1e-12)
    th = LO + np.random.default_rng(4).uniform(0.01, 0.99, (50, 12)) * (HI - LO)
    np.testing.assert_allclose(O.bound(torch.as_tensor(P.unbound(th, LO, HI, k, x0)), LO, HI, k, x0).numpy(), th,
                               rtol=1e-12)
    with pytest.raises(ValueError):
        P.tune_sigmoid(LO, HI, b, a)


def test_fit_skew_normal_recovers_parameters():
    truth = [(0.5, 1.3, 3.0), (-2.0, 0.7, -1.5), (1.0, 2.0, 0.0)]
    x = np.stack([stats.skewnorm.rvs(s, loc=xi, scale=om, size=400_000, random_state=i)
                  for i, (xi, om, s) in enumerate(truth)], axis=1)
    xi, om, s = P.fit_skew_normal(x)
    ref = [stats.skewnorm.fit(x[:20_000, j], c, loc=a, scale=b) for j, (a, b, c) in enumerate(truth)]
    for j, (a, b, c) in enumerate(truth):
        grid = np.linspace(a - 4 * b, a + 4 * b, 801)
        fit = stats.skewnorm.cdf(grid, s[j], loc=xi[j], scale=om[j])
        assert np.abs(fit - stats.skewnorm.cdf(grid, c, loc=a, scale=b)).max() < 3e-3
        assert np.abs(fit - stats.skewnorm.cdf(grid, ref[j][0], loc=ref[j][1], scale=ref[j][2])).max() < 1e-2
        if c != 0.0:                                   # well-determined shape
            assert xi[j] == pytest.approx(a, abs=0.03) and om[j] == pytest.approx(b, rel=0.02)
            assert s[j] == pytest.approx(c, rel=0.1)
    # the paper's recipe: Gaussian-ish draws of theta inside the bounds
    rng = np.random.default_rng(5)
    th = np.clip(rng.normal(0.5 * (LO + HI), 0.15 * (HI - LO), (100_000, 12)), LO + 1e-6 * (HI - LO),
                 HI - 1e-6 * (HI - LO))
    xi, om, s = P.skew_normal_prior(th, LO, HI)
    assert np.isfinite(xi).all() and (om > 0).all() and np.isfinite(s).all()
