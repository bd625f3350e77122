"""Pins of the HMC and diagnostics oracle (CPU only)."""
import math

import numpy as np
import pytest
import torch
from scipy import stats

import sps_workloads as W
from oracle import diagnostics as D
from oracle import hmc as H


def test_philox_words_are_uniform_and_decorrelated():
    n = 50_000
    ctr = np.zeros((n, 4), np.uint64)
    ctr[:, 0] = np.arange(n)
    key = np.tile(np.array([12345, 678], np.uint64), (n, 1))
    w = H.philox4x32_10(ctr, key)
    assert w.max() < 2 ** 32
    u = H.uniform01(w).ravel()
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # neighbouring counters give uncorrelated outputs
    a = H.uniform01(w[:-1, 0])
    b = H.uniform01(w[1:, 0])
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.02
    # one flipped counter bit changes about half of the 128 output bits
    ctr2 = ctr.copy()
    ctr2[:, 1] ^= np.uint64(1)
    w2 = H.philox4x32_10(ctr2, key)
    flips = np.unpackbits((w ^ w2).astype(">u4").view(np.uint8)).reshape(n, -1).sum(1)
    assert abs(flips.mean() - 64.0) < 0.5


def _triton_philox(keys, ctrs):
    """Philox-4x32-10 words from Triton's implementation of the generator,
    run by its CPU interpreter in a child process (see philox_triton_ref)."""
    import json
    import os
    import subprocess
    import sys
    pytest.importorskip("triton")
    here = os.path.dirname(os.path.abspath(__file__))
    job = json.dumps({"keys": [[int(a) for a in k] for k in keys],
                      "ctrs": [[int(a) for a in c] for c in ctrs]})
    r = subprocess.run([sys.executable, os.path.join(here, "philox_triton_ref.py")],
                       input=job, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return np.asarray(json.loads(r.stdout), dtype=np.uint64).reshape(len(keys), len(ctrs), 4)


def _philox_disagreement(keys, ctrs, ref):
    out = np.stack([H.philox4x32_10(np.asarray(ctrs, np.uint64),
                                    np.tile(np.asarray(k, np.uint64), (len(ctrs), 1)))
                    for k in keys])
    return int((out != ref).sum())


def test_philox_matches_an_independent_implementation(monkeypatch):
    """The oracle's Philox-4x32-10 equals, word for word, the generator as
    Triton implements it (run on the CPU by Triton's interpreter), on the
    all-zero and all-ones counter and key and on 256 random counters under
    four random keys.  A wrong multiplier, Weyl key increment or output
    word order, planted in the oracle, changes the words."""
    rng = np.random.default_rng(20110101)
    M = 0xFFFFFFFF
    ctrs = np.concatenate([[[0, 0, 0, 0], [M, M, M, M]],
                           rng.integers(0, 2 ** 32, (254, 4), dtype=np.uint64)])
    keys = np.concatenate([[[0, 0], [M, M]], rng.integers(0, 2 ** 32, (4, 2), dtype=np.uint64)])
    ref = _triton_philox(keys, ctrs)
    assert _philox_disagreement(keys, ctrs, ref) == 0
    for name, val in (("PHILOX_M0", H.PHILOX_M0 ^ 4), ("PHILOX_M1", H.PHILOX_M1 + 2),
                      ("PHILOX_W0", H.PHILOX_W0 + 1), ("PHILOX_W1", H.PHILOX_W1 ^ 0x100)):
        with monkeypatch.context() as m:
            m.setattr(H, name, val)
            assert _philox_disagreement(keys, ctrs, ref) > 0.9 * ref.size
    swapped = H.philox4x32_10
    with monkeypatch.context() as m:
        m.setattr(H, "philox4x32_10", lambda c, k: swapped(c, k)[..., [1, 0, 3, 2]])
        assert _philox_disagreement(keys, ctrs, ref) > 0.9 * ref.size


def test_philox_weyl_increments_from_their_definition():
    """Salmon et al. (2011) bump the Philox key by the golden ratio and by
    sqrt(3) - 1, each as a 32-bit fixed-point fraction."""
    import decimal
    decimal.getcontext().prec = 60
    phi = (1 + decimal.Decimal(5).sqrt()) / 2
    s3 = decimal.Decimal(3).sqrt()
    assert H.PHILOX_W0 == int((phi - 1) * (1 << 32))
    assert H.PHILOX_W1 == int((s3 - 1) * (1 << 32))


def test_momentum_and_length_draws():
    p, u, L = H.draws(99, np.arange(4000), 3, 8, 64)
    assert p.shape == (4000, 12)
    assert stats.kstest(p.ravel(), "norm").pvalue > 1e-3
    assert (u > 0).all() and (u < 1).all()
    assert L.min() == 8 and L.max() == 64
    counts = np.bincount(L - 8, minlength=57)
    assert stats.chisquare(counts).pvalue > 1e-3
    # counter-based: a chain's draws do not depend on which other chains run
    p1, _, L1 = H.draws(99, np.array([17]), 3, 8, 64)
    np.testing.assert_array_equal(p1[0], p[17])
    assert L1[0] == L[17]


class _Uniform:
    """Prior-only target: uniform in theta on [0, 1] => logistic in the
    unbounded coordinate (Eq. BoundingFunction with k = 1, x0 = 0)."""
    lo = torch.zeros(12, dtype=torch.float64)
    hi = torch.ones(12, dtype=torch.float64)

    def __call__(self, x, rows):
        x = np.asarray(x)
        lp = -(np.abs(x) + 2 * np.log1p(np.exp(-np.abs(x)))).sum(1)
        g = 1.0 - 2.0 / (1.0 + np.exp(-x))
        return lp, g


def test_hmc_samples_the_prior_when_no_band_is_observed():
    """With no data the posterior is the prior, uniform in each bounded
    parameter: checks detailed balance and the adaptation, independently
    of the oracle's photometry."""
    C = 64
    x0 = np.random.default_rng(0).normal(0, 2, size=(C, 12))
    out = H.run_hmc(_Uniform(), x0, np.zeros(C, int), seed=7, n_warm=150, n_samp=150,
                    L_min=4, L_max=12, adapt_mass=True)
    s = out["samples"].reshape(-1, 12)
    for k in range(12):
        assert stats.kstest(s[::7, k], "uniform").pvalue > 1e-4
    assert abs(s.mean() - 0.5) < 0.01
    assert abs(s.var() - 1 / 12) < 0.004
    # dual averaging drives the warm-up mean acceptance to its target; the
    # averaged step size used afterwards is smaller, so acceptance rises
    assert abs(out["warm_accept"].mean() - 0.8) < 0.03
    assert out["accept_prob"].mean() > out["warm_accept"].mean()


def _sps_target(n_gal=2):
    wl = W.config(3, n_gal=n_gal)
    from oracle import sps as O
    th = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    mobs = O.photometry(th, wl.z, wl.tables, "approx").numpy() + wl.noise
    t = H.ApproxTarget(wl.tables, wl.z, mobs, wl.sigma, wl.mask, W.PRIOR_LO, W.PRIOR_HI)
    x0 = W.unbounded_of(wl.theta_true)
    return t, x0


def test_leapfrog_is_reversible_and_second_order():
    t, x0 = _sps_target()
    rows = np.arange(2)
    lp0, g0 = t(x0, rows)
    p0 = np.random.default_rng(1).normal(size=x0.shape)
    L = np.array([10, 10])
    x1, p1, g1, lp1 = H.leapfrog(t, rows, x0, p0, g0, np.full(2, 1e-3), L)
    x2, p2, _, _ = H.leapfrog(t, rows, x1, -p1, g1, np.full(2, 1e-3), L)
    np.testing.assert_allclose(x2, x0, atol=1e-9)
    np.testing.assert_allclose(-p2, p0, atol=1e-7)
    # energy error shrinks ~ eps^2 at fixed trajectory length
    dh = []
    for eps, n in ((4e-4, 10), (2e-4, 20)):
        x1, p1, _, lp1 = H.leapfrog(t, rows, x0, p0, g0, np.full(2, eps), np.array([n, n]))
        dh.append(np.abs((-lp1 + 0.5 * (p1 * p1).sum(1)) - (-lp0 + 0.5 * (p0 * p0).sum(1))))
    ratio = dh[0] / dh[1]
    assert ((ratio > 3.0) & (ratio < 5.0)).all()


def test_ess_and_rhat_pins():
    rng = np.random.default_rng(3)
    iid = rng.normal(size=(4, 2000))
    assert D.ess(iid) == pytest.approx(8000, rel=0.1)
    assert D.split_rhat(iid) < 1.01
    rho = 0.9
    ar = np.zeros((4, 4000))
    e = rng.normal(size=(4, 4000))
    for t in range(1, 4000):
        ar[:, t] = rho * ar[:, t - 1] + math.sqrt(1 - rho ** 2) * e[:, t]
    assert D.ess(ar) == pytest.approx(16000 * (1 - rho) / (1 + rho), rel=0.25)
    shifted = iid + np.arange(4)[:, None]
    assert D.split_rhat(shifted) > 1.2
    tot, per = D.posteriors_at_ess(np.stack([iid.T, iid.T[::-1]], 0).reshape(2, 2000, 4)
                                   .transpose(0, 1, 2), chains_per_gal=1)
    assert tot == pytest.approx(2.0)


def test_warmup_windows_schedule():
    # 75 / 25, 50, 100, 200 / 50 for 500 warm-up iterations; shorter warm-ups
    # split 15% / 75% / 10%
    assert H.warmup_windows(500) == (75, [(75, 100), (100, 150), (150, 250), (250, 450)], 450)
    init, wins, term = H.warmup_windows(100)
    assert (init, term) == (15, 90) and wins[0][0] == 15 and wins[-1][1] == 90


class _Gauss:
    """Independent Gaussians with scales spanning three decades."""
    scale = np.array([0.01, 0.03, 0.1, 0.3, 1.0, 3.0, 0.02, 0.05, 0.2, 0.5, 2.0, 1.5])
    lo = torch.full((12,), -1e9, dtype=torch.float64)
    hi = torch.full((12,), 1e9, dtype=torch.float64)

    def __call__(self, x, rows):
        z = np.asarray(x) / self.scale
        return -0.5 * (z * z).sum(1), -z / self.scale


def test_metric_adaptation_learns_the_scales():
    C = 16
    x0 = np.random.default_rng(2).normal(size=(C, 12)) * _Gauss.scale
    out = H.run_hmc(_Gauss(), x0, np.zeros(C, int), seed=3, n_warm=300, n_samp=10, L_min=4,
                    L_max=12, adapt_mass=True)
    ratio = out["minv"] / _Gauss.scale ** 2
    assert np.median(ratio) == pytest.approx(1.0, rel=0.25)
    assert (ratio > 0.3).all() and (ratio < 3.0).all()
    # the adapted step size is set by the metric, not by the narrowest scale
    assert np.median(out["eps"]) > 0.2


class _CorrGauss:
    """A strongly correlated Gaussian (correlation 0.99 between pairs)."""
    lo = torch.full((12,), -1e9, dtype=torch.float64)
    hi = torch.full((12,), 1e9, dtype=torch.float64)
    cov = np.eye(12)
    for i in range(0, 12, 2):
        cov[i:i + 2, i:i + 2] = [[1.0, 0.99], [0.99, 1.0]]
    prec = np.linalg.inv(cov)

    def __call__(self, x, rows):
        x = np.asarray(x)
        return -0.5 * np.einsum("ci,ij,cj->c", x, self.prec, x), -x @ self.prec


def test_dense_metric_learns_the_covariance():
    C = 16
    x0 = np.random.default_rng(4).normal(size=(C, 12))
    out = H.run_hmc(_CorrGauss(), x0, np.zeros(C, int), seed=5, n_warm=300, n_samp=10, L_min=4,
                    L_max=12, adapt_mass=True, metric="dense")
    cov = np.einsum("cij,ckj->cik", out["chol"], out["chol"]).mean(0)
    np.testing.assert_allclose(cov, _CorrGauss.cov, atol=0.25)
    # the step size is no longer limited by the narrow direction (sd 0.1)
    assert np.median(out["eps"]) > 0.4
    diag = H.run_hmc(_CorrGauss(), x0, np.zeros(C, int), seed=5, n_warm=300, n_samp=10, L_min=4,
                     L_max=12, adapt_mass=True, metric="diag")
    assert np.median(out["eps"]) > 3 * np.median(diag["eps"])


def test_exact_target_is_the_oracle_exact_posterior():
    """ExactTarget (band weights computed once per galaxy) gives the same log
    posterior and gradient as the oracle's exact photometry evaluated afresh."""
    from oracle import sps as O
    wl = W.config(1, n_gal=3)
    mobs = O.photometry(wl.theta_true, wl.z, wl.tables, "exact").numpy() + wl.noise
    t = H.ExactTarget(wl.tables, wl.z, mobs, wl.sigma, wl.mask, W.PRIOR_LO, W.PRIOR_HI)
    x = W.unbounded_of(W.prior_draw(np.random.default_rng(4), 3))
    lp, g = t(x, np.arange(3))
    lp2, g2 = O.logpost_and_grad_unbounded(x, wl.z, wl.tables, mobs, wl.sigma, wl.mask, W.PRIOR_LO,
                                           W.PRIOR_HI, mode="exact")
    np.testing.assert_allclose(lp, lp2.numpy(), rtol=1e-13)
    np.testing.assert_allclose(g, g2.numpy(), rtol=1e-11, atol=1e-11 * np.abs(g2.numpy()).max())
