"""Convergence diagnostics for HMC output (TEST INFRASTRUCTURE ONLY).

The paper checks each fit with the Gelman-Rubin statistic (R-hat < 1.2,
Sec. 4).  This module restates split-R-hat and the multi-chain effective
sample size with Geyer's initial-monotone-sequence truncation, following
Gelman et al. (Bayesian Data Analysis, 3rd ed., Sec. 11.4-11.5).  The
autocovariance uses numpy's FFT (a library primitive)."""
from __future__ import annotations

import numpy as np


def _autocov(x):
    """Biased autocovariance of each row of x [M, N] at lags 0..N-1."""
    m, n = x.shape
    xc = x - x.mean(1, keepdims=True)
    nfft = 1 << (2 * n - 1).bit_length()
    f = np.fft.rfft(xc, nfft, axis=1)
    ac = np.fft.irfft(f * np.conj(f), nfft, axis=1)[:, :n]
    return ac / n


def ess(draws):
    """Multi-chain effective sample size of draws [M chains, N draws]."""
    x = np.asarray(draws, dtype=np.float64)
    m, n = x.shape
    if n < 4:
        return float(m * n)
    acov = _autocov(x)
    chain_var = acov[:, 0] * n / (n - 1.0)
    W = chain_var.mean()
    var_plus = W * (n - 1.0) / n
    if m > 1:
        var_plus += x.mean(1).var(ddof=1)
    if not np.isfinite(var_plus) or var_plus <= 0:
        return float(m * n)
    rho = 1.0 - (W - acov.mean(0)) / var_plus        # combined autocorrelation
    rho[0] = 1.0
    # Geyer: sum pairs P_k = rho_2k + rho_2k+1 while positive, monotone
    tau = -1.0
    prev = np.inf
    for k in range(0, n - 1, 2):
        pk = rho[k] + rho[k + 1]
        if pk < 0:
            break
        pk = min(pk, prev)
        prev = pk
        tau += 2.0 * pk
    tau = max(tau, 1.0 / np.log10(m * n))
    return float(m * n / tau)


def split_rhat(draws):
    """Split R-hat of draws [M, N] (each chain split into two halves)."""
    x = np.asarray(draws, dtype=np.float64)
    m, n = x.shape
    h = n // 2
    s = np.concatenate([x[:, :h], x[:, n - h:]], axis=0)
    mm, nn = s.shape
    W = s.var(1, ddof=1).mean()
    B = nn * s.mean(1).var(ddof=1)
    var_plus = (nn - 1.0) / nn * W + B / nn
    return float(np.sqrt(var_plus / W)) if W > 0 else np.inf


def posteriors_at_ess(samples, chains_per_gal, target=100.0):
    """sum_g min(1, ESS_g / target), ESS_g = min over parameters of the
    multi-chain ESS of galaxy g; samples [G*C, N, P]."""
    s = np.asarray(samples)
    gc, n, p = s.shape
    g = gc // chains_per_gal
    s = s.reshape(g, chains_per_gal, n, p)
    tot = 0.0
    per = np.zeros(g)
    for i in range(g):
        e = min(ess(s[i, :, :, k]) for k in range(p))
        per[i] = e
        tot += min(1.0, e / target)
    return tot, per
