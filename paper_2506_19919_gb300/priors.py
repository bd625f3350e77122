"""Host-side set-up of the bounding functions and the skew-normal prior (App. C).

The paper tunes each parameter's sigmoid hyper-parameters (k, x0) in advance
so that Eq. BoundingFunction is close to linear where the fit is expected,
then maps draws of an approximately Gaussian prior on theta into the
unbounded space and fits Eq. SkewNormPrior to them per parameter.  These
helpers do both; their results go into Context(sigmoid_k=..., sigmoid_x0=...,
skew=...).  Plain NumPy, run once per analysis; not on the sampling path.
"""
from __future__ import annotations

import math

import numpy as np


def tune_sigmoid(lo, hi, a, b):
    """(k, x0) per parameter such that F_B(-1) = a and F_B(+1) = b, i.e. the
    expected range [a, b] of theta (lo < a < b < hi) is the image of the unit
    interval around the sigmoid's centre: k = (logit p_b - logit p_a) / 2,
    x0 = 1 - logit(p_b) / k with p = (theta - lo) / (hi - lo)."""
    lo, hi, a, b = (np.asarray(v, dtype=np.float64) for v in (lo, hi, a, b))
    if not (np.all(lo < a) and np.all(a < b) and np.all(b < hi)):
        raise ValueError("need lo < a < b < hi for every parameter")
    pa, pb = (a - lo) / (hi - lo), (b - lo) / (hi - lo)
    la, lb = np.log(pa / (1 - pa)), np.log(pb / (1 - pb))
    k = 0.5 * (lb - la)
    return k, 1.0 - lb / k


def unbound(theta, lo, hi, k=1.0, x0=0.0):
    """Inverse of Eq. BoundingFunction: x = x0 + logit((theta - lo) / (hi - lo)) / k."""
    p = (np.asarray(theta, dtype=np.float64) - lo) / (np.asarray(hi) - lo)
    return np.asarray(x0) + np.log(p / (1.0 - p)) / np.asarray(k)


_SKEW_MAX = 0.99  # |sample skewness| is capped below the family's bound (~0.9953)


def _moments(x):
    """Method-of-moments start (Azzalini 1985): with delta = s / sqrt(1 + s^2)
    the family's skewness is (4 - pi)/2 (delta sqrt(2/pi))^3 /
    (1 - 2 delta^2/pi)^1.5, its variance omega^2 (1 - 2 delta^2 / pi) and its
    mean xi + omega delta sqrt(2/pi); the sample moments are solved for delta,
    omega, xi."""
    m = x.mean(0)
    v = x.var(0, ddof=1)
    g = ((x - m) ** 3).mean(0) / x.var(0) ** 1.5
    g = np.clip(g, -_SKEW_MAX, _SKEW_MAX)
    c = np.abs(g) ** (2.0 / 3.0)
    d = np.sign(g) * np.sqrt(0.5 * math.pi * c / (c + ((4.0 - math.pi) / 2.0) ** (2.0 / 3.0)))
    omega = np.sqrt(v / (1.0 - 2.0 * d * d / math.pi))
    xi = m - omega * d * math.sqrt(2.0 / math.pi)
    s = d / np.sqrt(1.0 - d * d)
    return xi, omega, s


def fit_skew_normal(x):
    """(xi, omega, s) of Eq. SkewNormPrior per column of x [n, d]: maximum
    likelihood, started from the method of moments (near-symmetric samples
    leave s weakly determined; the fitted densities still agree)."""
    from scipy import optimize, special

    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    xi0, om0, s0 = _moments(x)
    out = np.zeros((3, x.shape[1]))
    for j in range(x.shape[1]):
        v = x[:, j]

        def nll(q):
            xi, lom, s = q
            u = (v - xi) * np.exp(-lom)
            return -np.mean(-lom - 0.5 * u * u + special.log_ndtr(s * u))

        r = optimize.minimize(nll, [xi0[j], math.log(om0[j]), s0[j]], method="Nelder-Mead",
                              options={"xatol": 1e-8, "fatol": 1e-12, "maxiter": 4000})
        out[:, j] = r.x[0], math.exp(r.x[1]), r.x[2]
    return out[0], out[1], out[2]


def skew_normal_prior(theta_draws, lo, hi, k=1.0, x0=0.0):
    """The paper's recipe: draws of theta [n, 12] mapped through F_B^-1 and
    fitted per parameter; returns (xi, omega, s) for Context(skew=...)."""
    return fit_skew_normal(unbound(theta_draws, lo, hi, k, x0))
