"""FP64 CPU oracle of batched HMC for the SPS posterior (TEST INFRASTRUCTURE ONLY).

Restates the sampler of Sec. 4 and App. D.2: Hamiltonian Monte Carlo with a
leapfrog integrator, a fixed number of leapfrog steps per trajectory drawn
per iteration, a Metropolis accept on the energy difference, and step-size
adaptation during a warm-up phase.  The paper runs Blackjax HMC; it does not
print the adaptation constants or the trajectory-length rule, so the
declared readings are:

* trajectory length L ~ U{L_min .. L_max} per iteration; the inverse metric
  is the identity unless adapt_mass is set (the workloads adapt only the step
  size);
* step size adapted per chain by the dual-averaging scheme of Hoffman &
  Gelman (2014, Sec. 3.2.1) with target 0.8, gamma 0.05, t0 10, kappa 0.75,
  mu = log(10 eps0); warm-up uses eps_m, sampling uses the averaged eps-bar;
* a diagonal inverse metric (mass matrix) adapted per chain in the windowed
  scheme of the Stan reference manual (the paper's Blackjax window
  adaptation is of this family): an initial buffer of 75 iterations, slow
  windows of 25, 50, 100, ... iterations (the last one stretched to the
  terminal buffer), a terminal buffer of 50 (15% / 75% / 10% of the warm-up
  when it is shorter than 150).  At the end of each slow window holding at
  least two draws the inverse
  metric becomes the regularised variance n/(n+5) var + 1e-3 * 5/(n+5) of the
  window's positions (Welford, FP64) and dual averaging restarts with
  mu = log(10 eps).  Momenta p = z / sqrt(minv), kinetic energy
  sum minv p^2 / 2, drift x += eps minv p.  With adapt_mass False the metric
  stays the identity;
* metric="dense" adapts a dense inverse metric the same way (Stan's dense
  variant): the window's covariance (Welford), regularised as
  n/(n+5) cov + 1e-3 * 5/(n+5) I, with Cholesky factor L (cov = L L^T);
  momenta p = L^-T z, kinetic energy |L^T p|^2 / 2, drift x += eps L L^T p;
* random numbers from Philox-4x32-10 (Salmon et al. 2011), keyed by the
  64-bit seed, counter (iteration, block, chain, 0): blocks 0-2 give twelve
  uniforms -> six Box-Muller pairs of momenta, block 3 gives the accept
  uniform (word 0) and L (word 1, L = L_min + (word * n) >> 32 with
  n = L_max - L_min + 1, an exact integer rule).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import sps as O

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, SC'11).

    ctr: [..., 4] integers < 2^32, key: [..., 2].  Each round multiplies
    words 0 and 2 by M0, M1 (64-bit products), mixes the high halves with
    words 1, 3 and the key, and the key is bumped by the Weyl constants
    between rounds.  Returns [..., 4] uint64 holding 32-bit words.  Pinned
    word for word to an independent implementation of the generator (Triton's,
    run on the CPU) and its Weyl constants to their definitions."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & _MASK32 for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & _MASK32
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & _MASK32
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
        k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
        k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
    return np.stack(c, axis=-1)


def uniform01(words):
    """32-bit word -> (word + 1/2) / 2^32 in (0, 1), exact in float64."""
    return (np.asarray(words, dtype=np.float64) + 0.5) * 2.0 ** -32


def draws(seed: int, chains: np.ndarray, it: int, L_min: int, L_max: int):
    """Momenta [C, 12], accept uniforms [C] and trajectory lengths [C] of
    iteration `it` for the given chain ids (the counter layout above)."""
    chains = np.asarray(chains, dtype=np.uint64)
    n = chains.shape[0]
    key = np.zeros((n, 2), np.uint64)
    key[:, 0] = np.uint64(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint64((seed >> 32) & 0xFFFFFFFF)
    words = []
    for blk in range(4):
        ctr = np.zeros((n, 4), np.uint64)
        ctr[:, 0] = np.uint64(it)
        ctr[:, 1] = np.uint64(blk)
        ctr[:, 2] = chains & _MASK32
        words.append(philox4x32_10(ctr, key))
    u = uniform01(np.concatenate(words[:3], axis=1))               # [n, 12]
    u1, u2 = u[:, 0::2], u[:, 1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    p = np.empty((n, 12))
    p[:, 0::2] = r * np.cos(2.0 * math.pi * u2)
    p[:, 1::2] = r * np.sin(2.0 * math.pi * u2)
    u_acc = uniform01(words[3][:, 0])
    span = np.uint64(L_max - L_min + 1)
    L = (L_min + ((words[3][:, 1] * span) >> np.uint64(32))).astype(np.int64)
    return p, u_acc, L


class ApproxTarget:
    """log posterior in unbounded space, approximate photometry, with the
    per-galaxy redshift-dependent pieces (c_SSP, lambda_eff, N_b, distance
    factor) computed once, as Sec. 3 allows when z is known."""

    def __init__(self, tables, z, mag_obs, sigma, mask, lo, hi, k=1.0, x0=0.0, skew=None):
        z = O._t(z)
        self.tables = tables
        self.cssp = O.c_ssp(tables, z)                      # [G, B, K]
        self.lam_eff = O.lambda_eff(tables, z)              # [G, B]
        _, self.nb, _ = O.band_weights(tables, z)
        dl_cm = O.lum_dist_mpc(z.numpy()) * O.MPC_CM
        self.fac = (1.0 + z) * O.L_SUN_ERG_S / (4.0 * math.pi * dl_cm ** 2 * O.AB_ZP_CGS)
        self.t_obs = O.t_obs_gyr(z)
        self.mag_obs, self.sigma = O._t(mag_obs), O._t(sigma)
        self.mask = np.asarray(mask)
        self.lo, self.hi = O._t(lo), O._t(hi)
        self.k, self.x0, self.skew = k, x0, skew      # Eq. BoundingFunction / SkewNormPrior

    def mags(self, theta, rows):
        W, _, _, _ = O.ssp_weights(theta, self.tables, self.t_obs[rows])
        F = O.attenuation(self.lam_eff[rows], theta[:, 9:10], theta[:, 10:11], theta[:, 11:12])
        c = F * torch.einsum("nbk,nk->nb", self.cssp[rows], W.reshape(W.shape[0], -1))
        return -2.5 * torch.log10(self.fac[rows, None] * c / self.nb[rows])

    def __call__(self, x, rows):
        x = O._t(x).clone().requires_grad_(True)
        th = O.bound(x, self.lo, self.hi, self.k, self.x0)
        mag = self.mags(th, rows)
        lp = O.loglike(mag, self.mag_obs[rows], self.sigma[rows], self.mask[rows]) \
            + O.log_prior_unbounded(x, self.k, self.x0, self.skew)
        (g,) = torch.autograd.grad(lp.sum(), x)
        return lp.detach().numpy(), g.detach().numpy()


class ExactTarget(ApproxTarget):
    """log posterior in unbounded space on the exact photometry (Eq.
    photo_integral_exact): the SED contracted with the SSP table and the dust
    curve at every wavelength, then integrated through the redshifted filters
    (the band weights of each galaxy computed once, as its z is fixed)."""

    def __init__(self, tables, z, mag_obs, sigma, mask, lo, hi, k=1.0, x0=0.0, skew=None):
        super().__init__(tables, z, mag_obs, sigma, mask, lo, hi, k, x0, skew)
        self.w, _, _ = O.band_weights(tables, O._t(z))                 # [G, B, Lam]
        self.lam = torch.as_tensor(tables.lam_ang, dtype=O.DT)

    def mags(self, theta, rows):
        W, _, _, _ = O.ssp_weights(theta, self.tables, self.t_obs[rows])
        S = O.sed_rest(W, self.tables)
        F = O.attenuation(self.lam[None, :], theta[:, 9:10], theta[:, 10:11], theta[:, 11:12])
        c = O.band_flux(S, F, self.w[rows])
        return -2.5 * torch.log10(self.fac[rows, None] * c / self.nb[rows])


def warmup_windows(n_warm):
    """(end of the initial buffer, slow windows [(start, end)], start of the
    terminal buffer) of the windowed metric adaptation."""
    if n_warm >= 150:
        init, term, w = 75, 50, 25
    else:
        init, term = int(0.15 * n_warm), int(0.1 * n_warm)
        w = n_warm - init - term
    wins = []
    start, stop = init, n_warm - term
    while start < stop and w > 0:
        end = start + w
        if end + 2 * w > stop:
            end = stop
        wins.append((start, end))
        start, w = end, 2 * w
    return init, wins, stop


def leapfrog(target, rows, x, p, g, eps, L, minv=None, chol=None):
    """L leapfrog steps (half kick, drift, gradient, half kick), per chain
    lengths L; returns the end point, its momentum, log p and gradient.  The
    inverse metric is diagonal (minv) or dense (chol: its Cholesky factor)."""
    x, p, g = x.copy(), p.copy(), g.copy()
    minv = np.ones_like(x) if minv is None else minv
    lp = np.full(x.shape[0], np.nan)
    Lmax = int(np.max(L)) if len(L) else 0
    for step in range(Lmax):
        act = step < L
        if not act.any():
            break
        e = eps[act, None]
        p[act] += 0.5 * e * g[act]
        if chol is None:
            x[act] += e * minv[act] * p[act]
        else:
            Lc = chol[act]
            u = np.einsum("ckj,ck->cj", Lc, p[act])              # L^T p
            x[act] += e * np.einsum("ckj,cj->ck", Lc, u)           # L (L^T p)
        lpa, ga = target(x[act], rows[act])
        g[act] = ga
        lp[act] = lpa
        p[act] += 0.5 * e * g[act]
    return x, p, g, lp


def run_hmc(target, x0, gal_of_chain, seed, n_warm, n_samp, L_min=8, L_max=64,
            eps0=0.1, target_accept=0.8, gamma=0.05, t0=10.0, kappa=0.75,
            chain_ids=None, adapt_mass=False, metric="diag"):
    """Batched HMC over independent chains (Sec. 4, App. D.2).

    Returns dict with samples [C, n_samp, 12] (bounded parameters),
    accept_prob [C] (mean over sampling), eps [C], divergences [C],
    grad_evals [C]."""
    x = np.array(x0, dtype=np.float64)
    C = x.shape[0]
    rows = np.asarray(gal_of_chain)
    ids = np.arange(C) if chain_ids is None else np.asarray(chain_ids)
    lp, g = target(x, rows)
    eps = np.full(C, eps0)
    mu = np.full(C, math.log(10.0 * eps0))
    hbar = np.zeros(C)
    log_eps_bar = np.zeros(C)
    m_da = 0                                   # iterations since the last restart
    minv = np.ones_like(x)
    dense = metric == "dense"
    chol = np.tile(np.eye(x.shape[1]), (C, 1, 1)) if dense else None
    _, wins, _ = warmup_windows(n_warm) if adapt_mass else (0, [], 0)
    w_n, w_mean, w_m2 = 0, np.zeros_like(x), np.zeros_like(x)
    w_cov = np.zeros((C, x.shape[1], x.shape[1]))
    samples = np.zeros((C, n_samp, x.shape[1]))
    acc_sum = np.zeros(C)
    warm_acc = np.zeros(C)
    div = np.zeros(C, np.int64)
    nevals = np.zeros(C, np.int64)
    for it in range(n_warm + n_samp):
        z, u, L = draws(seed, ids, it, L_min, L_max)
        if dense:
            p = np.stack([np.linalg.solve(chol[i].T, z[i]) for i in range(C)])
            x1, p1, g1, lp1 = leapfrog(target, rows, x, p, g, eps, L, chol=chol)
            kin = lambda q: 0.5 * (np.einsum("ckj,ck->cj", chol, q) ** 2).sum(1)
        else:
            p = z / np.sqrt(minv)
            x1, p1, g1, lp1 = leapfrog(target, rows, x, p, g, eps, L, minv)
            kin = lambda q: 0.5 * (minv * q * q).sum(1)
        nevals += L
        h0 = -lp + kin(p)
        h1 = -lp1 + kin(p1)
        dh = h1 - h0
        finite = np.isfinite(dh)
        a = np.where(finite, np.minimum(1.0, np.exp(-np.where(finite, dh, 0.0))), 0.0)
        div += (~finite) | (np.where(finite, dh, 0.0) > 1000.0)
        take = finite & (np.log(u) < -np.where(finite, dh, np.inf))
        x[take], g[take], lp[take] = x1[take], g1[take], lp1[take]
        if it < n_warm:
            if it >= n_warm // 2:
                warm_acc += a
            m_da += 1
            m = m_da
            hbar = (1.0 - 1.0 / (m + t0)) * hbar + (target_accept - a) / (m + t0)
            log_eps = mu - math.sqrt(m) / gamma * hbar
            w = m ** -kappa
            log_eps_bar = w * log_eps + (1.0 - w) * log_eps_bar
            eps = np.exp(log_eps) if it < n_warm - 1 else np.exp(log_eps_bar)
            for (ws_, we_) in wins:
                if ws_ <= it < we_:
                    w_n += 1                     # Welford over the window's positions
                    d = x - w_mean
                    w_mean = w_mean + d / w_n
                    w_m2 = w_m2 + d * (x - w_mean)
                    w_cov = w_cov + np.einsum("ci,cj->cij", d, x - w_mean)
                    if it == we_ - 1 and w_n >= 2:       # variance needs two draws
                        if dense:
                            cov = w_cov / (w_n - 1.0)
                            reg = (w_n / (w_n + 5.0)) * cov + 1e-3 * (5.0 / (w_n + 5.0)) * np.eye(x.shape[1])
                            chol = np.linalg.cholesky(reg)
                        else:
                            var = w_m2 / (w_n - 1.0)
                            minv = (w_n / (w_n + 5.0)) * var + 1e-3 * (5.0 / (w_n + 5.0))
                    if it == we_ - 1:
                        w_n, w_mean, w_m2 = 0, np.zeros_like(x), np.zeros_like(x)
                        w_cov = np.zeros_like(w_cov)
                        mu = np.log(10.0 * eps)
                        hbar = np.zeros(C)
                        log_eps_bar = np.zeros(C)
                        m_da = 0
        else:
            s = it - n_warm
            th = O.bound(torch.as_tensor(x), target.lo, target.hi, getattr(target, "k", 1.0),
                         getattr(target, "x0", 0.0)).numpy()
            samples[:, s] = th
            acc_sum += a
    return dict(samples=samples, accept_prob=acc_sum / max(n_samp, 1), eps=eps, minv=minv, chol=chol,
                warm_accept=warm_acc / max(n_warm - n_warm // 2, 1),
                divergences=div, grad_evals=nevals)
