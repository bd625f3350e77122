"""FP64 CPU oracle of batched NUTS for the SPS posterior (TEST INFRASTRUCTURE ONLY).

The paper compares HMC with the No-U-Turn Sampler (Sec. 4, App. D.2), run
with Blackjax.  This module restates NUTS as the multinomial variant with
the generalised no-U-turn criterion (Hoffman & Gelman 2014; Betancourt 2017,
"A Conceptual Introduction to Hamiltonian Monte Carlo", Sec. A.4), identity
metric, one chain at a time, in the plainest form:

* an iteration draws a momentum p0 and grows a trajectory from (x0, p0) by
  doubling: at depth j a direction v = +-1 is drawn and a new subtree of 2^j
  leapfrog steps is built from the trajectory's end in that direction;
* every state s of the trajectory has weight exp(-H(s)); inside the new
  subtree a proposal is kept by progressive multinomial sampling over its
  leaves (leaf n replaces the proposal with probability w_n / sum_{m<=n} w_m);
  a complete subtree replaces the trajectory's proposal with probability
  min(1, W_subtree / W_trajectory) (biased progressive sampling);
* U-turn: a set of consecutive states with momentum sum rho and end momenta
  p_a, p_b has turned if rho . p_a <= 0 or rho . p_b <= 0.  Inside the new
  subtree every aligned block of 2^k leaves (k >= 1), taken as it completes,
  is checked; a turn, or a divergence (H - H0 > 1000 or non-finite), discards
  the subtree and ends the iteration.  After a subtree is merged the whole
  trajectory is checked; a turn ends the iteration, and so does depth max_depth;
* step size: dual averaging as in oracle.hmc (target 0.8, gamma 0.05, t0 10,
  kappa 0.75, mu = log(10 eps0)) on the statistic mean over the leaves built
  of min(1, exp(H0 - H)); warm-up uses eps_m, sampling eps-bar;
* random numbers from Philox-4x32-10 keyed by the seed: the momentum from
  counters (iteration, 0..2, chain, 0) exactly as oracle.hmc; at depth j the
  counter (iteration, 16 + j, chain, 0) gives the direction (word 0, top bit
  set -> v = +1) and the subtree's acceptance uniform (word 1); leaf n of the
  depth-j subtree uses (iteration, 64 + j, chain, n), word 0.  Every draw is
  keyed by where it is used, not by the order of use.

Everything is FP64; leaves are stored in lists and each block sum is formed
directly from them.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import hmc as H
from . import sps as O


def _words(seed, it, blk, chain, leaf):
    key = np.array([[seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]], np.uint64)
    ctr = np.array([[it, blk, chain, leaf]], np.uint64)
    return H.philox4x32_10(ctr, key)[0]


def level_draws(seed, it, chain, j):
    """Direction (+1 / -1) and acceptance uniform of the depth-j subtree."""
    w = _words(seed, it, 16 + j, chain, 0)
    v = 1 if (int(w[0]) >> 31) & 1 else -1
    return v, float(H.uniform01(w[1]))


def leaf_uniforms(seed, it, chain, j):
    """Uniforms of the 2^j leaves of the depth-j subtree, leaf n at [n]."""
    n = 2 ** j
    key = np.zeros((n, 2), np.uint64)
    key[:, 0], key[:, 1] = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    ctr = np.zeros((n, 4), np.uint64)
    ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3] = it, 64 + j, chain, np.arange(n)
    return H.uniform01(H.philox4x32_10(ctr, key)[:, 0])


def _logaddexp(a, b):
    return np.logaddexp(a, b)


def nuts_iteration(target, row, x0, g0, lp0, p0, eps, seed, it, chain, max_depth):
    """One NUTS transition of one chain from (x0, p0).  Returns the new state
    (x, g, lp), the acceptance statistic, the number of leaves built, the
    depth reached and whether a divergence ended it."""
    rows = np.array([row])

    def step(x, p, g, v):
        ph = p + 0.5 * v * eps * g
        x1 = x + v * eps * ph
        lp1, g1 = target(x1[None, :], rows)
        lp1, g1 = float(lp1[0]), g1[0]
        return x1, ph + 0.5 * v * eps * g1, g1, lp1

    h0 = -lp0 + 0.5 * float(p0 @ p0)
    left = right = (x0, p0, g0)
    rho = p0.copy()
    lw = -h0
    prop = (x0, g0, lp0)
    acc_sum, n_leaves, depth, divergent = 0.0, 0, 0, False
    for j in range(max_depth):
        v, u_tree = level_draws(seed, it, chain, j)
        x, p, g = right if v > 0 else left
        moms, states = [], []
        u_leaf = leaf_uniforms(seed, it, chain, j)
        lw_sub, prop_sub, ok = -np.inf, None, True
        for n in range(2 ** j):
            x, p, g, lp = step(x, p, g, v)
            h = -lp + 0.5 * float(p @ p)
            dh = h - h0
            n_leaves += 1
            if not np.isfinite(dh) or dh > 1000.0:
                divergent, ok = True, False
                break
            acc_sum += min(1.0, math.exp(-dh))
            moms.append(p)
            states.append((x, p, g))
            lw_sub = _logaddexp(lw_sub, -h)
            if u_leaf[n] < math.exp(-h - lw_sub):
                prop_sub = (x, g, lp)
            k = 1
            while (n + 1) % (2 ** k) == 0 and k <= j:       # aligned blocks ending at n
                blk = moms[n + 1 - 2 ** k:n + 1]
                r = np.sum(blk, axis=0)
                if r @ blk[0] <= 0.0 or r @ blk[-1] <= 0.0:
                    ok = False
                    break
                k += 1
            if not ok:
                break
        if not ok:
            break
        if u_tree < math.exp(min(0.0, lw_sub - lw)):
            prop = prop_sub
        lw = _logaddexp(lw, lw_sub)
        rho = rho + np.sum(moms, axis=0)
        if v > 0:
            right = states[-1]
        else:
            left = states[-1]
        depth = j + 1
        if rho @ left[1] <= 0.0 or rho @ right[1] <= 0.0:
            break
    return prop, acc_sum / max(n_leaves, 1), n_leaves, depth, divergent


def run_nuts(target, x0, gal_of_chain, seed, n_warm, n_samp, eps0=0.1, target_accept=0.8,
             gamma=0.05, t0=10.0, kappa=0.75, max_depth=10, chain_ids=None):
    """Batched NUTS over independent chains (identity metric).

    Returns dict with samples [C, n_samp, 12] (bounded parameters),
    samples_x (the same draws in unbounded space),
    accept_prob [C] (mean statistic over sampling), eps [C], divergences [C],
    grad_evals [C] (leaves built, plus the initial evaluation), depth [C]
    (mean over sampling)."""
    x = np.array(x0, dtype=np.float64)
    C, D = x.shape
    rows = np.asarray(gal_of_chain)
    ids = np.arange(C) if chain_ids is None else np.asarray(chain_ids)
    lp, g = target(x, rows)
    lp = np.array(lp, dtype=np.float64)
    g = np.array(g, dtype=np.float64)
    eps = np.full(C, eps0)
    mu = np.full(C, math.log(10.0 * eps0))
    hbar = np.zeros(C)
    log_eps_bar = np.zeros(C)
    samples = np.zeros((C, n_samp, D))
    samples_x = np.zeros((C, n_samp, D))
    acc_sum = np.zeros(C)
    depth_sum = np.zeros(C)
    div = np.zeros(C, np.int64)
    nevals = np.ones(C, np.int64)
    for it in range(n_warm + n_samp):
        z, _, _ = H.draws(seed, ids, it, 1, 1)
        for c in range(C):
            prop, a, nl, dep, dv = nuts_iteration(target, rows[c], x[c], g[c], lp[c], z[c, :D], eps[c],
                                                  seed, it, int(ids[c]), max_depth)
            x[c], g[c], lp[c] = prop
            nevals[c] += nl
            div[c] += int(dv)
            if it < n_warm:
                m = it + 1
                hbar[c] = (1.0 - 1.0 / (m + t0)) * hbar[c] + (target_accept - a) / (m + t0)
                log_eps = mu[c] - math.sqrt(m) / gamma * hbar[c]
                w = m ** -kappa
                log_eps_bar[c] = w * log_eps + (1.0 - w) * log_eps_bar[c]
                eps[c] = math.exp(log_eps) if it < n_warm - 1 else math.exp(log_eps_bar[c])
            else:
                acc_sum[c] += a
                depth_sum[c] += dep
        if it >= n_warm:
            samples_x[:, it - n_warm] = x
            samples[:, it - n_warm] = O.bound(torch.as_tensor(x), target.lo, target.hi, getattr(target, "k", 1.0),
                                              getattr(target, "x0", 0.0)).numpy()
    ns = max(n_samp, 1)
    return dict(samples=samples, samples_x=samples_x, accept_prob=acc_sum / ns, eps=eps, divergences=div,
                grad_evals=nevals, depth=depth_sum / ns)
