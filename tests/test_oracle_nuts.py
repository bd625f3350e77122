"""Pins of the NUTS oracle (CPU only).

The oracle builds each trajectory leaf by leaf; these tests pin it against
what NUTS must do whatever the bookkeeping: the stationary distribution
(exact draws stay exact, moments of Gaussian targets), the trajectory rule
restated over time-indexed states (every aligned block of the doubled
trajectory checked for a U-turn), the reduction to one-step HMC at depth 1,
and divergence handling."""
import math

import numpy as np
import torch
from scipy import special, stats

from oracle import hmc as H
from oracle import nuts as N


class _Quartic:
    """log p = -x^4 / 4 in one dimension; CDF through the regularised lower
    incomplete gamma function: F(x) = 1/2 + sign(x) P(1/4, x^4/4) / 2."""
    lo = torch.zeros(1, dtype=torch.float64)
    hi = torch.ones(1, dtype=torch.float64)

    def __call__(self, x, rows):
        x = np.asarray(x)
        return -0.25 * (x ** 4).sum(1), -x ** 3

    @staticmethod
    def cdf(x):
        return 0.5 + 0.5 * np.sign(x) * special.gammainc(0.25, x ** 4 / 4.0)

    @staticmethod
    def exact(rng, n):
        """Rejection from N(0, 1): exp(-x^4/4) <= exp(1/4) exp(-x^2/2)."""
        out = []
        while len(out) < n:
            z = rng.normal(size=4 * n)
            u = rng.random(4 * n)
            out.extend(z[u < np.exp(-z ** 4 / 4 + z ** 2 / 2 - 0.25)])
        return np.array(out[:n])


class _Gauss:
    def __init__(self, cov):
        self.cov = np.asarray(cov, dtype=np.float64)
        self.P = np.linalg.inv(self.cov)
        d = self.cov.shape[0]
        self.lo = torch.zeros(d, dtype=torch.float64)
        self.hi = torch.ones(d, dtype=torch.float64)

    def __call__(self, x, rows):
        x = np.asarray(x)
        y = x @ self.P
        return -0.5 * np.einsum("ci,ci->c", y, x), -y


def test_exact_draws_stay_exact_quartic():
    """Invariance: chains started at exact draws of a non-Gaussian target are
    still exact after NUTS transitions (KS against the closed-form CDF)."""
    t = _Quartic()
    x0 = t.exact(np.random.default_rng(1), 3000)
    r = N.run_nuts(t, x0[:, None], np.zeros(len(x0), int), seed=7, n_warm=0, n_samp=2, eps0=1.0,
                   max_depth=8)
    for k in range(2):
        assert stats.kstest(r["samples_x"][:, k, 0], t.cdf).pvalue > 1e-3
    assert 1.2 < r["depth"].mean() < 2.0


def test_invariance_check_detects_a_planted_selection_mistake(monkeypatch):
    """Taking the last state built instead of the multinomial draw (all
    uniforms zero) breaks invariance, and the check above sees it."""
    t = _Quartic()
    x0 = t.exact(np.random.default_rng(1), 3000)
    level = N.level_draws
    monkeypatch.setattr(N, "leaf_uniforms", lambda seed, it, chain, j: np.zeros(2 ** j))
    monkeypatch.setattr(N, "level_draws", lambda seed, it, chain, j: (level(seed, it, chain, j)[0], 0.0))
    r = N.run_nuts(t, x0[:, None], np.zeros(len(x0), int), seed=7, n_warm=0, n_samp=2, eps0=1.0,
                   max_depth=8)
    assert stats.kstest(r["samples_x"][:, 1, 0], t.cdf).pvalue < 1e-6


def test_standard_normal_moments_with_adaptation():
    D = 12
    r = N.run_nuts(_Gauss(np.eye(D)), np.zeros((4, D)), np.zeros(4, int), seed=5, n_warm=100, n_samp=300,
                   eps0=0.5)
    xs = r["samples_x"].reshape(-1, D)
    n = xs.shape[0]
    assert (np.abs(xs.mean(0)) < 5.0 / math.sqrt(n)).all()
    assert (np.abs(xs.var(0) - 1.0) < 5.0 * math.sqrt(2.0 / n)).all()
    # dual averaging reaches its target: the sampling phase uses the averaged
    # (smaller) step, so the statistic sits at or above 0.8
    assert (r["accept_prob"] > 0.75).all() and (r["accept_prob"] < 0.97).all()
    assert (r["eps"] > 0.3).all() and (r["eps"] < 1.5).all()


def test_correlated_gaussian_covariance():
    cov = np.array([[1.0, 2.7], [2.7, 9.0]])        # correlation 0.9, scales 1 and 3
    r = N.run_nuts(_Gauss(cov), np.zeros((4, 2)), np.zeros(4, int), seed=11, n_warm=150, n_samp=500,
                   eps0=0.3)
    xs = r["samples_x"].reshape(-1, 2)
    est = np.cov(xs.T)
    assert np.abs(est - cov).max() / 9.0 < 0.15
    assert abs(np.corrcoef(xs.T)[0, 1] - 0.9) < 0.04
    # the long axis needs several doublings per iteration
    assert (r["depth"] > 2.0).all()


def _span_states(t, x0, p0, eps, T):
    """States at times -T..T of the leapfrog flow through (x0, p0): forward
    with +eps, backward with -eps; index i <-> time i - T."""
    D = x0.shape[0]
    rows = np.zeros(1, int)
    lp0, g0 = t(x0[None, :], rows)
    X = np.zeros((2 * T + 1, D))
    P = np.zeros((2 * T + 1, D))
    LP = np.zeros(2 * T + 1)
    X[T], P[T], LP[T] = x0, p0, lp0[0]
    for sgn in (1, -1):
        x, p, g = x0[None, :].copy(), p0[None, :].copy(), g0.copy()
        for k in range(1, T + 1):
            x, p, g, lp = H.leapfrog(t, rows, x, p, g, np.array([sgn * eps]), np.array([1]))
            X[T + sgn * k], P[T + sgn * k], LP[T + sgn * k] = x[0], p[0], lp[0]
    return X, P, LP


def _turned(P, a, b):
    rho = P[a:b + 1].sum(0)
    return rho @ P[a] <= 0.0 or rho @ P[b] <= 0.0


def _tree_by_time(P, LP, T, dirs, max_depth):
    """The trajectory rule over time-indexed states.  At depth j the subtree
    B_j of 2^j states is appended on side dirs[j]; it is rejected if any of
    its aligned blocks of 2^k states (k >= 1, aligned to B_j's start in time)
    U-turns or one of its states diverges, and the leaves built up to the
    first such failure (in build order: away from the trajectory) count as
    evaluated.  An accepted subtree extends the span; the span is then checked
    as a whole.  Returns (depth, leaves built, span, statistic sum)."""
    h0 = -LP[T] + 0.5 * P[T] @ P[T]
    H_ = -LP + 0.5 * np.einsum("ij,ij->i", P, P)
    lo = hi = T
    depth, leaves, acc = 0, 0, 0.0
    for j in range(max_depth):
        size = 2 ** j
        if dirs[j] > 0:
            blk = np.arange(hi + 1, hi + 1 + size)
            order = blk                                 # build order
        else:
            blk = np.arange(lo - size, lo)
            order = blk[::-1]
        build_idx = {int(s): n for n, s in enumerate(order)}
        fail_at = math.inf
        for s in order:                                 # divergent leaves
            dh = H_[s] - h0
            if not np.isfinite(dh) or dh > 1000.0:
                fail_at = min(fail_at, build_idx[int(s)])
        k = 1
        while 2 ** k <= size:
            for a in range(blk[0], blk[0] + size, 2 ** k):
                b = a + 2 ** k - 1
                if _turned(P, a, b):
                    fail_at = min(fail_at, max(build_idx[a], build_idx[b]))
            k += 1
        if fail_at < math.inf:
            built = order[:fail_at + 1]
            leaves += len(built)
            acc += sum(min(1.0, math.exp(h0 - H_[s])) for s in built
                       if np.isfinite(H_[s] - h0) and H_[s] - h0 <= 1000.0)
            return depth, leaves, (lo, hi), acc
        leaves += size
        acc += sum(min(1.0, math.exp(h0 - H_[s])) for s in order)
        lo, hi = min(lo, blk[0]), max(hi, blk[-1])
        depth = j + 1
        if _turned(P, lo, hi):
            break
    return depth, leaves, (lo, hi), acc


def _check_tree_rule(t, D, eps, n_cases, max_depth, seed):
    rng = np.random.default_rng(seed)
    T = 2 ** max_depth
    depths = []
    for case in range(n_cases):
        x0 = rng.normal(size=D) * 1.5
        p0 = rng.normal(size=D)
        lp0, g0 = t(x0[None, :], np.zeros(1, int))
        prop, a, nl, dep, div = N.nuts_iteration(t, 0, x0, g0[0], float(lp0[0]), p0, eps, seed, case, 3,
                                                 max_depth)
        dirs = [N.level_draws(seed, case, 3, j)[0] for j in range(max_depth)]
        X, P, LP = _span_states(t, x0, p0, eps, T)
        d2, nl2, (lo, hi), acc2 = _tree_by_time(P, LP, T, dirs, max_depth)
        assert (dep, nl) == (d2, nl2), case
        assert abs(a * nl - acc2) < 1e-9 * max(1.0, acc2)
        # the draw is a state of the accepted span, with its own log density
        dist = np.abs(X[lo:hi + 1] - prop[0]).max(1)
        i = int(np.argmin(dist))
        assert dist[i] < 1e-12 and abs(LP[lo + i] - prop[2]) < 1e-9 * max(1.0, abs(prop[2]))
        depths.append(dep)
    return np.array(depths)


def test_trajectory_rule_matches_time_indexed_restatement():
    """Depth, leaves built, statistic and the span holding the draw agree with
    the rule restated over states indexed by time, on targets where the tree
    stops for different reasons (whole-trajectory U-turns, U-turns inside a
    subtree, the depth limit)."""
    d1 = _check_tree_rule(_Quartic(), 1, 0.3, 60, 6, seed=21)
    d2 = _check_tree_rule(_Gauss(np.array([[1.0, 2.7], [2.7, 9.0]])), 2, 0.2, 60, 7, seed=22)
    d3 = _check_tree_rule(_Gauss(np.eye(12)), 12, 0.1, 30, 5, seed=23)
    assert len(set(d1.tolist())) >= 3 and len(set(d2.tolist())) >= 3
    assert (d3 == 5).any()                              # depth limit reached


def test_depth_one_is_one_step_hmc():
    """With max_depth 1 the tree is one leapfrog step in direction v, kept
    with probability min(1, exp(-dH)) by the subtree's uniform: HMC with L = 1
    started from momentum v p0."""
    t = _Gauss(np.diag(np.linspace(0.5, 2.0, 12)))
    rng = np.random.default_rng(3)
    kept = 0
    for case in range(200):
        x0, p0 = rng.normal(size=12), rng.normal(size=12)
        lp0, g0 = t(x0[None, :], np.zeros(1, int))
        eps = 0.8
        prop, a, nl, dep, div = N.nuts_iteration(t, 0, x0, g0[0], float(lp0[0]), p0, eps, 9, case, 1, 1)
        v, u = N.level_draws(9, case, 1, 0)
        x1, p1, g1, lp1 = H.leapfrog(t, np.zeros(1, int), x0[None, :], v * p0[None, :], g0, np.array([eps]),
                                     np.array([1]))
        dh = (-lp1[0] + 0.5 * p1[0] @ p1[0]) - (-lp0[0] + 0.5 * p0 @ p0)
        take = u < min(1.0, math.exp(-dh))
        np.testing.assert_allclose(prop[0], x1[0] if take else x0, rtol=0, atol=1e-13)
        assert abs(a - min(1.0, math.exp(-dh))) < 1e-12 and nl == 1 and dep == 1 and not div
        kept += take
    assert 20 < kept < 200


def test_divergent_first_leaf_keeps_the_start():
    t = _Quartic()
    x0 = np.array([1.0])
    lp0, g0 = t(x0[None, :], np.zeros(1, int))
    prop, a, nl, dep, div = N.nuts_iteration(t, 0, x0, g0[0], float(lp0[0]), np.array([0.5]), 50.0, 1, 0, 0, 10)
    assert div and nl == 1 and dep == 0 and a == 0.0
    np.testing.assert_array_equal(prop[0], x0)


def test_draws_are_keyed_by_use():
    """Direction bits are fair and the leaf uniforms of a subtree do not depend
    on the depth it is built at beyond the counter."""
    v = np.array([N.level_draws(4, it, c, j)[0] for it in range(20) for c in range(10) for j in range(5)])
    assert abs(v.mean()) < 0.15
    u = N.leaf_uniforms(4, 0, 0, 10)
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    np.testing.assert_array_equal(N.leaf_uniforms(4, 0, 0, 3), N.leaf_uniforms(4, 0, 0, 3))
    assert not np.array_equal(N.leaf_uniforms(4, 0, 0, 3), N.leaf_uniforms(4, 0, 0, 4)[:8])
