"""HMC on the exact photometry (sps_hmc_run with mode EXACT) against the FP64
oracle's sampler on the same target (oracle/hmc.py: ExactTarget).

Three galaxies of the production grid (107 x 12 x 5994, six Gaussian bands)
x four chains, started near the truth: at a fixed step size (no warm-up) the
chains follow the oracle's draw by draw for the FP32 contraction (SIMT) and
for 3xTF32 on the tensor cores, to within the bars of the leapfrog tests; with
BF16 (whose gradient is good to ~1e-2) the run is checked for valid draws and
acceptance.  A short warm-up adapts the step size like the oracle's, and the
gradient-evaluation count equals the leapfrog steps plus the initial one."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import hmc as OH
from oracle import sps as O

pytestmark = pytest.mark.gpu

G, C = 3, 4


@pytest.fixture(scope="module")
def exact3():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(1, n_gal=G)
    mobs = O.photometry(wl.theta_true, wl.z, wl.tables, "exact").numpy() + wl.noise
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=False)
    x0 = np.repeat(W.unbounded_of(wl.theta_true), C, axis=0)
    x0 = (x0 + np.random.default_rng(8).normal(0, 0.02, x0.shape)).astype(np.float32)
    tgt = OH.ExactTarget(wl.tables, wl.z, mobs, wl.sigma, wl.mask, W.PRIOR_LO, W.PRIOR_HI)
    yield wl, ctx, mobs, x0, tgt
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-5), ("tf32x3", 2e-3)])
def test_exact_hmc_matches_oracle_draws(exact3, prec, tol):
    wl, ctx, mobs, x0, tgt = exact3
    kw = dict(n_warm=0, n_samp=6, L_min=6, L_max=6, seed=41, eps0=2e-3)
    out = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, chains_per_gal=C, mode="exact", prec=prec, **kw)
    s = out["samples"].cpu().numpy()
    ref = OH.run_hmc(tgt, x0.astype(np.float64), np.repeat(np.arange(G), C), **kw)
    span = W.PRIOR_HI - W.PRIOR_LO
    d = np.abs((s - ref["samples"]) / span).max(axis=(1, 2))
    assert (d < tol).mean() >= 11 / 12, d
    assert (out["grad_evals"].cpu().numpy() == 1 + 6 * 6).all()


def test_exact_hmc_bf16_and_adaptation(exact3):
    wl, ctx, mobs, x0, tgt = exact3
    out = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, chains_per_gal=C, mode="exact", prec="bf16",
                      n_warm=30, n_samp=10, L_min=4, L_max=8, seed=5, eps0=1e-2)
    s = out["samples"].cpu().numpy()
    assert np.isfinite(s).all()
    lo, hi = W.PRIOR_LO, W.PRIOR_HI
    assert ((s >= lo) & (s <= hi)).all()
    eps = out["step_size"].cpu().numpy()
    assert (eps != 1e-2).all() and np.isfinite(eps).all()
    assert float(out["accept_prob"].mean()) > 0.3
    # the oracle's adapted step sizes on the same chains (FP64, same draws)
    ref = OH.run_hmc(tgt, x0.astype(np.float64), np.repeat(np.arange(G), C), n_warm=30, n_samp=10,
                     L_min=4, L_max=8, seed=5, eps0=1e-2)
    r = eps / ref["eps"]
    assert np.median(r) > 0.5 and np.median(r) < 2.0
    ev = out["grad_evals"].cpu().numpy()
    _, _, L = zip(*[OH.draws(5, np.arange(G * C), it, 4, 8) for it in range(40)])
    np.testing.assert_array_equal(ev, 1 + np.sum(np.stack(L), axis=0))
