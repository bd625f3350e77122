"""Age-dependent metallicity distribution (non-separable SSP weights) on the
GPU: weights, photometry, log L + gradient (approximate and exact paths) and
the samplers (the one-chain-per-warp, per-age-q variant of the persistent
kernel), against the FP64 oracle on the production grid.  Tolerances as in
test_gpu_parity."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import hmc as OH
from oracle import nuts as ON
from oracle import sps as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mdf96():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(1, n_gal=96)
    wl.tables = W.with_mdf_offset(wl.tables, W.mzr_offsets(wl.tables.age_yr, slope=0.4))
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    yield wl, ctx
    ctx.close()


def test_nonseparable_weights(mdf96):
    wl, ctx = mdf96
    Wg, Mg = ctx.weights(wl.theta)
    th = torch.as_tensor(wl.theta, dtype=torch.float64)
    Wr, Mr, _, q = O.ssp_weights(th, wl.tables, O.t_obs_gyr(torch.as_tensor(wl.z)))
    assert q.dim() == 3                                      # P_met depends on the age bin
    Wr = Wr.reshape(wl.theta.shape[0], -1).numpy()
    err = np.abs(Wg.cpu().numpy() - Wr).max(1) / Wr.max(1)
    assert err.max() < 2e-5


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-3), ("exact", "fp32", 1e-3),
                                           ("exact", "bf16", 5e-3)])
def test_nonseparable_photometry(mdf96, mode, prec, tol):
    wl, ctx = mdf96
    m = ctx.photometry(wl.theta, mode=mode, prec=prec).cpu().numpy()
    ref = O.photometry(wl.theta, wl.z, wl.tables, mode).numpy()
    assert np.abs(m - ref).max() < tol
    sep = O.photometry(wl.theta, wl.z, W.with_mdf_offset(wl.tables, None), mode).numpy()
    assert np.abs(sep - ref).max() > 10 * tol                # the offsets matter at this tolerance


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-4), ("exact", "fp32", 1e-4),
                                           ("exact", "bf16", 1e-2)])
def test_nonseparable_loglike_grad(mdf96, mode, prec, tol):
    """Gradient through the per-age MDF (columns lgZ and sigma_lgZ included)."""
    wl, ctx = mdf96
    th_true = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    mobs = O.photometry(th_true, wl.z, wl.tables, mode).numpy() + wl.noise
    ev = W.prior_draw(np.random.default_rng(23), wl.n_gal)
    ll, g = ctx.loglike_grad(ev, mobs, wl.sigma, wl.mask, mode=mode, prec=prec)
    llr, gr, _ = O.loglike_and_grad(ev, wl.z, wl.tables, mobs, wl.sigma, wl.mask, mode)
    np.testing.assert_allclose(ll.cpu().numpy(), llr.numpy(), rtol=2e-4 if prec == "fp32" else 5e-3)
    g, gr = g.cpu().numpy().astype(np.float64), gr.numpy()
    assert (np.abs(g - gr).max(1) / np.abs(gr).max(1)).max() < tol
    scale = np.abs(gr).max(1)
    assert (np.abs(g[:, 7:9] - gr[:, 7:9]).max(1) / scale).max() < tol


@pytest.mark.parametrize("sampler", ["hmc", "nuts"])
def test_nonseparable_samplers_match_oracle_draws(mdf96, sampler):
    wl, ctx = mdf96
    G, C = 3, 4
    th_true = torch.as_tensor(wl.theta_true[:G], dtype=torch.float64)
    mobs = O.photometry(th_true, wl.z[:G], wl.tables, "approx").numpy() + wl.noise[:G]
    mobs_all = np.full((wl.n_gal, 6), 30.0)
    mobs_all[:G] = mobs
    mask = np.zeros(wl.n_gal, np.uint32)
    mask[:G] = wl.mask[:G]
    x0 = np.repeat(W.unbounded_of(wl.theta_true[:G]), C, axis=0)
    x0 = (x0 + np.random.default_rng(9).normal(0, 0.02, x0.shape)).astype(np.float32)
    x0_all = np.zeros((wl.n_gal * C, 12), np.float32)
    x0_all[:G * C] = x0
    tgt = OH.ApproxTarget(wl.tables, wl.z[:G], mobs, wl.sigma[:G], wl.mask[:G], W.PRIOR_LO, W.PRIOR_HI)
    rows = np.repeat(np.arange(G), C)
    if sampler == "hmc":
        out = ctx.hmc_run(x0_all, mobs_all, wl.sigma, mask, chains_per_gal=C, n_warm=0, n_samp=6, L_min=6,
                          L_max=6, seed=43, eps0=2e-3, autotune=False)
        ref = OH.run_hmc(tgt, x0.astype(np.float64), rows, seed=43, n_warm=0, n_samp=6, L_min=6, L_max=6,
                         eps0=2e-3)
    else:
        out = ctx.hmc_run(x0_all, mobs_all, wl.sigma, mask, chains_per_gal=C, n_warm=0, n_samp=3, seed=47,
                          eps0=1e-2, autotune=False, sampler="nuts", max_depth=5)
        ref = ON.run_nuts(tgt, x0.astype(np.float64), rows, seed=47, n_warm=0, n_samp=3, eps0=1e-2,
                          max_depth=5)
    s = out["samples"].cpu().numpy()[:G * C]
    span = W.PRIOR_HI - W.PRIOR_LO
    d = np.abs((s - ref["samples"]) / span).max(axis=(1, 2))
    assert (d < 2e-5).mean() >= 11 / 12
    assert (out["grad_evals"].cpu().numpy()[:G * C] == ref["grad_evals"] + (1 if sampler == "hmc" else 0)).mean() \
        >= 11 / 12


def test_forward_mode_baselines_refuse_the_nonseparable_model(mdf96):
    from paper_2506_19919_gb300 import SpsError
    wl, ctx = mdf96
    with pytest.raises(SpsError):
        ctx.loglike_grad_forward_mode(wl.theta, np.full((wl.n_gal, 6), 23.0), wl.sigma, wl.mask)
