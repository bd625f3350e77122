"""The large bursty-SFH survey batch at full size: 1,000,000 galaxies x 2
chains, 20 Gaussian bands 300-2400 nm with 6-20 observed per galaxy, burst
component on, z ~ U(0.05, 3).  One context holds the whole batch (the
per-galaxy approximate tables are 103 GB of HBM); the exact path runs with
BF16 operands, the approximate path in FP32.  Sampled rows and chains are
checked against the FP64 oracle.

Tolerances as in test_gpu_parity: 1e-3 mag (FP32), 5e-3 mag (BF16), gradients
1e-4 (FP32) / 1e-2 (BF16) of the largest component per row."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import hmc as OH
from oracle import sps as O

pytestmark = pytest.mark.gpu

G_FULL = 1_000_000


@pytest.fixture(scope="module")
def survey():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(4)
    assert wl.n_gal == G_FULL and wl.tables.n_band == 20
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    pick = np.unique(np.concatenate([[0, 1, 31, 32, G_FULL - 2, G_FULL - 1],
                                     np.random.default_rng(41).integers(0, G_FULL, 10)]))
    yield wl, ctx, pick
    ctx.close()


def test_survey_photometry_sampled_rows(survey):
    """Whole-batch photometry in one call per path; sampled rows vs the oracle."""
    wl, ctx, pick = survey
    th = torch.as_tensor(wl.theta_true, dtype=torch.float32, device="cuda")
    m_ap = ctx.photometry(th, mode="approx").cpu().numpy()
    m_bf = ctx.photometry(th, mode="exact", prec="bf16").cpu().numpy()
    assert m_ap.shape == (G_FULL, 20) and np.isfinite(m_ap).all() and np.isfinite(m_bf).all()
    ref_ap = O.photometry(wl.theta_true[pick], wl.z[pick], wl.tables, "approx").numpy()
    ref_ex = O.photometry(wl.theta_true[pick], wl.z[pick], wl.tables, "exact").numpy()
    assert np.abs(m_ap[pick] - ref_ap).max() < 1e-3
    assert np.abs(m_bf[pick] - ref_ex).max() < 5e-3


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-4), ("exact", "bf16", 1e-2)])
def test_survey_loglike_grad_sampled_rows(survey, mode, prec, tol):
    """log L and its gradient for every galaxy with its own band mask (6-20
    observed bands); sampled rows vs the oracle."""
    wl, ctx, pick = survey
    mobs = (np.full((G_FULL, 20), 23.0) + wl.noise).astype(np.float32)
    ev = W.prior_draw(np.random.default_rng(43), G_FULL)
    ll, g = ctx.loglike_grad(ev, mobs, wl.sigma, wl.mask, mode=mode, prec=prec)
    llr, gr, _ = O.loglike_and_grad(ev[pick], wl.z[pick], wl.tables, mobs[pick].astype(np.float64),
                                    wl.sigma[pick], wl.mask[pick], mode)
    np.testing.assert_allclose(ll.cpu().numpy()[pick], llr.numpy(), rtol=2e-4 if prec == "fp32" else 5e-3)
    g, gr = g.cpu().numpy()[pick].astype(np.float64), gr.numpy()
    assert (np.abs(g - gr).max(1) / np.abs(gr).max(1)).max() < tol


def test_survey_hmc_full_batch_sampled_chains(survey):
    """The batched sampler over all 2,000,000 chains in one launch; at a fixed
    step size the chains of sampled galaxies follow the oracle's HMC draw by
    draw (20 bands, uneven masks, burst on)."""
    wl, ctx, pick = survey
    C = 2
    th_true = torch.as_tensor(wl.theta_true[pick], dtype=torch.float64)
    mobs = np.full((G_FULL, 20), 30.0, np.float32)
    mobs_pick = O.photometry(th_true, wl.z[pick], wl.tables, "approx").numpy() + wl.noise[pick]
    mobs[pick] = mobs_pick
    x0 = W.unbounded_of(np.repeat(wl.theta_true, C, axis=0))
    x0 = (x0 + np.random.default_rng(47).normal(0, 0.02, x0.shape)).astype(np.float32)
    out = ctx.hmc_run(x0, mobs, wl.sigma, wl.mask, chains_per_gal=C, n_warm=0, n_samp=3,
                      L_min=6, L_max=6, seed=13, eps0=2e-3)
    s = out["samples"]
    assert s.shape == (G_FULL * C, 3, 12)
    assert bool(torch.isfinite(s).all())
    acc = out["accept_prob"].cpu().numpy()
    assert ((acc >= 0) & (acc <= 1)).all()
    assert (out["grad_evals"].cpu().numpy() == 1 + 3 * 6).all()
    chains = (pick[:, None] * C + np.arange(C)[None, :]).ravel()
    tgt = OH.ApproxTarget(wl.tables, wl.z[pick], mobs_pick, wl.sigma[pick], wl.mask[pick],
                          W.PRIOR_LO, W.PRIOR_HI)
    ref = OH.run_hmc(tgt, x0[chains].astype(np.float64), np.repeat(np.arange(len(pick)), C), seed=13,
                     n_warm=0, n_samp=3, L_min=6, L_max=6, eps0=2e-3, chain_ids=chains)
    span = W.PRIOR_HI - W.PRIOR_LO
    d = np.abs((s.cpu().numpy()[chains] - ref["samples"]) / span).max(axis=(1, 2))
    assert (d < 2e-5).mean() >= 0.9
