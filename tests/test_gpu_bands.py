"""Tabulated filter curves on the GPU: photometry (approximate, exact FP32 /
BF16 / 3xTF32), log L + gradient and the HMC kernel with a filter set that
mixes tabulated curves (linear interpolant of uniform samples) with
Gaussian and top-hat bands, against the FP64 oracle on the production grid.
Tolerances as in test_gpu_parity."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import hmc as OH
from oracle import sps as O
from paper_2506_19919_gb300 import loaders as Ld

pytestmark = pytest.mark.gpu


def _mixed_bands():
    """Six bands 320-1060 nm: synthetic measured-style curves, with band 1 a
    Gaussian and band 4 a top-hat so every kind is dispatched."""
    k, p0, p1, n, T = W.tabulated_bands(np.random.default_rng(77), [320, 400, 552, 691, 818, 922, 1060])
    offs = np.concatenate([[0], np.cumsum(n)])
    bands = []
    for b in range(6):
        if b == 1:
            bands.append(("gauss", 4760.0, 1000.0))
        elif b == 4:
            bands.append(("tophat", 8180.0, 9220.0))
        else:
            bands.append(Ld.Curve(float(p0[b]), float(p1[b]), T[offs[b]:offs[b + 1]]))
    return Ld.filter_set(bands)


@pytest.fixture(scope="module")
def tab96():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(1, n_gal=96)
    wl.tables = W.with_bands(wl.tables, *_mixed_bands())
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    yield wl, ctx
    ctx.close()


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-3), ("exact", "fp32", 1e-3),
                                           ("exact", "bf16", 5e-3), ("exact", "tf32x3", 1e-3)])
def test_tabulated_band_photometry(tab96, mode, prec, tol):
    wl, ctx = tab96
    m = ctx.photometry(wl.theta, mode=mode, prec=prec).cpu().numpy()
    ref = O.photometry(wl.theta, wl.z, wl.tables, mode).numpy()
    assert np.isfinite(m).all()
    assert np.abs(m - ref).max() < tol


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-4), ("exact", "fp32", 1e-4),
                                           ("exact", "bf16", 1e-2)])
def test_tabulated_band_loglike_grad(tab96, mode, prec, tol):
    wl, ctx = tab96
    th_true = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    ref_mode = "exact" if mode == "exact" else "approx"
    mobs = O.photometry(th_true, wl.z, wl.tables, ref_mode).numpy() + wl.noise
    ev = W.prior_draw(np.random.default_rng(19), wl.n_gal)
    ll, g = ctx.loglike_grad(ev, mobs, wl.sigma, wl.mask, mode=mode, prec=prec)
    llr, gr, _ = O.loglike_and_grad(ev, wl.z, wl.tables, mobs, wl.sigma, wl.mask, ref_mode)
    np.testing.assert_allclose(ll.cpu().numpy(), llr.numpy(), rtol=2e-4 if prec == "fp32" else 5e-3)
    g, gr = g.cpu().numpy().astype(np.float64), gr.numpy()
    assert (np.abs(g - gr).max(1) / np.abs(gr).max(1)).max() < tol


def test_tabulated_band_hmc_matches_oracle_draws(tab96):
    """The persistent HMC kernel on c_SSP tables built from tabulated curves:
    draws follow the oracle's chain by chain at a fixed step size."""
    wl, ctx = tab96
    G, C = 3, 4
    th_true = torch.as_tensor(wl.theta_true[:G], dtype=torch.float64)
    mobs = O.photometry(th_true, wl.z[:G], wl.tables, "approx").numpy() + wl.noise[:G]
    mobs_all = np.full((wl.n_gal, 6), 30.0)
    mobs_all[:G] = mobs
    mask = np.zeros(wl.n_gal, np.uint32)
    mask[:G] = wl.mask[:G]
    x0 = np.repeat(W.unbounded_of(wl.theta_true[:G]), C, axis=0)
    x0 = (x0 + np.random.default_rng(8).normal(0, 0.02, x0.shape)).astype(np.float32)
    x0_all = np.zeros((wl.n_gal * C, 12), np.float32)
    x0_all[:G * C] = x0
    out = ctx.hmc_run(x0_all, mobs_all, wl.sigma, mask, chains_per_gal=C, n_warm=0, n_samp=6, L_min=6, L_max=6,
                      seed=41, eps0=2e-3, autotune=False)
    s = out["samples"].cpu().numpy()[:G * C]
    tgt = OH.ApproxTarget(wl.tables, wl.z[:G], mobs, wl.sigma[:G], wl.mask[:G], W.PRIOR_LO, W.PRIOR_HI)
    ref = OH.run_hmc(tgt, x0.astype(np.float64), np.repeat(np.arange(G), C), seed=41, n_warm=0, n_samp=6,
                     L_min=6, L_max=6, eps0=2e-3)
    span = W.PRIOR_HI - W.PRIOR_LO
    d = np.abs((s - ref["samples"]) / span).max(axis=(1, 2))
    assert (d < 2e-5).mean() >= 11 / 12
