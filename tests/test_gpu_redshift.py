"""The redshift column of the gradient (sps_loglike_grad_z) against the FP64
oracle's d log L / dz.

96 galaxies (one full 64-row tile and a ragged one) of the production grid
(107 x 12 x 5994), z ~ U(0.05, 3), an evaluation point independent of the
data, the burst on in most rows.  Bar: per row, max over the 13 columns of
|g - g_ref| / max |g_ref| <= 1e-4 for the FP32 paths (approximate, exact
SIMT), 2e-3 for 3xTF32 and 1e-2 for the BF16 contraction (the bars of the
12-column gradient tests); the first 12 columns also equal those of
sps_loglike_grad to the same bar.  Gaussian bands (six, R = 3.4-25.5) and a
tabulated filter set; a top-hat set is refused."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O

pytestmark = pytest.mark.gpu


def _rel(g, ref):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    return (np.abs(g - ref).max(1) / np.abs(ref).max(1)).max()


def _where(g, ref):
    """Row and column of the largest relative error, and that column's error
    over all rows (for the assertion message)."""
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    e = np.abs(g - ref) / np.abs(ref).max(1, keepdims=True)
    r, k = np.unravel_index(np.argmax(e), e.shape)
    return f"row {r} col {k}: {e[r, k]:.3g} (g {g[r, k]:.6g} ref {ref[r, k]:.6g}); per-column max {e.max(0).round(7).tolist()}"


def _case(tabs, n=96, seed=5):
    rng = np.random.default_rng(seed)
    z = np.round(rng.uniform(0.05, 3.0, n), 4).astype(np.float32).astype(np.float64)
    truth = W.prior_draw(rng, n)
    ev = W.prior_draw(rng, n)
    mask = np.full(n, (1 << tabs.n_band) - 1, np.uint32)
    mask[::3] &= ~np.uint32(0b101)                       # uneven band sets
    sigma = np.full((n, tabs.n_band), 0.05)
    return z, truth, ev, mask, sigma


def _ctx(tabs, z):
    import paper_2506_19919_gb300 as pkg
    ctx = pkg.Context(tabs, device=0)
    ctx.set_galaxies(z, build_approx=True)
    return ctx


@pytest.fixture(scope="module")
def gauss96():
    tabs = W.config(1, n_gal=1).tables
    z, truth, ev, mask, sigma = _case(tabs)
    ctx = _ctx(tabs, z)
    yield tabs, z, truth, ev, mask, sigma, ctx
    ctx.close()


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-4), ("exact", "fp32", 1e-4),
                                           ("exact", "tf32x3", 2e-3), ("exact", "bf16", 1e-2)])
def test_redshift_gradient_gaussian_bands(gauss96, mode, prec, tol):
    tabs, z, truth, ev, mask, sigma, ctx = gauss96
    mobs = O.photometry(truth, z, tabs, mode).numpy() + 0.02
    ll, g = ctx.loglike_grad_z(ev, mobs, sigma, mask, mode=mode, prec=prec)
    llr, gr, _ = O.loglike_and_grad(ev, z, tabs, mobs, sigma, mask, mode, wrt_z=True)
    g = g.cpu().numpy()
    assert g.shape == (96, 13)
    assert _rel(g, gr.numpy()) < tol, _where(g, gr.numpy())
    # the z column on its own scale as well
    zr = np.abs(g[:, 12] - gr.numpy()[:, 12]) / np.abs(gr.numpy()).max(1)
    assert zr.max() < tol
    ll12, g12 = ctx.loglike_grad(ev, mobs, sigma, mask, mode=mode, prec=prec)
    assert _rel(g[:, :12], g12.cpu().numpy()) < tol
    np.testing.assert_allclose(ll.cpu().numpy(), ll12.cpu().numpy(), rtol=1e-5, atol=1e-3)


@pytest.mark.parametrize("mode,prec,tol", [("approx", "fp32", 1e-4), ("exact", "fp32", 1e-4),
                                           ("exact", "bf16", 1e-2)])
def test_redshift_gradient_tabulated_bands(mode, prec, tol):
    base = W.config(1, n_gal=1).tables
    tabs = W.with_bands(base, *W.tabulated_bands(np.random.default_rng(3),
                                                 [360, 482, 604, 726, 848, 970, 1092]))
    z, truth, ev, mask, sigma = _case(tabs, n=70, seed=9)
    ctx = _ctx(tabs, z)
    mobs = O.photometry(truth, z, tabs, mode).numpy() + 0.02
    gi = np.arange(70, dtype=np.int32)[::-1].copy()      # rows through gal_idx
    _, g = ctx.loglike_grad_z(ev[gi], mobs, sigma, mask, gal_idx=gi, mode=mode, prec=prec)
    _, gr, _ = O.loglike_and_grad(ev[gi], z[gi], tabs, mobs[gi], sigma[gi], mask[gi], mode, wrt_z=True)
    g = g.cpu().numpy()
    assert _rel(g, gr.numpy()) < tol, _where(g, gr.numpy())
    ctx.close()


def test_redshift_gradient_refuses_top_hat_bands():
    import paper_2506_19919_gb300 as pkg
    from paper_2506_19919_gb300 import _lib
    wl = W.config(0, n_gal=8)
    ctx = _ctx(wl.tables, wl.z)
    with pytest.raises(pkg.SpsError) as e:
        ctx.loglike_grad_z(wl.theta, np.full((8, 6), 22.0), wl.sigma, wl.mask, mode="approx")
    assert _lib.STATUS_NAMES[e.value.status] == "SPS_E_UNSUPPORTED"
    ctx.close()
