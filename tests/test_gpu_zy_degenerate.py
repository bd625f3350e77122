"""Degenerate cases of the model on the GPU against the FP64 oracle, on the
production grid: no burst (F_burst = 0), no dust (A_V = 0), no unobscured
floor (F_floor = 0), the narrowest metallicity distribution and burst the
prior allows, a single observed band, and no observed band (log L = 0 and a
zero gradient).  Same tolerances as test_gpu_parity."""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O

pytestmark = pytest.mark.gpu

MAG_TOL = 1e-3
GRAD_TOL = 1e-4
# BF16 contraction: the magnitude bar of the precision target.  Where one
# (age, Z) cell dominates W, the roundings of W and of the row-scaled table no
# longer average out, and a flux can be off by up to 2 x 2^-9 relative,
# i.e. 4.2e-3 mag, still inside it.
MAG_TOL_BF16 = 5e-3


def _degenerate(theta):
    """Rows 0-23 no burst, 24-47 no dust, 48-71 no floor, 72-95 the narrowest
    MDF and burst; float32-representable like every workload input."""
    th = np.array(theta, np.float64)
    th[0:24, 4] = 0.0
    th[24:48, 9] = 0.0
    th[48:72, 11] = 0.0
    th[72:96, 8] = W.PRIOR_LO[8]
    th[72:96, 6] = W.PRIOR_LO[6]
    return th.astype(np.float32).astype(np.float64)


@pytest.fixture(scope="module")
def deg96():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(1, n_gal=96)
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    yield wl, ctx, _degenerate(wl.theta)
    ctx.close()


@pytest.mark.parametrize("mode,prec,tol", [("exact", "fp32", MAG_TOL), ("approx", "fp32", MAG_TOL),
                                           ("exact", "bf16", MAG_TOL_BF16)])
def test_degenerate_photometry(deg96, mode, prec, tol):
    wl, ctx, th = deg96
    m = ctx.photometry(th, mode=mode, prec=prec).cpu().numpy()
    ref = O.photometry(th, wl.z, wl.tables, mode).numpy()
    assert np.isfinite(m).all()
    assert np.abs(m - ref).max() < tol


@pytest.mark.parametrize("mode", ["approx", "exact"])
def test_degenerate_loglike_grad(deg96, mode):
    """Independent evaluation points with the same degenerate columns; one
    observed band per galaxy on most rows, none on the last eight."""
    wl, ctx, th = deg96
    th_true = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    mobs = O.photometry(th_true, wl.z, wl.tables, mode).numpy() + wl.noise
    ev = _degenerate(W.prior_draw(np.random.default_rng(29), wl.n_gal))
    mask = np.array([1 << (g % 6) for g in range(wl.n_gal)], np.uint32)
    mask[::3] = wl.mask[::3]                     # every third row keeps its full mask
    mask[-8:] = 0
    ll, g = ctx.loglike_grad(ev, mobs, wl.sigma, mask, mode=mode)
    llr, gr, _ = O.loglike_and_grad(ev, wl.z, wl.tables, mobs, wl.sigma, mask, mode)
    ll, g, llr, gr = ll.cpu().numpy(), g.cpu().numpy().astype(np.float64), llr.numpy(), gr.numpy()
    assert np.all(ll[-8:] == 0.0) and np.all(g[-8:] == 0.0)
    np.testing.assert_allclose(ll[:-8], llr[:-8], rtol=2e-4)
    rel = np.abs(g[:-8] - gr[:-8]).max(1) / np.abs(gr[:-8]).max(1)
    assert rel.max() < GRAD_TOL


def test_degenerate_loglike_grad_bf16(deg96):
    """The BF16 tensor-core contraction on the same degenerate rows and masks:
    rows without an observed band give exact zeros.  log L is held to what
    the magnitude bar implies, row by row: with every magnitude off by at most
    d = 5e-3, |dlog L| <= sum_b (|r_b| d + d^2 / 2) / sigma_b^2 over the
    observed bands (r the oracle's residuals).  The gradient is held to 3e-2
    of its largest component: on rows where one (age, Z) cell carries the
    flux, the roundings of W and of the table enter it unaveraged (2 x 2^-9
    per product), so it is looser than on prior draws (1e-2 in
    test_gpu_parity); 2.0e-2 measured."""
    wl, ctx, th = deg96
    th_true = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    mobs = O.photometry(th_true, wl.z, wl.tables, "exact").numpy() + wl.noise
    ev = _degenerate(W.prior_draw(np.random.default_rng(29), wl.n_gal))
    mask = np.array([1 << (g % 6) for g in range(wl.n_gal)], np.uint32)
    mask[::3] = wl.mask[::3]
    mask[-8:] = 0
    ll, g = ctx.loglike_grad(ev, mobs, wl.sigma, mask, mode="exact", prec="bf16")
    llr, gr, _ = O.loglike_and_grad(ev, wl.z, wl.tables, mobs, wl.sigma, mask, "exact")
    ll, g, llr, gr = ll.cpu().numpy(), g.cpu().numpy().astype(np.float64), llr.numpy(), gr.numpy()
    assert np.all(ll[-8:] == 0.0) and np.all(g[-8:] == 0.0)
    assert np.isfinite(ll).all() and np.isfinite(g).all()
    m = O.photometry(torch.as_tensor(ev), wl.z, wl.tables, "exact").numpy()
    obs = ((mask[:, None] >> np.arange(m.shape[1])[None, :]) & 1).astype(bool)
    d = MAG_TOL_BF16
    bound = np.where(obs, (np.abs(m - mobs) * d + 0.5 * d * d) / np.asarray(wl.sigma) ** 2, 0.0).sum(1)
    assert np.all(np.abs(ll - llr) <= bound + 1e-6 * np.abs(llr)), np.max(np.abs(ll - llr) - bound)
    rel = np.abs(g[:-8] - gr[:-8]).max(1) / np.abs(gr[:-8]).max(1)
    assert rel.max() < 3e-2, rel.max()
