"""The torch.autograd.Function around the library's hand-written adjoint,
driven through the real CUDA library.

On 96 galaxies of the production grid (107 x 12 x 5994, six Gaussian bands),
log L is computed by `autograd.loglike` with a theta that requires grad, and
torch.autograd.grad gives d log L / d theta.  It is checked
  * against the FP64 oracle's gradient (reverse-mode autodiff of its own
    definition), max-component relative error per row <= 1e-4 for the FP32
    paths (approximate; exact on the SIMT and TF32x3 tensor-core kernels:
    the latter at its stated 2e-3) and <= 1e-2 for the BF16 contraction;
  * against central differences of the library's own FP32 log L with
    h = 1e-3 x the prior span, at a point away from the data (FP32 rounding of
    log L ~ 1e4 gives ~1e-5 of the gradient's scale at that step, and the
    truncation error is O(h^2)), to 2e-3 of the largest component;
  * for the backward pass's scaling: a weighted sum of log L back-propagates
    the weights times the gradient.
"""
import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O

pytestmark = pytest.mark.gpu


def _rel(g, ref):
    g, ref = np.asarray(g, np.float64), np.asarray(ref, np.float64)
    return (np.abs(g - ref).max(1) / np.abs(ref).max(1)).max()


@pytest.fixture(scope="module")
def prod96():
    import paper_2506_19919_gb300 as pkg
    wl = W.config(1, n_gal=96)
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    th_true = torch.as_tensor(wl.theta_true, dtype=torch.float64)
    data = {}
    for mode in ("approx", "exact"):
        mobs = O.photometry(th_true, wl.z, wl.tables, mode).numpy() + wl.noise
        data[mode] = mobs
    yield wl, ctx, data
    ctx.close()


# (mode, precision, log L relative tolerance, gradient tolerance): the bars of
# the parity tests for each path
@pytest.mark.parametrize("mode,prec,ltol,tol", [("approx", "fp32", 2e-4, 1e-4), ("exact", "fp32", 2e-4, 1e-4),
                                                ("exact", "tf32x3", 5e-4, 2e-3),
                                                ("exact", "bf16", 5e-3, 1e-2)])
def test_autograd_matches_oracle_gradient(prod96, mode, prec, ltol, tol):
    from paper_2506_19919_gb300 import autograd as AG
    wl, ctx, data = prod96
    dev = torch.device("cuda", 0)
    mobs = torch.as_tensor(data[mode], dtype=torch.float32, device=dev)
    sg = torch.as_tensor(wl.sigma, dtype=torch.float32, device=dev)
    mk = torch.as_tensor(wl.mask.view(np.int32), device=dev)
    ev = W.prior_draw(np.random.default_rng(23), wl.n_gal)         # independent evaluation point
    theta = torch.as_tensor(ev, dtype=torch.float32, device=dev).requires_grad_(True)
    ll = AG.loglike(theta, ctx, mobs, sg, mk, mode=mode, prec=prec)
    assert ll.requires_grad and ll.shape == (wl.n_gal,)
    w = torch.linspace(0.5, 2.0, wl.n_gal, device=dev)
    (gw,) = torch.autograd.grad((w * ll).sum(), theta)
    llr, gr, _ = O.loglike_and_grad(ev, wl.z, wl.tables, data[mode], wl.sigma, wl.mask, mode)
    np.testing.assert_allclose(ll.detach().cpu().numpy(), llr.numpy(), rtol=ltol)
    g = (gw / w[:, None]).cpu().numpy()
    assert _rel(g, gr.numpy()) < tol


def test_autograd_matches_central_differences_of_the_library(prod96):
    from paper_2506_19919_gb300 import autograd as AG
    wl, ctx, data = prod96
    dev = torch.device("cuda", 0)
    n = 32
    gi = torch.arange(n, dtype=torch.int32, device=dev)
    ev = W.prior_draw(np.random.default_rng(29), n)
    theta = torch.as_tensor(ev, dtype=torch.float32, device=dev).requires_grad_(True)
    # the data arrays cover all galaxies of the set; rows pick theirs by gal_idx
    mobs_all = torch.as_tensor(data["approx"], dtype=torch.float32, device=dev)
    sg_all = torch.as_tensor(wl.sigma, dtype=torch.float32, device=dev)
    mk_all = torch.as_tensor(wl.mask.view(np.int32), device=dev)
    ll = AG.loglike(theta, ctx, mobs_all, sg_all, mk_all, gal_idx=gi, mode="approx")
    (g,) = torch.autograd.grad(ll.sum(), theta)
    g = g.cpu().numpy().astype(np.float64)
    span = (W.PRIOR_HI - W.PRIOR_LO)
    fd = np.zeros_like(g)
    for k in range(12):
        h = 1e-3 * span[k]
        tp = ev.copy()
        tm = ev.copy()
        tp[:, k] += h
        tm[:, k] -= h
        lp, _ = ctx.loglike_grad(tp, mobs_all, sg_all, mk_all, gal_idx=gi, mode="approx", grad=False)
        lm, _ = ctx.loglike_grad(tm, mobs_all, sg_all, mk_all, gal_idx=gi, mode="approx", grad=False)
        # the step actually taken, after rounding theta +- h to float32
        hk = (tp[:, k].astype(np.float32).astype(np.float64) - tm[:, k].astype(np.float32).astype(np.float64))
        fd[:, k] = (lp.cpu().numpy().astype(np.float64) - lm.cpu().numpy().astype(np.float64)) / hk
    assert np.abs(ll.detach().cpu().numpy()).min() > 10.0            # away from the data
    assert _rel(g, fd) < 2e-3
