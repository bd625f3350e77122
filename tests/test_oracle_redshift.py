"""Pins of the oracle's redshift derivative (the 13th gradient column).

d log L / dz runs through t_obs(z) (age bins, M_star, burst clipping), the
observed-frame filter T((1+z) lambda), N_b(z), d_L(z) and the (1+z)
bandwidth factor.  The two cosmological derivatives are held to textbook
identities and to central differences of the FP64 quadrature; the whole
column to central differences of the oracle's own log L in z; a dropped
term planted in the oracle fails the same check."""
import math

import numpy as np
import pytest
import torch
from scipy import integrate

import sps_workloads as W
from oracle import sps as O

DT = torch.float64


def test_cosmic_age_derivative_is_minus_one_over_one_plus_z_H():
    """dt/dz = -1 / ((1+z) H(z)) for any Friedmann model."""
    z = torch.tensor([0.05, 0.5, 1.3, 3.0], dtype=DT, requires_grad=True)
    (g,) = torch.autograd.grad(O.t_obs_gyr(z).sum(), z)
    ref = -O.hubble_time_gyr() / ((1 + z.detach()) * O.hubble_e(z.detach()))
    torch.testing.assert_close(g, ref, rtol=1e-12, atol=0)


def test_luminosity_distance_derivative():
    """d d_L / dz against central differences of the adaptive quadrature
    (h = 1e-5, truncation ~1e-11) and against the comoving-distance identity
    d_C' = c / H(z) evaluated by an independent SciPy integral."""
    z = torch.tensor([0.05, 0.5, 1.3, 3.0], dtype=DT, requires_grad=True)
    (g,) = torch.autograd.grad(O.lum_dist_mpc_t(z).sum(), z)
    h = 1e-5
    zn = z.detach().numpy()
    fd = (O.lum_dist_mpc(zn + h) - O.lum_dist_mpc(zn - h)) / (2 * h)
    torch.testing.assert_close(g, fd, rtol=1e-8, atol=0)
    for zi, gi in zip(zn, g.tolist()):
        dc, _ = integrate.quad(lambda x: 1.0 / math.sqrt(0.3 * (1 + x) ** 3 + 0.7), 0, zi,
                               epsabs=0, epsrel=1e-13)
        dc *= O.C_KMS / O.H0_KMS_MPC
        ref = dc + (1 + zi) * O.C_KMS / O.H0_KMS_MPC / math.sqrt(0.3 * (1 + zi) ** 3 + 0.7)
        assert gi == pytest.approx(ref, rel=1e-11)


def _fd_z(theta, z, tables, mobs, sigma, mask, mode, h):
    lp = O.loglike(O.photometry(theta, z + h, tables, mode), mobs, sigma, mask)
    lm = O.loglike(O.photometry(theta, z - h, tables, mode), mobs, sigma, mask)
    return (lp - lm) / (2 * h)


def _z_case(tabs):
    rng = np.random.default_rng(41)
    n = 6
    th = torch.as_tensor(W.prior_draw(rng, n), dtype=DT)
    th[:, 4] = torch.linspace(0.0, 0.2, n, dtype=DT)          # burst on in most rows
    z = torch.as_tensor([0.07, 0.3, 0.8, 1.4, 2.2, 2.9], dtype=DT)
    mobs = O.photometry(torch.as_tensor(W.prior_draw(rng, n), dtype=DT), z, tabs, "exact") + 0.2
    sigma = np.full((n, tabs.n_band), 0.05)
    mask = np.full(n, (1 << tabs.n_band) - 1, np.uint32)
    return th, z, mobs, sigma, mask


@pytest.mark.parametrize("mode", ["exact", "approx"])
@pytest.mark.parametrize("bands", ["gauss", "tabulated"])
def test_redshift_gradient_against_central_differences(mode, bands):
    tabs = W.config(1, n_gal=1).tables
    if bands == "tabulated":
        tabs = W.with_bands(tabs, *W.tabulated_bands(np.random.default_rng(3),
                                                     [360, 482, 604, 726, 848, 970]))
    th, z, mobs, sigma, mask = _z_case(tabs)
    ll, g, _ = O.loglike_and_grad(th, z, tabs, mobs, sigma, mask, mode, wrt_z=True)
    ll0, g0, _ = O.loglike_and_grad(th, z, tabs, mobs, sigma, mask, mode)
    torch.testing.assert_close(g[:, :12], g0, rtol=0, atol=0)
    torch.testing.assert_close(ll, ll0, rtol=0, atol=0)
    fd = _fd_z(th, z, tabs, mobs, sigma, mask, mode, 1e-6)
    # Gaussian bands: smooth in z (truncation ~1e-12); tabulated: the linear
    # interpolant has kinks every sample, crossed by a few grid points
    tol = 1e-8 if bands == "gauss" else 3e-5
    assert ((g[:, 12] - fd).abs() / fd.abs()).max() < tol


def test_redshift_gradient_rejects_planted_mistakes(monkeypatch):
    """Dropping the (1+z)^2 c/(H0 E) part of d_L', or the t_obs dependence of
    the age bins, breaks agreement with central differences."""
    tabs = W.config(1, n_gal=1).tables
    th, z, mobs, sigma, mask = _z_case(tabs)
    fd = _fd_z(th, z, tabs, mobs, sigma, mask, "exact", 1e-6)

    def err():
        _, g, _ = O.loglike_and_grad(th, z, tabs, mobs, sigma, mask, "exact", wrt_z=True)
        return float(((g[:, 12] - fd).abs() / fd.abs()).max())

    assert err() < 1e-8
    with monkeypatch.context() as m:
        m.setattr(O._LumDist, "backward",
                  staticmethod(lambda ctx, gr: gr * ctx.saved_tensors[1] / (1 + ctx.saved_tensors[0])))
        assert err() > 1e-3
    with monkeypatch.context() as m:
        t_obs = O.t_obs_gyr
        m.setattr(O, "t_obs_gyr", lambda zz, *a, **k: t_obs(zz.detach(), *a, **k))
        assert err() > 1e-3
