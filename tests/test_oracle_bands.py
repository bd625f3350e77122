"""Tabulated filter curves (user-supplied throughputs): pins of the oracle's
linear-interpolant transmission and the host loaders (CPU only)."""
import math

import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O
from paper_2506_19919_gb300 import loaders as Ld

DT = torch.float64
FWHM_TO_SIGMA = 1.0 / (2.0 * math.sqrt(2.0 * math.log(2.0)))


def _gauss_curve(centre, fwhm, step):
    s = fwhm * FWHM_TO_SIGMA
    lam = np.arange(centre - 9 * s, centre + 9 * s + step, step)
    return Ld.Curve(float(lam[0]), step, np.exp(-0.5 * ((lam - centre) / s) ** 2))


def _tables(bands):
    base = W.config(1, n_gal=1).tables
    return W.with_bands(base, *Ld.filter_set(bands))


def test_sampled_gaussian_converges_to_the_analytic_band_at_second_order():
    """A Gaussian band sampled every h and linearly interpolated gives the
    analytic Gaussian band's magnitudes up to O(h^2)."""
    z = torch.tensor([0.2, 1.3], dtype=DT)
    th = torch.as_tensor(W.config(1, n_gal=2).theta_true[:2])
    ref = O.photometry(th, z, _tables([("gauss", 6000.0, 1500.0), ("gauss", 9000.0, 800.0)]), "exact")
    errs = []
    for h in (40.0, 20.0, 10.0):
        tabs = _tables([_gauss_curve(6000.0, 1500.0, h), _gauss_curve(9000.0, 800.0, h)])
        errs.append(float((O.photometry(th, z, tabs, "exact") - ref).abs().max()))
    assert errs[-1] < 2e-4
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_interpolant_is_exact_at_samples_and_linear_between():
    tabs = _tables([Ld.Curve(4000.0, 50.0, np.array([0.0, 0.3, 0.9, 0.6, 0.0]))])
    lam = torch.tensor([[3999.0, 4000.0, 4050.0, 4075.0, 4100.0, 4137.5, 4200.0, 4200.01]], dtype=DT)
    T = O.transmission(tabs, lam)[0, 0].numpy()
    np.testing.assert_allclose(T, [0.0, 0.0, 0.3, 0.6, 0.9, 0.675, 0.0, 0.0], atol=1e-14)


def test_flat_fnu_source_gives_ab_zero_point_with_tabulated_bands():
    k, p0, p1, n, T = W.tabulated_bands(np.random.default_rng(3), [320, 400, 552, 691, 818, 922, 1060])
    base = W.config(1, n_gal=1).tables
    tabs = W.with_bands(base, k, p0, p1, n, T)
    z = torch.tensor([0.3, 1.7], dtype=DT)
    w, nb, _ = O.band_weights(tabs, z)
    sed = torch.full((2, tabs.n_lam), 7.5, dtype=DT)
    m = O.magnitudes(O.band_flux(sed, torch.ones_like(sed), w), nb, z)
    dl = O.lum_dist_mpc(z.numpy()) * O.MPC_CM
    ref = -2.5 * torch.log10((1 + z) * O.L_SUN_ERG_S * 7.5 / (4 * math.pi * dl ** 2 * O.AB_ZP_CGS))
    torch.testing.assert_close(m, ref[:, None].expand_as(m), rtol=0, atol=1e-12)
    # lambda_eff of each band lies inside its rest-frame support
    le = O.lambda_eff(tabs, z).numpy()
    lo = p0[None, :] / (1 + z.numpy()[:, None])
    hi = (p0 + (n - 1) * p1)[None, :] / (1 + z.numpy()[:, None])
    assert np.all(le > lo) and np.all(le < hi)


def test_loader_reads_and_resamples_a_throughput_file(tmp_path):
    lam_nm = np.array([500.0, 500.5, 501.0, 502.0, 503.5, 504.0])
    thr = np.array([0.0, 0.2, 0.5, 0.7, 0.4, 0.0])
    f = tmp_path / "band.dat"
    f.write_text("# wavelength(nm) throughput\n" + "\n".join(f"{a} {b}" for a, b in zip(lam_nm, thr)))
    c = Ld.load_filter_curve(f, unit="nm")
    assert c.start == pytest.approx(5000.0) and c.step == pytest.approx(5.0) and len(c.T) == 9
    tabs = _tables([c])
    T = O.transmission(tabs, torch.as_tensor(lam_nm * 10.0)[None, :])[0, 0].numpy()
    np.testing.assert_allclose(T, thr, atol=1e-12)            # samples on the new grid are kept
    c2 = Ld.load_filter_curve(f, unit="nm", step_ang=2.5)
    assert len(c2.T) == 17
    with pytest.raises(ValueError):
        Ld.resample_curve([1.0, 1.0, 2.0], [0.1, 0.2, 0.3])


def test_loader_reads_an_ssp_file(tmp_path):
    rng = np.random.default_rng(0)
    lgmet = np.array([-1.0, -0.5, 0.0])
    lgage = np.linspace(-3, 1.1, 7)
    wave = np.geomspace(1000, 20000, 50)
    flux = rng.uniform(0.1, 1.0, (3, 7, 50))
    p = tmp_path / "ssp.npz"
    np.savez(p, ssp_lgmet=lgmet, ssp_lg_age_gyr=lgage, ssp_wave=wave, ssp_flux=flux)
    t = Ld.tables(p, [("gauss", 5000.0, 1000.0), _gauss_curve(7000.0, 1200.0, 10.0)])
    assert t.ssp.shape == (7, 3, 50) and t.n_band == 2
    np.testing.assert_array_equal(t.ssp[:, 1, :], flux[1])
    np.testing.assert_allclose(t.age_yr, 10 ** (lgage + 9))
    assert list(t.band_kind) == [1, 2] and t.band_tab_n[0] == 0 and t.band_tab_T.size == t.band_tab_n[1]
