"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: a closed
form, an independent library integrator, brute force on a fine grid, an
invariant or a limiting case.  None of these tests needs a GPU."""
import math

import numpy as np
import pytest
import torch
from scipy import integrate, stats

import sps_workloads as W
from oracle import sps as O

DT = torch.float64


# ---------------------------------------------------------------- constants
def test_physical_constants_against_independent_sources():
    """The oracle's unit constants, against SciPy's CODATA / IAU values and
    the published definitions they follow (the pins below reuse them)."""
    from scipy import constants as K
    assert O.C_KMS == K.c / 1e3                                   # exact by definition
    assert O.MPC_KM == pytest.approx(K.parsec * 1e6 / 1e3, rel=1e-12)
    assert O.MPC_CM == pytest.approx(K.parsec * 1e6 * 1e2, rel=1e-12)
    assert O.GYR_S == pytest.approx(1e9 * K.Julian_year, rel=1e-15)
    assert O.AB_ZP_CGS == pytest.approx(3631 * 1e-26 * 1e3, rel=1e-15)   # 3631 Jy; 1 Jy = 1e-26 W/m^2/Hz
    assert O.L_SUN_ERG_S == pytest.approx(3.828e26 * 1e7, rel=1e-15)      # IAU 2015 B3 nominal, W -> erg/s
    # the Hubble time 977.8 / H0 Gyr (H0 in km/s/Mpc)
    assert O.hubble_time_gyr() == pytest.approx(977.792 / 70.0, rel=1e-5)


# ---------------------------------------------------------------- cosmology
def test_cosmic_age_matches_time_integral():
    th = O.hubble_time_gyr()
    for z in (0.0, 0.5, 3.0):
        direct, _ = integrate.quad(
            lambda x: 1.0 / ((1 + x) * math.sqrt(0.3 * (1 + x) ** 3 + 0.7)), z, np.inf,
            epsabs=0, epsrel=1e-13, limit=500)
        assert float(O.t_obs_gyr(z)) == pytest.approx(th * direct, rel=1e-10)


def test_lum_dist_einstein_de_sitter_closed_form():
    # Omega_m = 1: d_L = (2c/H0)(1+z)(1 - (1+z)^-1/2)
    for z in (0.1, 1.0, 3.0):
        dl = float(O.lum_dist_mpc(z, om=1.0))
        ref = 2 * O.C_KMS / O.H0_KMS_MPC * (1 + z) * (1 - (1 + z) ** -0.5)
        assert dl == pytest.approx(ref, rel=1e-11)


def test_lum_dist_low_z_expansion():
    # d_L = (c z / H0)(1 + (1 - q0) z / 2 + O(z^2)), q0 = Om/2 - OL
    z = 1e-3
    q0 = 0.15 - 0.7
    ref = O.C_KMS * z / O.H0_KMS_MPC * (1 + 0.5 * (1 - q0) * z)
    assert float(O.lum_dist_mpc(z)) == pytest.approx(ref, rel=2e-6)


# ---------------------------------------------------------------- triweight (Eq. triweight)
def test_triweight_is_unit_gaussian_stand_in():
    f = lambda x: float(O.triweight(torch.tensor(x, dtype=DT)))
    norm, _ = integrate.quad(f, -3, 3, epsabs=1e-15)
    var, _ = integrate.quad(lambda x: x * x * f(x), -3, 3, epsabs=1e-15)
    assert norm == pytest.approx(1.0, abs=1e-13)
    assert var == pytest.approx(1.0, abs=1e-13)     # clip at 3 sigma of a unit-sd bump
    h = 1e-6
    assert abs(f(3 - h) - f(3 - 2 * h)) < 1e-12     # vanishing slope at the clip
    assert f(3.0001) == 0.0 and f(-3.0001) == 0.0


def test_triweight_cdf_against_quadrature():
    for x in (-3.5, -2.0, -0.3, 0.0, 1.1, 2.9, 4.0):
        ref, _ = integrate.quad(lambda s: float(O.triweight(torch.tensor(s, dtype=DT))),
                                -3, min(max(x, -3), 3), epsabs=1e-15)
        assert float(O.triweight_cdf(torch.tensor(x, dtype=DT))) == pytest.approx(ref, abs=1e-14)


# ---------------------------------------------------------------- smooth SFH
def _theta(n=6, seed=1):
    return torch.as_tensor(W.prior_draw(np.random.default_rng(seed), n), dtype=DT)


def _plain_sfr(t, tau, a, b):
    return 1.0 / ((t / tau) ** a + (t / tau) ** (-b))


def test_bin_masses_against_adaptive_quadrature():
    tabs = W.config(0).tables
    th = _theta(5)
    z = torch.tensor([0.05, 0.3, 1.0, 2.0, 3.0], dtype=DT)
    t_obs = O.t_obs_gyr(z)
    lo, hi = O.cosmic_time_bins(tabs.age_yr, t_obs)
    m = O.smooth_bin_masses(th, lo, hi)
    for r in range(5):
        tau, a, b = (float(th[r, k]) for k in (1, 2, 3))
        amp = 10 ** float(th[r, 0]) * 1e9
        for i in range(tabs.n_age):
            l, h = float(lo[r, i]), float(hi[r, i])
            if h <= l:
                assert float(m[r, i]) == 0.0
                continue
            ref, _ = integrate.quad(_plain_sfr, l, h, args=(tau, a, b), epsabs=0,
                                    epsrel=1e-13, limit=400)
            assert float(m[r, i]) == pytest.approx(amp * ref, rel=2e-10, abs=1e-300)


def test_bin_masses_alpha_beta_one_closed_form():
    # alpha = beta = 1: int dt / (t/tau + tau/t) = (tau/2) ln(t^2 + tau^2)
    tabs = W.config(3, n_gal=1).tables
    th = _theta(3)
    th[:, 2] = 1.0
    th[:, 3] = 1.0
    t_obs = O.t_obs_gyr(torch.tensor([0.1, 1.0, 2.5], dtype=DT))
    lo, hi = O.cosmic_time_bins(tabs.age_yr, t_obs)
    m = O.smooth_bin_masses(th, lo, hi)
    tau = th[:, 1:2]
    ref = 10 ** th[:, 0:1] * 1e9 * 0.5 * tau * torch.log1p((hi - lo) * (hi + lo) / (lo ** 2 + tau ** 2))
    torch.testing.assert_close(m, ref, rtol=1e-12, atol=0)


def test_bin_mass_brute_force_midpoint():
    th = _theta(1, seed=7)
    th[0, 1:4] = torch.tensor([2.0, 3.0, 0.4], dtype=DT)
    lo = torch.tensor([[0.0, 0.7, 5.0]], dtype=DT)
    hi = torch.tensor([[0.7, 5.0, 5.01]], dtype=DT)
    m = O.smooth_bin_masses(th, lo, hi)[0] / (10 ** th[0, 0] * 1e9)
    n = 2_000_000
    for i in range(3):
        a, b = float(lo[0, i]), float(hi[0, i])
        t = a + (np.arange(n) + 0.5) * (b - a) / n
        bf = _plain_sfr(t, 2.0, 3.0, 0.4).sum() * (b - a) / n
        assert float(m[i]) == pytest.approx(bf, rel=1e-7)


def test_bin_masses_sum_to_total_mass_formed():
    wl = W.config(3, n_gal=64)
    th = torch.as_tensor(wl.theta[::4], dtype=DT)
    t_obs = O.t_obs_gyr(wl.z)
    lo, hi = O.cosmic_time_bins(wl.tables.age_yr, t_obs)
    tot = O.smooth_bin_masses(th, lo, hi).sum(1)
    torch.testing.assert_close(tot, O.total_mass_formed(th, t_obs), rtol=1e-10, atol=0)
    # and the bins tile [0, t_obs] exactly
    torch.testing.assert_close((hi - lo).sum(1), t_obs, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- burst + MDF + weights
def test_burst_weights_normalised_and_brute_force():
    tabs = W.config(0).tables
    th = _theta(4, seed=3)
    z = torch.tensor([0.05, 0.5, 1.0, 3.0], dtype=DT)
    t_obs = O.t_obs_gyr(z)
    pb = O.burst_weights(th, tabs.age_yr, t_obs)
    torch.testing.assert_close(pb.sum(1), torch.ones(4, dtype=DT), rtol=0, atol=1e-14)
    e = O.age_bin_edges_yr(tabs.age_yr)
    for r in range(4):
        mu, sg = float(th[r, 5]), float(th[r, 6]) / 3
        lt = math.log10(float(t_obs[r]) * 1e9)
        x = np.linspace(mu - 3 * sg, mu + 3 * sg, 2_000_001)
        x = 0.5 * (x[1:] + x[:-1])
        dens = (35 / 96) * np.clip(1 - ((x - mu) / sg / 3) ** 2, 0, None) ** 3 / sg
        dens = np.where(x < lt, dens, 0.0)
        le = np.log10(np.where(e > 0, e, 1e-300))
        ref = np.array([dens[(x >= le[i]) & (x < le[i + 1])].sum() for i in range(len(e) - 1)])
        ref /= ref.sum()
        np.testing.assert_allclose(pb[r].numpy(), ref, atol=2e-6)


def test_composite_age_weights_limits():
    wl = W.config(0, n_gal=8)
    th = torch.as_tensor(wl.theta, dtype=DT)
    t_obs = O.t_obs_gyr(wl.z)
    lo, hi = O.cosmic_time_bins(wl.tables.age_yr, t_obs)
    m = O.smooth_bin_masses(th, lo, hi)
    p_smooth = m / m.sum(1, keepdim=True)
    pb = O.burst_weights(th, wl.tables.age_yr, t_obs)
    for fb, ref in ((0.0, p_smooth), (1.0, pb)):
        t2 = th.clone()
        t2[:, 4] = fb
        _, _, p_sfh, _ = O.ssp_weights(t2, wl.tables, t_obs)
        torch.testing.assert_close(p_sfh, ref, rtol=0, atol=1e-15)


def test_burst_peak_shifts_ages_younger():
    # App. A.1 figure on T_peak: smaller T_peak -> younger burst population
    tabs = W.config(0).tables
    th = _theta(2)
    th[:, 6] = 0.6
    th[0, 5], th[1, 5] = 6.5, 8.0
    pb = O.burst_weights(th, tabs.age_yr, O.t_obs_gyr(torch.tensor([0.5, 0.5], dtype=DT)))
    la = torch.log10(torch.as_tensor(tabs.age_yr, dtype=DT))
    mean = (pb * la).sum(1)
    assert mean[0] < mean[1]
    assert float(mean[0]) == pytest.approx(6.5, abs=0.1)


def test_met_weights_against_normal_cdf_and_limits():
    lgz = np.linspace(-2, 0.2, 12)
    th = _theta(5, seed=11)
    q = O.met_weights(th, lgz)
    torch.testing.assert_close(q.sum(1), torch.ones(5, dtype=DT), rtol=0, atol=1e-15)
    e = np.concatenate([[-np.inf], 0.5 * (lgz[1:] + lgz[:-1]), [np.inf]])
    for r in range(5):
        ref = np.diff(stats.norm.cdf(e, loc=float(th[r, 7]), scale=float(th[r, 8])))
        np.testing.assert_allclose(q[r].numpy(), ref, atol=1e-15)
    # narrow limit: all weight on the grid point nearest the mean
    th2 = th.clone()
    th2[:, 7] = torch.as_tensor(lgz[[0, 3, 5, 8, 11]], dtype=DT) + 0.01
    th2[:, 8] = 1e-4
    q2 = O.met_weights(th2, lgz)
    assert torch.allclose(q2.max(1).values, torch.ones(5, dtype=DT))
    assert (q2.argmax(1).numpy() == [0, 3, 5, 8, 11]).all()


def test_weights_sum_to_mass_formed():
    wl = W.config(0, n_gal=16)
    th = torch.as_tensor(wl.theta, dtype=DT)
    Wt, ms, _, _ = O.ssp_weights(th, wl.tables, O.t_obs_gyr(wl.z))
    torch.testing.assert_close(Wt.sum((1, 2)), ms, rtol=1e-14, atol=0)


# ---------------------------------------------------------------- dust (App. A.3)
def test_dust_identities_and_normalisation():
    lam = torch.as_tensor(np.geomspace(912, 25000, 300), dtype=DT)[None, :]
    one = torch.ones(1, 1, dtype=DT)
    for av, dl, ff in ((0.0, -0.5, 0.2), (2.0, 0.3, 1.0)):
        F = O.attenuation(lam, av * one, dl * one, ff * one)
        torch.testing.assert_close(F, torch.ones_like(F), rtol=0, atol=0)
    # the Calzetti curve is normalised so that A(V) ~= A_V, with Calzetti et
    # al.'s (2000) published R_V = 4.05 (k'(V) = R_V)
    k_v = float(O.calzetti_k0(torch.tensor(0.55, dtype=DT)))
    assert k_v == pytest.approx(4.05, abs=0.01)
    F = O.attenuation(torch.tensor([[5500.0]], dtype=DT), 1.0 * one, 0.0 * one, 0.0 * one)
    assert float(-2.5 * torch.log10(F)) == pytest.approx(1.0, abs=0.01)
    # its two fitted branches (UV-optical below 0.63 um, red above) meet at
    # 0.63 um to within 1%, and the curve is small but positive at 2.2 um,
    # the red end of the fit
    kb, kr = O.calzetti_k0(torch.tensor([0.63 - 1e-9, 0.63], dtype=DT)).tolist()
    assert abs(kb - kr) < 0.05
    assert 0.0 < float(O.calzetti_k0(torch.tensor(2.2, dtype=DT))) < 0.5
    # the slope change (lambda / lambda_V)^delta pivots at V: A(V) ~= A_V for any delta
    for dl in (-0.8, -0.3, 0.3, 0.4):
        F = O.attenuation(torch.tensor([[5500.0]], dtype=DT), 1.0 * one, dl * one, 0.0 * one)
        assert float(-2.5 * torch.log10(F)) == pytest.approx(1.0, abs=0.005)
    # attenuation decreases with wavelength over the fitted range
    k = O.calzetti_k0(torch.as_tensor(np.geomspace(0.12, 2.2, 200), dtype=DT))
    assert (k[1:] < k[:-1]).all()
    # Drude profile: unit peak at lambda_0 and FWHM = Delta
    d = O.drude_shape(torch.as_tensor(np.linspace(0.15, 0.3, 300001), dtype=DT))
    lam_um = np.linspace(0.15, 0.3, 300001)
    assert float(d.max()) == pytest.approx(1.0, abs=1e-9)
    # the 2175 A bump of the cited dust literature: centre 2175 A, width 350 A
    assert lam_um[int(d.argmax())] == pytest.approx(0.2175, abs=1e-6)
    above = lam_um[(d >= 0.5).numpy()]
    assert above[-1] - above[0] == pytest.approx(0.035, rel=0.01)


def _calzetti_join_gap():
    """k' just below minus k' at the 0.63 um join of the two fitted branches."""
    kb, kr = O.calzetti_k0(torch.tensor([0.63 - 1e-12, 0.63], dtype=DT)).tolist()
    return kb - kr


def _calzetti_colour_normalisation():
    """k'(B) - k'(V), which is 1 by the definition k' = A / E(B - V) at the
    B (4400 A) and V (5500 A) points of the fit."""
    kB, kV = O.calzetti_k0(torch.tensor([0.44, 0.55], dtype=DT)).tolist()
    return kB - kV


def test_calzetti_branches_against_their_defining_properties(monkeypatch):
    """Calzetti et al. (2000) give k'(lambda) as two fitted branches that
    meet at 0.63 um, normalised so that k'(V) = R_V = 4.05 and
    k'(B) - k'(V) = 1 (k' = A / E(B - V)).  With the published, rounded
    coefficients the red branch starts 0.025 above the blue one at the join;
    the red branch is pinned by that signed mismatch, which moves by 0.044-
    0.049 for a 1% change of either red coefficient and by 0.0055 for a 1%
    change of the common 2.659 factor on the red branch alone.  The red
    branch is linear in 1/lambda and reaches zero beyond the fitted 2.2 um."""
    assert -0.028 < _calzetti_join_gap() < -0.022
    assert _calzetti_colour_normalisation() == pytest.approx(1.0, abs=0.02)
    assert float(O.calzetti_k0(torch.tensor(0.55, dtype=DT))) == pytest.approx(4.05, abs=0.01)
    inv = np.linspace(1 / 2.2, 1 / 0.63, 7)
    k = O.calzetti_k0(torch.as_tensor(1 / inv, dtype=DT)).numpy()
    fit = np.polyfit(inv, k, 1)
    assert np.abs(np.polyval(fit, inv) - k).max() < 1e-12
    assert fit[0] / -fit[1] > 2.2                    # k' = 0 past the fitted range (in um)
    # planted mistakes in the oracle's coefficients fail the same pins
    for red in ((-1.857 * 1.01, 1.040), (-1.857 * 0.99, 1.040),
                (-1.857, 1.040 * 1.01), (-1.857, 1.040 * 0.99)):
        with monkeypatch.context() as m:
            m.setattr(O, "CALZ_RED", red)
            assert not -0.028 < _calzetti_join_gap() < -0.022
    with monkeypatch.context() as m:
        m.setattr(O, "RV_CALZ", 4.05 * 1.01)
        assert abs(float(O.calzetti_k0(torch.tensor(0.55, dtype=DT))) - 4.05) > 0.01


def _bump_fit(delta):
    """Read the UV-bump strength out of the oracle's attenuation curve as a
    black box.  Eq. DustAtt gives, at the Drude centre lambda_0 = 2175 A
    where the unit profile is 1, A(lambda_0) / (A_V / 4.05) =
    K r^delta + E_b(delta), r = lambda_0 / lambda_V and K = k_0(lambda_0)
    unknown; with E_b = e0 + e1 delta, a least-squares fit over several delta
    recovers (K, e0, e1) and the residual of the model."""
    one = torch.ones(len(delta), 1, dtype=DT)
    d = torch.as_tensor(delta, dtype=DT)[:, None]
    F = O.attenuation(torch.tensor([[2175.0]], dtype=DT), 4.05 * one, d, 0.0 * one)
    y = (-2.5 * torch.log10(F))[:, 0].numpy()
    r = 0.2175 / 0.55
    X = np.stack([r ** np.asarray(delta), np.ones(len(delta)), np.asarray(delta)], 1)
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    return coef, np.abs(X @ coef - y).max()


def _bump_pin_holds(delta):
    (K, e0, e1), res = _bump_fit(delta)
    return (res < 1e-12 and abs(e0 - 0.85) < 1e-9 and abs(e1 + 1.9) < 1e-9
            and abs(K / float(O.calzetti_k0(torch.tensor(0.2175, dtype=DT))) - 1) < 1e-9)


def test_bump_strength_follows_kriek_conroy(monkeypatch):
    """The bump the oracle's curve carries at 2175 A has the strength of
    Kriek & Conroy (2013): E_b = 0.85 at the Calzetti slope (delta = 0),
    falling by 1.9 per unit delta, and no bump once that reaches zero
    (delta > 0.447).  A sign error, a wrong intercept or the bump moved
    inside the power-law tilt fails the fit."""
    dl = np.linspace(-1.0, 0.4, 8)
    assert _bump_pin_holds(dl)
    hi = np.linspace(0.45, 1.0, 5)                  # clamp: the continuum alone
    (_, e0h, e1h), resh = _bump_fit(hi)
    assert resh < 1e-12 and abs(e0h) < 1e-9 and abs(e1h) < 1e-9
    for name, val in (("BUMP_E1", 1.9), ("BUMP_E1", -1.9 * 1.01), ("BUMP_E0", 0.85 * 1.01)):
        with monkeypatch.context() as m:
            m.setattr(O, name, val)
            assert not _bump_pin_holds(dl)
    with monkeypatch.context() as m:               # bump inside the tilt
        m.setattr(O, "bump_strength", lambda d: (0.85 - 1.9 * d).clamp(min=0)
                  * (0.2175 / 0.55) ** d)
        assert not _bump_pin_holds(dl)


# ---------------------------------------------------------------- filter integrals
def test_flat_fnu_source_gives_ab_zero_point():
    tabs = W.config(1, n_gal=1).tables
    z = torch.tensor([0.3, 1.7], dtype=DT)
    w, nb, _ = O.band_weights(tabs, z)
    sed = torch.full((2, tabs.n_lam), 7.5, dtype=DT)
    c = O.band_flux(sed, torch.ones_like(sed), w)
    m = O.magnitudes(c, nb, z)
    dl = O.lum_dist_mpc(z.numpy()) * O.MPC_CM
    ref = -2.5 * torch.log10((1 + z) * O.L_SUN_ERG_S * 7.5 / (4 * math.pi * dl ** 2 * O.AB_ZP_CGS))
    torch.testing.assert_close(m, ref[:, None].expand_as(m), rtol=0, atol=1e-12)


def _analytic_tables(n_lam=6000):
    """Two ages x two metallicities, every SSP the same analytic spectrum
    L(lam) = 1e-16 (0.05 + exp(-(ln lam - ln 5000)^2 / (2 0.3^2)))."""
    lam = np.geomspace(91.0, 25000.0, n_lam)
    spec = 1e-16 * (0.05 + np.exp(-0.5 * ((np.log(lam) - math.log(5000.0)) / 0.3) ** 2))
    ssp = np.broadcast_to(spec, (2, 2, n_lam)).copy()
    kind = np.array([1, 1, 0], np.int32)
    p0 = np.array([4500.0, 8000.0, 6000.0])
    p1 = np.array([4500.0 / 4, 8000.0 / 12, 9000.0])
    tabs = W.Tables(np.array([1e7, 5e9]), np.array([-1.0, 0.0]), lam, ssp, kind, p0, p1)
    f = lambda l: 1e-16 * (0.05 + math.exp(-0.5 * ((math.log(l) - math.log(5000.0)) / 0.3) ** 2))
    return tabs, f


def test_single_population_magnitudes_equal_filter_integrated_ssp():
    """All SSPs identical => the composite SED is M_star L(lambda), so with
    A_V = 0 every magnitude equals the directly filter-integrated SSP shifted
    by the mass (the single-age single-Z check)."""
    tabs, f = _analytic_tables()
    th = _theta(3, seed=5)
    th[:, 9] = 0.0
    z = torch.tensor([0.2, 1.0, 2.4], dtype=DT)
    m = O.photometry(th, z, tabs, "exact")
    _, ms, _, _ = O.ssp_weights(th, tabs, O.t_obs_gyr(z))
    dl = O.lum_dist_mpc(z.numpy()) * O.MPC_CM
    for r in range(3):
        zr = float(z[r])
        for b in range(3):
            if tabs.band_kind[b] == 1:
                s = tabs.band_p1[b] / (2 * math.sqrt(2 * math.log(2)))
                T = lambda l: math.exp(-0.5 * (((1 + zr) * l - tabs.band_p0[b]) / s) ** 2)
                lo, hi = (tabs.band_p0[b] - 9 * s) / (1 + zr), (tabs.band_p0[b] + 9 * s) / (1 + zr)
            else:
                T = lambda l: 1.0
                lo, hi = tabs.band_p0[b] / (1 + zr), tabs.band_p1[b] / (1 + zr)
            num, _ = integrate.quad(lambda l: f(l) * T(l) / l, lo, hi, epsrel=1e-12, limit=400)
            den, _ = integrate.quad(lambda l: T(l) / l, lo, hi, epsrel=1e-12, limit=400)
            fac = (1 + zr) * O.L_SUN_ERG_S / (4 * math.pi * float(dl[r]) ** 2 * O.AB_ZP_CGS)
            ref = -2.5 * math.log10(fac * float(ms[r]) * num / den)
            # trapezoid on the grid: O(h^2) for smooth bands, O(h) at top-hat edges
            tol = 2e-6 if tabs.band_kind[b] == 1 else 2e-3
            assert float(m[r, b]) == pytest.approx(ref, abs=tol)


def test_redshift_moves_band_to_bluer_rest_wavelength():
    tabs, _ = _analytic_tables()
    tabs.band_kind = np.array([1], np.int32)
    tabs.band_p0 = np.array([8000.0])
    tabs.band_p1 = np.array([80.0])          # R = 100
    z = torch.tensor([0.0, 0.6, 2.0], dtype=DT)
    le = O.lambda_eff(tabs, z)[:, 0]
    torch.testing.assert_close(le, 8000.0 / (1 + z), rtol=1e-4, atol=0)


def _lambda_eff_photon_weighted(tables, z):
    """A plausible misreading of Eq. lambda_eff, kept here only to show that
    the pin below tells it apart: the photon-counting 1/lambda weight of the
    band integrals carried into the effective wavelength."""
    lam = torch.as_tensor(tables.lam_ang, dtype=DT)
    q = O.trapezoid_weights(tables.lam_ang)
    T = O.transmission(tables, (1.0 + z)[:, None] * lam[None, :])
    return (T * q[None, None, :]).sum(-1) / (T * (q / lam)[None, None, :]).sum(-1)


def _lambda_eff_pin(tabs, z):
    """Largest relative deviation of the oracle's lambda_eff from c / (1+z)
    (Gaussian band, centre c) and (lo + hi) / 2 / (1+z) (top-hat)."""
    ref = torch.stack([3600.0 / (1 + z), 6500.0 / (1 + z)], dim=1)
    rel = ((O.lambda_eff(tabs, z) - ref) / ref).abs()
    return float(rel[:, 0].max()), float(rel[:, 1].max()), float(rel.min())


def test_lambda_eff_is_the_unweighted_band_mean_at_low_resolution(monkeypatch):
    """Eq. lambda_eff weighs wavelength by the transmission alone.  For a
    Gaussian band of observed centre c, substituting lambda_obs = (1+z)
    lambda makes the ratio of integrals exactly c / (1+z) at any width; for
    a top-hat [lo, hi] it is (lo + hi) / 2 / (1+z).  At the paper's lowest
    resolution R = 3.4 (App. B) the photon-weighted variant lies 1.6% below
    (Gaussian) and 1.8% (top-hat), so planting it in the oracle fails."""
    lam = np.geomspace(91.0, 25000.0, 20000)
    tabs = W.Tables(np.array([1e7, 5e9]), np.array([-1.0, 0.0]), lam,
                    np.ones((2, 2, lam.size)), np.array([1, 0], np.int32),
                    np.array([3600.0, 5000.0]), np.array([3600.0 / 3.4, 8000.0]))
    z = torch.tensor([0.0, 0.7, 2.1], dtype=DT)
    gauss_err, hat_err, _ = _lambda_eff_pin(tabs, z)
    assert gauss_err < 1e-6        # trapezoid on a smooth band: O(h^2)
    assert hat_err < 1e-3          # discontinuous edges: O(h / width)
    with monkeypatch.context() as m:
        m.setattr(O, "lambda_eff", _lambda_eff_photon_weighted)
        assert _lambda_eff_pin(tabs, z)[2] > 0.01


# ---------------------------------------------------------------- approximation (Sec. 3)
def test_approx_equals_exact_without_dust():
    wl = W.config(0, n_gal=6)
    wl.tables.band_kind[:] = 1
    wl.tables.band_p0[:] = np.linspace(3600, 9700, 6)
    wl.tables.band_p1[:] = wl.tables.band_p0 / 5.0
    th = torch.as_tensor(wl.theta, dtype=DT)
    for col, val in ((9, 0.0), (11, 1.0)):
        t2 = th.clone()
        t2[:, col] = val
        me = O.photometry(t2, wl.z, wl.tables, "exact")
        ma = O.photometry(t2, wl.z, wl.tables, "approx")
        torch.testing.assert_close(ma, me, rtol=0, atol=1e-11)


def test_approx_converges_to_exact_as_bands_narrow():
    wl = W.config(1, n_gal=8)
    th = torch.as_tensor(wl.theta, dtype=DT)
    th[:, 9] = 1.5
    th[:, 11] = 0.0
    errs = []
    for R in (4.0, 16.0, 64.0):
        wl.tables.band_p1[:] = wl.tables.band_p0 / R
        d = O.photometry(th, wl.z, wl.tables, "approx") - O.photometry(th, wl.z, wl.tables, "exact")
        errs.append(float(d.abs().max()))
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 8.0          # second order in the band width


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("mode", ["exact", "approx"])
def test_gradient_against_central_differences(mode):
    wl = W.config(0 if mode == "exact" else 1, n_gal=3)
    th = torch.as_tensor(wl.theta, dtype=DT)
    mobs = O.photometry(torch.as_tensor(wl.theta_true, dtype=DT), wl.z, wl.tables, mode) + 0.3
    ll, g, _ = O.loglike_and_grad(th, wl.z, wl.tables, mobs, wl.sigma, wl.mask, mode)
    h = 1e-5
    fd = torch.zeros_like(g)
    for k in range(12):
        e = torch.zeros_like(th)
        e[:, k] = h * (W.PRIOR_HI[k] - W.PRIOR_LO[k])
        lp = O.loglike(O.photometry(th + e, wl.z, wl.tables, mode), mobs, wl.sigma, wl.mask)
        lm = O.loglike(O.photometry(th - e, wl.z, wl.tables, mode), mobs, wl.sigma, wl.mask)
        fd[:, k] = (lp - lm) / (2 * e[:, k])
    scale = g.abs().max(1, keepdim=True).values
    assert ((fd - g).abs() / scale).max() < 1e-6
