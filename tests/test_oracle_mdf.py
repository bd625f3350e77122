"""Pins of the oracle's non-separable metallicity distribution (MDF mean
shifted per age bin) (CPU only)."""
import numpy as np
import torch
from scipy import integrate, stats

import sps_workloads as W
from oracle import sps as O

DT = torch.float64


def _theta(n, seed):
    return torch.as_tensor(W.prior_draw(np.random.default_rng(seed), n))


def test_zero_offsets_are_the_separable_model():
    wl = W.config(0, n_gal=4)
    th = torch.as_tensor(wl.theta_true)
    t_obs = O.t_obs_gyr(torch.as_tensor(wl.z))
    W0, M0, _, _ = O.ssp_weights(th, wl.tables, t_obs)
    W1, M1, _, q = O.ssp_weights(th, W.with_mdf_offset(wl.tables, np.zeros(wl.tables.n_age)), t_obs)
    torch.testing.assert_close(W1, W0, rtol=1e-15, atol=0)
    assert q.shape == (4, wl.tables.n_age, wl.tables.n_met)


def test_constant_offset_shifts_the_mean():
    wl = W.config(0, n_gal=4)
    th = torch.as_tensor(wl.theta_true)
    t_obs = O.t_obs_gyr(torch.as_tensor(wl.z))
    d = 0.13
    W1, _, _, _ = O.ssp_weights(th, W.with_mdf_offset(wl.tables, np.full(wl.tables.n_age, d)), t_obs)
    th2 = th.clone()
    th2[:, 7] += d
    W2, _, _, _ = O.ssp_weights(th2, wl.tables, t_obs)
    torch.testing.assert_close(W1, W2, rtol=1e-13, atol=0)


def test_rows_are_normalised_and_match_brute_force():
    """Each age row of P_met sums to one and equals the Gaussian mass between
    the metallicity-bin edges (quadrature), mean lgZ + offset_i."""
    lgZ = np.array([-2.0, -1.5, -1.0, -0.5, 0.0, 0.2])
    off = np.array([-0.6, -0.2, 0.0, 0.35])
    th = _theta(3, 5)
    q = O.met_weights(th, lgZ, off).numpy()                          # [3, 4, 6]
    np.testing.assert_allclose(q.sum(-1), 1.0, rtol=0, atol=1e-14)
    edges = np.concatenate([[-np.inf], 0.5 * (lgZ[1:] + lgZ[:-1]), [np.inf]])
    for r in range(3):
        mu0, sd = float(th[r, 7]), float(th[r, 8])
        for i, o in enumerate(off):
            pdf = stats.norm(mu0 + o, sd).pdf
            for j in range(6):
                ref, _ = integrate.quad(pdf, edges[j], edges[j + 1], epsabs=1e-13)
                assert abs(q[r, i, j] - ref) < 1e-10


def test_ssp_weights_sum_to_mstar_with_offsets():
    wl = W.config(0, n_gal=5)
    tabs = W.with_mdf_offset(wl.tables, W.mzr_offsets(wl.tables.age_yr))
    th = torch.as_tensor(wl.theta_true)
    Wt, M, _, _ = O.ssp_weights(th, tabs, O.t_obs_gyr(torch.as_tensor(wl.z)))
    torch.testing.assert_close(Wt.sum((1, 2)), M, rtol=1e-12, atol=0)
