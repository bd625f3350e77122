"""User-supplied SSP grid and measured filter curves (the paper's MIST SSPs and
LSST throughputs are not in this repository).  With

    SPS_SSP_FILE=/path/ssp.npz                     (DSPS-style keys, see loaders.load_ssp)
    SPS_FILTER_FILES=/path/u.dat,/path/g.dat,...   (two columns: wavelength, throughput)
    SPS_FILTER_UNIT=nm                             (or angstrom / um; default nm)

it reads those files; without them it writes synthetic stand-ins in the same
formats first (a 107-age x 12-metallicity x 5994-wavelength grid and six
flat-topped curves with a ripple at LSST-like edges, one sampled unevenly) and
reads them back through the same loaders.

It checks the GPU against the FP64 oracle on those tables (exact FP32 and BF16,
approximate, log L + gradient) and reports the approximate path's error
against the exact one over a redshift range, the paper's accuracy check
(App. B quotes differences up to ~0.06 mag for its bands)."""
import os

import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O

pytestmark = pytest.mark.gpu


def _write_stand_in_files(d):
    """Synthetic files in the loaders' formats: the SSP grid as a DSPS-style
    .npz ([n_met, n_age, n_wave] flux, log ages in Gyr) and one two-column
    text file per filter (wavelength in nm, throughput)."""
    rng = np.random.default_rng(W.SEED_BASE + 77)
    tabs = W.make_tables(rng, 107, 12, 5994, 91.0, 25000.0, W._gauss_bands([5000.0]))
    ssp = os.path.join(d, "ssp.npz")
    np.savez(ssp, ssp_lgmet=tabs.lgZ, ssp_lg_age_gyr=np.log10(tabs.age_yr / 1e9),
             ssp_wave=tabs.lam_ang, ssp_flux=tabs.ssp.transpose(1, 0, 2))
    _, start, step, n, T = W.tabulated_bands(rng, [320, 400, 552, 691, 818, 922, 1060])
    files, off = [], 0
    for b in range(len(n)):
        lam_nm = (start[b] + step[b] * np.arange(n[b])) / 10.0
        Tb = T[off:off + n[b]]
        off += n[b]
        if b == 2:                       # an unevenly sampled file: drop some interior samples
            keep = np.ones(n[b], bool)
            keep[1:-1] = rng.uniform(size=n[b] - 2) > 0.3
            keep[1::7] = True            # keep the smallest spacing at one step
            lam_nm, Tb = lam_nm[keep], Tb[keep]
        f = os.path.join(d, f"band{b}.dat")
        np.savetxt(f, np.stack([lam_nm, Tb], 1), header="wavelength_nm throughput")
        files.append(f)
    return ssp, files, "nm"


@pytest.fixture(scope="module")
def user(tmp_path_factory):
    import paper_2506_19919_gb300 as pkg
    from paper_2506_19919_gb300 import loaders as Ld
    if os.environ.get("SPS_SSP_FILE") and os.environ.get("SPS_FILTER_FILES"):
        ssp, files, unit = (os.environ["SPS_SSP_FILE"], os.environ["SPS_FILTER_FILES"].split(","),
                            os.environ.get("SPS_FILTER_UNIT", "nm"))
    else:
        ssp, files, unit = _write_stand_in_files(str(tmp_path_factory.mktemp("user_tables")))
    curves = [Ld.load_filter_curve(f, unit=unit) for f in files]
    tabs = Ld.tables(ssp, curves)
    rng = np.random.default_rng(2506199190)
    n = 64
    theta = W.prior_draw(rng, n)
    z = np.round(rng.uniform(0.05, 3.0, n), 4).astype(np.float32).astype(np.float64)
    ctx = pkg.Context(tabs, device=0)
    ctx.set_galaxies(z, build_approx=True)
    yield tabs, theta, z, ctx
    ctx.close()


@pytest.mark.parametrize("mode,prec,tol", [("exact", "fp32", 1e-3), ("exact", "bf16", 5e-3),
                                           ("approx", "fp32", 1e-3)])
def test_user_tables_photometry_parity(user, mode, prec, tol):
    tabs, theta, z, ctx = user
    m = ctx.photometry(theta, mode=mode, prec=prec).cpu().numpy()
    ref = O.photometry(theta, z, tabs, mode).numpy()
    assert np.abs(m - ref).max() < tol


def test_user_tables_loglike_grad_parity(user):
    tabs, theta, z, ctx = user
    th_true = torch.as_tensor(theta, dtype=torch.float64)
    mobs = O.photometry(th_true, z, tabs, "approx").numpy() + 0.05
    sigma = np.full_like(mobs, 0.05)
    mask = np.full(len(z), (1 << tabs.n_band) - 1, np.uint32)
    ev = W.prior_draw(np.random.default_rng(7), len(z))
    ll, g = ctx.loglike_grad(ev, mobs, sigma, mask, mode="approx")
    llr, gr, _ = O.loglike_and_grad(ev, z, tabs, mobs, sigma, mask, "approx")
    np.testing.assert_allclose(ll.cpu().numpy(), llr.numpy(), rtol=2e-4)
    g, gr = g.cpu().numpy().astype(np.float64), gr.numpy()
    assert (np.abs(g - gr).max(1) / np.abs(gr).max(1)).max() < 1e-4


def test_user_tables_approximation_error(user):
    """The effective-wavelength approximation against the exact integral on
    the user's curves (both FP64 in the oracle, and on the GPU): reported, and
    held to the paper's order of magnitude."""
    tabs, theta, z, ctx = user
    d_gpu = (ctx.photometry(theta, mode="approx").cpu().numpy()
             - ctx.photometry(theta, mode="exact").cpu().numpy())
    d_ref = (O.photometry(theta, z, tabs, "approx") - O.photometry(theta, z, tabs, "exact")).numpy()
    print(f"approx - exact: max |d| {np.abs(d_ref).max():.4f} mag, median {np.median(np.abs(d_ref)):.4f} mag")
    assert np.abs(d_gpu - d_ref).max() < 2e-3
    assert np.abs(d_ref).max() < 0.3
