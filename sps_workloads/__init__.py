"""Seeded synthetic inputs for the SPS photometry / likelihood / HMC workloads.

This module is the only code shared by the FP64 oracle (``oracle/``) and the
CUDA path (``paper_2506_19919_gb300``).  It holds no arithmetic of the method
itself: it draws grids, a synthetic SSP spectral table, filter descriptions,
parameter vectors, redshifts, band masks and noise.  Everything the method
computes from these (SFH weights, dust, redshifted filter weights, magnitudes,
likelihoods, gradients, HMC) lives on either side of the boundary, never here.

The paper's inputs are MIST SSP spectra, a simulated 20,000-galaxy sample and
Gaussian (and LSST) transmission curves (Sec. 2, App. B, App. D.1).  None of
them is available here, so these seeded stand-ins take their shapes:

* SSP table L[age, Z, lambda]: positive, smooth spectra, each a floor plus a
  sum of 8 Gaussians in ln(lambda), with an amplitude that falls with age and
  an extra fall-off of the blue (< 4000 A) components with age, so that young
  populations are blue.  Units: L_sun / Hz per solar mass formed.
* Age grid log-spaced 1e6 .. 1.4e10 yr; metallicity grid linear in
  log10(Z/Z_sun) over [-2, 0.2]; wavelength grid log-spaced (rest frame, A).
* Bands: top-hat (edges in observed-frame A) or Gaussian (centre, FWHM in
  observed-frame A) with resolution R = centre / FWHM spread geometrically
  from 3.4 to 25.5 as in App. B.
* Parameters drawn uniformly in the inner 98% of each prior range (App. C
  gives the bounded-parameter construction but prints no ranges; the ranges
  below are this package's declared convention).

All floating-point values handed to either side are rounded to float32 first
(``theta``, ``z``, ``sigma``, noise), so that the oracle and the float32 CUDA
path see bit-identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2506199190

# Column order of the 12 physical parameters (Sec. 2, App. A.1-A.3).
PARAM_NAMES = (
    "lgM",       # log10 of the SFR amplitude M_formed [M_sun / yr]
    "tau",       # turnover time of the double power law [Gyr]
    "alpha",     # falling slope
    "beta",      # rising slope
    "F_burst",   # burst mass fraction
    "lgT_peak",  # log10 burst peak age [yr]
    "dlgT",      # log10 T_max - log10 T_peak [dex]
    "lgZ",       # mean of the Gaussian in log10(Z / Z_sun)
    "sigma_lgZ", # width of that Gaussian [dex]
    "A_V",       # V-band attenuation normalisation [mag]
    "delta",     # power-law tilt of the attenuation curve
    "F_floor",   # unobscured fraction of sight lines
)
N_PARAM = len(PARAM_NAMES)

# Prior bounds [lo, hi] of each physical parameter (declared convention).
PRIOR_LO = np.array([-1.5, 0.5, 0.1, 0.1, 0.0, 6.0, 0.05, -2.0, 0.05, 0.0, -1.0, 0.0])
PRIOR_HI = np.array([2.5, 12.0, 5.0, 5.0, 0.2, 8.5, 1.5, 0.2, 0.5, 3.0, 0.4, 0.5])

BAND_TOPHAT = 0
BAND_GAUSS = 1
BAND_TABLE = 2


@dataclass
class Tables:
    """Model grids, the SSP table and the filter set (host, float64)."""
    age_yr: np.ndarray        # [A] increasing
    lgZ: np.ndarray           # [Zn] increasing, log10(Z/Z_sun)
    lam_ang: np.ndarray       # [Lam] rest-frame wavelength, increasing
    ssp: np.ndarray           # [A, Zn, Lam] L_sun/Hz per M_sun formed
    band_kind: np.ndarray     # [B] int32: BAND_TOPHAT, BAND_GAUSS or BAND_TABLE
    band_p0: np.ndarray       # [B] top-hat lower edge, Gaussian centre or table start (A, observed)
    band_p1: np.ndarray       # [B] top-hat upper edge, Gaussian FWHM or table step (A, observed)
    band_tab_n: np.ndarray = None   # [B] int32 samples per tabulated band (0 otherwise)
    band_tab_T: np.ndarray = None   # [sum n] the tabulated bands' samples, band after band
    mdf_offset: np.ndarray = None   # [A] age-dependent shift of the MDF mean (None: separable)

    @property
    def n_age(self) -> int:
        return self.age_yr.shape[0]

    @property
    def n_met(self) -> int:
        return self.lgZ.shape[0]

    @property
    def n_lam(self) -> int:
        return self.lam_ang.shape[0]

    @property
    def n_band(self) -> int:
        return self.band_kind.shape[0]


@dataclass
class Workload:
    name: str
    tables: Tables
    z: np.ndarray             # [G] float32-representable
    theta: np.ndarray         # [G*C, 12] physical parameters (evaluation point)
    theta_true: np.ndarray    # [G, 12] parameters that generated the data
    mask: np.ndarray          # [G] uint32 bit b set <=> band b observed
    sigma: np.ndarray         # [G, B] photometric noise (mag)
    noise: np.ndarray         # [G, B] N(0, sigma) draws to add to model mags
    chains: int = 1
    extra: dict = field(default_factory=dict)

    @property
    def n_gal(self) -> int:
        return self.z.shape[0]


def tabulated_bands(rng: np.random.Generator, edges_nm, step_ang: float = 10.0):
    """Synthetic broad-band throughput curves sampled every step_ang (A) on
    the observed frame, one band per [lo, hi) pair of edges_nm: a smooth
    flat-topped profile (product of two logistic edges of width ~2% of the
    band centre) with a seeded ripple of a few per cent and a peak between
    0.5 and 0.9.  Returns (kind, start, step, n, T) in the Tables layout.
    (Input synthesis only.)"""
    kind, p0, p1, ns, Ts = [], [], [], [], []
    for lo_nm, hi_nm in zip(edges_nm[:-1], edges_nm[1:]):
        lo, hi = 10.0 * lo_nm, 10.0 * hi_nm
        w = 0.02 * 0.5 * (lo + hi)
        start = step_ang * np.floor((lo - 8 * w) / step_ang)
        n = int(np.ceil((hi + 8 * w - start) / step_ang)) + 1
        lam = start + step_ang * np.arange(n)
        prof = 1.0 / (1.0 + np.exp(-(lam - lo) / w)) / (1.0 + np.exp((lam - hi) / w))
        ph, amp, per = rng.uniform(0, 2 * np.pi), rng.uniform(0.01, 0.04), rng.uniform(200.0, 600.0)
        T = rng.uniform(0.5, 0.9) * prof * (1.0 + amp * np.sin(2 * np.pi * lam / per + ph))
        T[0] = T[-1] = 0.0
        kind.append(BAND_TABLE)
        p0.append(start)
        p1.append(step_ang)
        ns.append(n)
        Ts.append(T)
    return (np.array(kind, np.int32), np.array(p0), np.array(p1), np.array(ns, np.int32),
            np.concatenate(Ts))


def with_bands(tables: Tables, kind, p0, p1, tab_n=None, tab_T=None) -> Tables:
    """The same SSP grid with another filter set."""
    return Tables(tables.age_yr, tables.lgZ, tables.lam_ang, tables.ssp, np.asarray(kind, np.int32),
                  np.asarray(p0, np.float64), np.asarray(p1, np.float64),
                  None if tab_n is None else np.asarray(tab_n, np.int32),
                  None if tab_T is None else np.asarray(tab_T, np.float64), tables.mdf_offset)


def mzr_offsets(age_yr, slope: float = 0.25, t_ref_gyr: float = 1.0) -> np.ndarray:
    """An age-dependent shift of the MDF mean of the kind an evolving
    mass-metallicity relation produces: older stars formed earlier from less
    enriched gas, dlgZ_i = -slope * log10(1 + age_i / t_ref) (input synthesis
    only; any [A] vector may be supplied)."""
    return -slope * np.log10(1.0 + np.asarray(age_yr, dtype=np.float64) / (t_ref_gyr * 1e9))


def with_mdf_offset(tables: Tables, offset) -> Tables:
    """The same tables with an age-dependent MDF mean (non-separable W)."""
    return Tables(tables.age_yr, tables.lgZ, tables.lam_ang, tables.ssp, tables.band_kind, tables.band_p0,
                  tables.band_p1, tables.band_tab_n, tables.band_tab_T,
                  None if offset is None else np.asarray(offset, np.float64))


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def ssp_table(rng: np.random.Generator, age_yr, lgZ, lam_ang, n_comp: int = 8) -> np.ndarray:
    """Synthetic positive smooth SSP spectra (input synthesis only)."""
    lnlam = np.log(lam_ang)
    mu = rng.uniform(lnlam[0], lnlam[-1], size=n_comp)
    s = rng.uniform(0.05, 0.5, size=n_comp)
    zn = len(lgZ)
    amp = rng.uniform(0.2, 1.0, size=(n_comp, zn)) * (1.0 + 0.1 * np.arange(zn))[None, :]
    shapes = np.exp(-0.5 * ((lnlam[None, :] - mu[:, None]) / s[:, None]) ** 2)  # [g, Lam]
    age_gyr = np.asarray(age_yr) / 1e9
    a_i = 1e-15 * age_gyr ** -0.7                                               # [A]
    blue = mu < np.log(4000.0)
    extra = np.where(blue[None, :], age_gyr[:, None] ** -0.5, 1.0)              # [A, g]
    # L[i, j, n] = a_i * (0.02 + sum_g amp[g, j] * extra[i, g] * shape[g, n])
    comp = np.einsum("gj,ig,gn->ijn", amp, extra, shapes)
    return a_i[:, None, None] * (0.02 + comp)


def _gauss_bands(centres, r_lo=3.4, r_hi=25.5):
    centres = np.asarray(centres, dtype=np.float64)
    res = np.geomspace(r_lo, r_hi, len(centres))
    return (np.full(len(centres), BAND_GAUSS, np.int32), centres, centres / res)


def _tophat_bands(edges_nm):
    e = np.asarray(edges_nm, dtype=np.float64) * 10.0
    return (np.full(len(e) - 1, BAND_TOPHAT, np.int32), e[:-1].copy(), e[1:].copy())


def make_tables(rng, n_age, n_met, n_lam, lam_lo, lam_hi, bands) -> Tables:
    age = np.logspace(6.0, np.log10(1.4e10), n_age)
    lgz = np.linspace(-2.0, 0.2, n_met)
    lam = np.geomspace(lam_lo, lam_hi, n_lam)
    ssp = ssp_table(rng, age, lgz, lam)
    kind, p0, p1 = bands
    return Tables(age, lgz, lam, ssp, kind, p0, p1)


def prior_draw(rng, n: int, inner: float = 0.98) -> np.ndarray:
    """Physical parameters uniform in the inner `inner` fraction of each range."""
    lo, hi = PRIOR_LO, PRIOR_HI
    pad = 0.5 * (1.0 - inner) * (hi - lo)
    u = rng.uniform(size=(n, N_PARAM))
    return _f32(lo + pad + u * (hi - lo - 2 * pad))


def unbounded_of(theta: np.ndarray) -> np.ndarray:
    """Inverse of the logistic bounding map with k = 1, x0 = 0, for drawing
    HMC start points in unbounded space (input synthesis)."""
    s = (theta - PRIOR_LO) / (PRIOR_HI - PRIOR_LO)
    return _f32(np.log(s) - np.log1p(-s))


def _masks(rng, n_gal, n_band, n_min, n_max):
    k = rng.integers(n_min, n_max + 1, size=n_gal)
    order = np.argsort(rng.uniform(size=(n_gal, n_band)), axis=1)   # random subset order
    rank = np.empty_like(order)
    np.put_along_axis(rank, order, np.arange(n_band)[None, :].repeat(n_gal, 0), axis=1)
    bits = (rank < k[:, None]).astype(np.uint64) << np.arange(n_band, dtype=np.uint64)[None, :]
    return bits.sum(axis=1).astype(np.uint32)


CONFIG_NAMES = (
    "parity_exact_64gal_tophat6",
    "photometry_100kgal_gauss6",
    "loglike_grad_100kpairs_gauss6",
    "hmc_4096gal_x4chains_gauss12",
    "survey_1Mgal_x2chains_gauss20_burst",
)


def config(idx: int, n_gal: int | None = None, seed_offset: int = 0) -> Workload:
    """The five seeded workloads; `n_gal` shrinks the galaxy count (tables,
    bands and distributions unchanged)."""
    rng = np.random.default_rng(SEED_BASE + idx + 1000 * seed_offset)
    if idx == 0:
        tabs = make_tables(rng, 50, 6, 2000, 1000.0, 12000.0,
                           _tophat_bands([320, 400, 550, 700, 820, 920, 1060]))
        G = 64 if n_gal is None else n_gal
        zlo, zhi, chains = 0.05, 1.0, 1
    elif idx in (1, 2):
        tabs = make_tables(rng, 107, 12, 5994, 91.0, 25000.0,
                           _gauss_bands(np.linspace(3600.0, 9700.0, 6)))
        G = 100_000 if n_gal is None else n_gal
        zlo, zhi, chains = 0.05, 3.0, 1
    elif idx == 3:
        tabs = make_tables(rng, 107, 12, 5994, 91.0, 25000.0,
                           _gauss_bands(np.geomspace(3000.0, 24000.0, 12)))
        G = 4096 if n_gal is None else n_gal
        zlo, zhi, chains = 0.05, 3.0, 4
    elif idx == 4:
        tabs = make_tables(rng, 107, 12, 5994, 91.0, 25000.0,
                           _gauss_bands(np.geomspace(3000.0, 24000.0, 20)))
        G = 1_000_000 if n_gal is None else n_gal
        zlo, zhi, chains = 0.05, 3.0, 2
    else:
        raise ValueError(f"no workload {idx}")
    B = tabs.n_band
    z = _f32(rng.uniform(zlo, zhi, size=G))
    theta_true = prior_draw(rng, G)
    if idx == 2:
        theta = prior_draw(rng, G)            # independent evaluation point
    else:
        theta = np.repeat(theta_true, chains, axis=0)
    if idx == 3:
        mask = _masks(rng, G, B, 3, 12)
    elif idx == 4:
        mask = _masks(rng, G, B, 6, 20)
    else:
        mask = np.full(G, np.uint32((1 << B) - 1), dtype=np.uint32)
    sigma = _f32(np.full((G, B), 0.05))
    noise = _f32(rng.normal(0.0, 0.05, size=(G, B)))
    wl = Workload(CONFIG_NAMES[idx], tabs, z, theta, theta_true, mask, sigma, noise, chains)
    if idx in (3, 4):
        wl.extra["theta0_unb"] = unbounded_of(prior_draw(rng, G * chains))
        wl.extra["n_warm"] = 500 if idx == 3 else 300
        wl.extra["n_samp"] = 500 if idx == 3 else 300
        wl.extra["L_min"], wl.extra["L_max"] = 8, 64
    return wl


def tiny_tables(rng=None, n_age=5, n_met=3, n_lam=400, lam_lo=1000.0, lam_hi=12000.0,
                bands=None) -> Tables:
    """Small grids for brute-force checks."""
    rng = np.random.default_rng(SEED_BASE + 99) if rng is None else rng
    bands = _tophat_bands([320, 450, 600, 800]) if bands is None else bands
    return make_tables(rng, n_age, n_met, n_lam, lam_lo, lam_hi, bands)


__all__ = [
    "SEED_BASE", "PARAM_NAMES", "N_PARAM", "PRIOR_LO", "PRIOR_HI", "BAND_TOPHAT",
    "BAND_GAUSS", "BAND_TABLE", "tabulated_bands", "with_bands", "mzr_offsets", "with_mdf_offset", "Tables", "Workload", "config", "prior_draw", "unbounded_of",
    "tiny_tables", "make_tables", "ssp_table", "CONFIG_NAMES",
]
