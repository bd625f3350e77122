"""Loaders for user-supplied SSP tables and filter throughput curves (host).

The paper fits MIST SSPs through LSST's measured throughput curves (Sec. 2,
Sec. 5).  These helpers read such files into the arrays sps_create takes:

* ``load_filter_curve``: a two-column text file (wavelength, throughput;
  ``#`` comments), wavelengths in nm or Angstrom, resampled onto a uniform
  observed-frame grid (the library's tabulated-band convention: the
  transmission is the linear interpolant of uniform samples).  The step
  defaults to the smallest spacing of the file, so a curve already sampled
  uniformly is kept as it is.
* ``filter_set``: any mix of tabulated curves, Gaussian and top-hat bands,
  in the band order of the fit.
* ``load_ssp``: an ``.npz`` (or, when h5py is installed, ``.h5``) file with
  the SSP grid under the DSPS-style names ``ssp_lgmet`` (log10 Z/Z_sun),
  ``ssp_lg_age_gyr`` (log10 age / Gyr), ``ssp_wave`` (Angstrom) and
  ``ssp_flux`` [n_met, n_age, n_wave] in L_sun / Hz per solar mass.

Plain NumPy, run once per analysis; not on the computational path.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np

BAND_TOPHAT, BAND_GAUSS, BAND_TABLE = 0, 1, 2


@dataclass
class SpsTables:
    """Everything sps_create needs (Context(tables=...) reads these names)."""
    age_yr: np.ndarray        # [A]
    lgZ: np.ndarray           # [Zn]
    lam_ang: np.ndarray       # [Lam] rest frame
    ssp: np.ndarray           # [A, Zn, Lam]
    band_kind: np.ndarray     # [B] int32
    band_p0: np.ndarray       # [B]
    band_p1: np.ndarray       # [B]
    band_tab_n: np.ndarray    # [B] int32
    band_tab_T: np.ndarray    # [sum n]

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
class Curve:
    """A tabulated throughput: T[m] at start + m * step (Angstrom, observed)."""
    start: float
    step: float
    T: np.ndarray


def resample_curve(lam_ang, T, step_ang=None) -> Curve:
    """Linear interpolant of (lam_ang, T) on a uniform grid from the first to
    the last sample (step: the smallest spacing unless given); negative
    throughputs are clipped to zero."""
    lam = np.asarray(lam_ang, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    if lam.ndim != 1 or lam.shape != T.shape or lam.size < 2:
        raise ValueError("need matching 1-D wavelength and throughput arrays with >= 2 samples")
    order = np.argsort(lam, kind="stable")
    lam, T = lam[order], T[order]
    if np.any(np.diff(lam) <= 0) or not np.all(np.isfinite(T)) or lam[0] <= 0:
        raise ValueError("wavelengths must be positive and distinct, throughputs finite")
    step = float(np.min(np.diff(lam))) if step_ang is None else float(step_ang)
    if not step > 0:
        raise ValueError("step must be positive")
    n = int(np.floor((lam[-1] - lam[0]) / step + 1e-9)) + 1
    grid = lam[0] + step * np.arange(max(n, 2))
    return Curve(float(lam[0]), step, np.clip(np.interp(grid, lam, T, left=0.0, right=0.0), 0.0, None))


def load_filter_curve(path, unit="nm", step_ang=None) -> Curve:
    """Two-column text file (wavelength, throughput) -> uniform Curve."""
    data = np.loadtxt(path, comments="#", usecols=(0, 1), ndmin=2)
    scale = {"nm": 10.0, "angstrom": 1.0, "A": 1.0, "um": 1e4}[unit]
    return resample_curve(data[:, 0] * scale, data[:, 1], step_ang)


def filter_set(bands):
    """bands: sequence of Curve, ("gauss", centre_A, fwhm_A) or
    ("tophat", lo_A, hi_A).  Returns (kind, p0, p1, tab_n, tab_T)."""
    kind, p0, p1, tn, tT = [], [], [], [], []
    for b in bands:
        if isinstance(b, Curve):
            kind.append(BAND_TABLE)
            p0.append(b.start)
            p1.append(b.step)
            tn.append(len(b.T))
            tT.append(np.asarray(b.T, dtype=np.float64))
        else:
            name, a, c = b
            kind.append({"tophat": BAND_TOPHAT, "gauss": BAND_GAUSS}[name])
            p0.append(float(a))
            p1.append(float(c))
            tn.append(0)
    return (np.array(kind, np.int32), np.array(p0), np.array(p1), np.array(tn, np.int32),
            np.concatenate(tT) if tT else np.zeros(0))


def load_ssp(path):
    """SSP grid -> (age_yr [A], lgZ [Zn], lam_ang [Lam], ssp [A, Zn, Lam])."""
    ext = os.path.splitext(str(path))[1].lower()
    if ext in (".h5", ".hdf5"):
        try:
            import h5py
        except ImportError as e:                    # pragma: no cover - depends on the image
            raise ImportError("reading .h5 SSP files needs h5py; convert to .npz") from e
        with h5py.File(path, "r") as f:
            d = {k: np.asarray(f[k]) for k in ("ssp_lgmet", "ssp_lg_age_gyr", "ssp_wave", "ssp_flux")}
    else:
        with np.load(path) as f:
            d = {k: np.asarray(f[k]) for k in ("ssp_lgmet", "ssp_lg_age_gyr", "ssp_wave", "ssp_flux")}
    lgZ = d["ssp_lgmet"].astype(np.float64)
    age_yr = 10.0 ** (d["ssp_lg_age_gyr"].astype(np.float64) + 9.0)
    lam = d["ssp_wave"].astype(np.float64)
    flux = d["ssp_flux"].astype(np.float64)
    if flux.shape != (lgZ.size, age_yr.size, lam.size):
        raise ValueError(f"ssp_flux has shape {flux.shape}, expected {(lgZ.size, age_yr.size, lam.size)}")
    return age_yr, lgZ, lam, np.ascontiguousarray(flux.transpose(1, 0, 2))


def tables(ssp_path, bands) -> SpsTables:
    """SpsTables from an SSP file and a band list (see filter_set)."""
    age_yr, lgZ, lam, ssp = load_ssp(ssp_path)
    return SpsTables(age_yr, lgZ, lam, ssp, *filter_set(bands))
