"""The C-ABI library loads and exports every symbol include/sps.h declares;
the ctypes structs match the C layouts; host-only entry points work without
a GPU (no compute call needs one here)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sps.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2506_19919_gb300 import build as b
    b.build()
    from paper_2506_19919_gb300 import _lib
    return _lib.load()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sps_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (sps_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def test_ctypes_layouts_match_c(tmp_path):
    from paper_2506_19919_gb300 import _lib
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "sps.h"\n'
                   "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu\\n\","
                   "sizeof(sps_tables), sizeof(sps_config), sizeof(sps_hmc_config),"
                   "sizeof(sps_hmc_stats), sizeof(sps_info), offsetof(sps_config, sfh_panel),"
                   "offsetof(sps_hmc_config, seed), offsetof(sps_info, n_gal));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    c_sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    py = [C.sizeof(_lib.sps_tables), C.sizeof(_lib.sps_config), C.sizeof(_lib.sps_hmc_config),
          C.sizeof(_lib.sps_hmc_stats), C.sizeof(_lib.sps_info), _lib.sps_config.sfh_panel.offset,
          _lib.sps_hmc_config.seed.offset, _lib.sps_info.n_gal.offset]
    assert c_sizes == py


def test_defaults_and_error_strings(lib):
    from paper_2506_19919_gb300 import _lib
    import sps_workloads as W
    cfg = _lib.sps_config()
    assert lib.sps_config_default(C.byref(cfg)) == 0
    np.testing.assert_array_equal(np.array(cfg.prior_lo[:]), W.PRIOR_LO)
    np.testing.assert_array_equal(np.array(cfg.prior_hi[:]), W.PRIOR_HI)
    assert cfg.sfh_gl_order == 6 and cfg.h0_kms_mpc == 70.0
    h = _lib.sps_hmc_config()
    assert lib.sps_hmc_config_default(C.byref(h)) == 0
    assert (h.L_min, h.L_max, h.n_warm, h.n_samp) == (8, 64, 500, 500)
    for s in range(9):
        assert lib.sps_error_string(s)
    assert lib.sps_config_default(None) == 1


def test_bad_tables_rejected_on_host(lib):
    """Argument checks run before any device work: invalid tables return
    SPS_E_SHAPE / SPS_E_INVALID_ARG."""
    from paper_2506_19919_gb300 import _lib
    import sps_workloads as W
    t = W.tiny_tables()
    keep = [np.ascontiguousarray(x) for x in (t.age_yr, t.lgZ, t.lam_ang, t.ssp,
                                              t.band_kind.astype(np.int32), t.band_p0, t.band_p1)]
    def mk(n_age):
        return _lib.sps_tables(n_age, len(t.lgZ), len(t.lam_ang), len(t.band_kind),
                               *[k.ctypes.data for k in keep])
    h = C.c_void_p()
    tab = mk(300)
    assert lib.sps_create(C.byref(h), C.byref(tab), None) == 2
    bad_age = keep[0].copy()
    bad_age[2] = bad_age[1]
    keep2 = [bad_age] + keep[1:]
    tab2 = _lib.sps_tables(len(t.age_yr), len(t.lgZ), len(t.lam_ang), len(t.band_kind),
                           *[k.ctypes.data for k in keep2])
    assert lib.sps_create(C.byref(h), C.byref(tab2), None) == 1


def test_bad_tabulated_bands_rejected_on_host(lib):
    """sps_create checks tabulated filter curves before any device work: too
    few samples, a negative throughput."""
    from paper_2506_19919_gb300 import _lib
    import sps_workloads as W
    t = W.tiny_tables()
    kind = np.array([2, 0, 0, 0], np.int32)
    p0 = np.array([4000.0, 4500, 6000, 8000])
    p1 = np.array([10.0, 6000, 8000, 9000])

    def create(tab_n, tab_T):
        keep = [np.ascontiguousarray(x) for x in (t.age_yr, t.lgZ, t.lam_ang, t.ssp, kind, p0, p1,
                                                  np.asarray(tab_n, np.int32), np.asarray(tab_T, np.float64))]
        tab = _lib.sps_tables(len(t.age_yr), len(t.lgZ), len(t.lam_ang), 4, *[k.ctypes.data for k in keep])
        h = C.c_void_p()
        return lib.sps_create(C.byref(h), C.byref(tab), None)

    assert create([1, 0, 0, 0], [0.5]) == 1
    assert create([2, 0, 0, 0], [-0.1, 0.2]) == 1


def test_host_diagnostics_match_oracle(lib):
    from oracle import diagnostics as D
    import paper_2506_19919_gb300 as pkg
    rng = np.random.default_rng(5)
    G, Cc, N, P = 3, 4, 400, 2
    s = rng.normal(size=(G * Cc, N, P)).astype(np.float32)
    # an autocorrelated parameter and a shifted chain
    for i in range(1, N):
        s[:, i, 1] = 0.8 * s[:, i - 1, 1] + 0.6 * s[:, i, 1]
    s[1, :, 0] += 2.0
    ess, rh = pkg.diagnostics(s, G, Cc)
    for g in range(G):
        for p in range(P):
            x = s[g * Cc:(g + 1) * Cc, :, p].astype(np.float64)
            assert ess[g, p] == pytest.approx(D.ess(x), rel=1e-9)
            assert rh[g, p] == pytest.approx(D.split_rhat(x), rel=1e-9)


class _Tab:
    """sps_tables over numpy arrays kept alive by this object (tiny grid)."""

    def __init__(self, **over):
        import sps_workloads as W
        t = W.tiny_tables()
        a = dict(age_yr=t.age_yr, lgZ=t.lgZ, lam_ang=t.lam_ang, ssp=t.ssp,
                 band_kind=t.band_kind.astype(np.int32), band_p0=t.band_p0, band_p1=t.band_p1,
                 band_tab_n=None, band_tab_T=None, mdf_offset=None)
        a.update(over)
        self.keep = {k: (None if v is None else np.ascontiguousarray(v)) for k, v in a.items()}
        dims = [len(self.keep["age_yr"]), len(self.keep["lgZ"]), len(self.keep["lam_ang"]),
                len(self.keep["band_kind"])]
        from paper_2506_19919_gb300 import _lib
        ptr = lambda k: None if self.keep[k] is None else self.keep[k].ctypes.data
        self.s = _lib.sps_tables(*dims, *[ptr(k) for k in ("age_yr", "lgZ", "lam_ang", "ssp", "band_kind",
                                                             "band_p0", "band_p1", "band_tab_n",
                                                             "band_tab_T", "mdf_offset")])


def _create(lib, tab, cfg=None):
    h = C.c_void_p()
    st = lib.sps_create(C.byref(h), C.byref(tab.s), None if cfg is None else C.byref(cfg))
    msg = lib.sps_last_error_message()
    msg = msg.decode() if isinstance(msg, bytes) else str(msg)
    if st == 0:
        lib.sps_destroy(h)
    else:
        assert not h.value                     # no context is handed out on failure
    return st, msg


def _cfg(lib, **over):
    from paper_2506_19919_gb300 import _lib
    cfg = _lib.sps_config()
    assert lib.sps_config_default(C.byref(cfg)) == 0
    for k, v in over.items():
        if isinstance(v, tuple):                # (index, value) into an array field
            getattr(cfg, k)[v[0]] = v[1]
        else:
            setattr(cfg, k, v)
    return cfg


@pytest.mark.parametrize("over,phrase", [
    (dict(sigmoid_k=(3, 0.0)), "sigmoid_k"),
    (dict(sigmoid_k=(3, float("inf"))), "sigmoid_k"),
    (dict(sigmoid_x0=(0, float("nan"))), "sigmoid_x0"),
    (dict(prior=2), "prior"),
    (dict(prior=1, skew_omega=(5, 0.0)), "skew-normal"),
    (dict(prior=1, skew_s=(2, float("inf"))), "skew-normal"),
    (dict(prior=1, skew_xi=(7, float("nan"))), "skew-normal"),
    (dict(sfh_gl_order=1), "sfh_gl_order"),
    (dict(sfh_gl_order=17), "sfh_gl_order"),
    (dict(sfh_panel=0.0), "sfh_panel"),
    (dict(sfh_panel=2.5), "sfh_panel"),
    (dict(sfh_panel=0.01), "panel budget"),
    (dict(omega_m=1.0), "cosmology"),
    (dict(h0_kms_mpc=0.0), "cosmology"),
    (dict(prior_hi=(4, 0.0)), "prior_hi"),
])
def test_bad_config_rejected_on_host(lib, over, phrase):
    """Every sps_config field is checked before any device work."""
    st, msg = _create(lib, _Tab(), _cfg(lib, **over))
    assert st == 1 and phrase in msg, (st, msg)


def _bad(name):
    import sps_workloads as W
    t = W.tiny_tables()
    if name == "mdf_nan":
        o = np.zeros(len(t.age_yr)); o[1] = np.nan
        return dict(mdf_offset=o), "mdf_offset"
    if name == "mdf_large":
        o = np.zeros(len(t.age_yr)); o[0] = 10.5
        return dict(mdf_offset=o), "mdf_offset"
    if name == "ssp_negative":
        s = t.ssp.copy(); s.reshape(-1)[17] = -1e-30
        return dict(ssp=s), "SSP table"
    if name == "ssp_nan":
        s = t.ssp.copy(); s.reshape(-1)[-1] = np.nan
        return dict(ssp=s), "SSP table"
    if name == "band_kind":
        k = t.band_kind.astype(np.int32).copy(); k[2] = 3
        return dict(band_kind=k), "band kind"
    if name == "tophat_reversed":
        k = np.zeros(len(t.band_kind), np.int32)
        p0, p1 = t.band_p0.copy(), t.band_p1.copy(); p0[1], p1[1] = p1[1], p0[1]
        return dict(band_kind=k, band_p0=p0, band_p1=p1), "top-hat"
    if name == "gauss_fwhm":
        k = np.ones(len(t.band_kind), np.int32)
        p0 = np.array([4000.0, 5000, 6000, 7000]); p1 = np.array([500.0, 0.0, 500, 500])
        return dict(band_kind=k, band_p0=p0, band_p1=p1), "Gaussian band"
    if name == "lgz_order":
        z = t.lgZ.copy(); z[1] = z[0]
        return dict(lgZ=z), "lgZ"
    if name == "lam_order":
        lam = t.lam_ang.copy(); lam[10] = lam[9]
        return dict(lam_ang=lam), "wavelength grid"
    raise KeyError(name)


@pytest.mark.parametrize("name", ["mdf_nan", "mdf_large", "ssp_negative", "ssp_nan", "band_kind",
                                  "tophat_reversed", "gauss_fwhm", "lgz_order", "lam_order"])
def test_bad_table_values_rejected_on_host(lib, name):
    over, phrase = _bad(name)
    st, msg = _create(lib, _Tab(**over))
    assert st == 1 and phrase in msg, (st, msg)


def test_bad_table_sizes_rejected_on_host(lib):
    tab = _Tab()
    for field, value in (("n_met", 0), ("n_band", 33), ("n_lam", 1), ("n_age", 1), ("n_age", 129)):
        saved = getattr(tab.s, field)
        setattr(tab.s, field, value)
        st, _ = _create(lib, tab)
        setattr(tab.s, field, saved)
        assert st == 2, (field, value, st)


def test_valid_tables_without_a_device_are_unsupported(lib):
    """The checks pass on valid input; with no CUDA device the call then
    reports SPS_E_UNSUPPORTED (on a GPU machine it would create a context)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, msg = _create(lib, _Tab())
    assert st == 6 and "device" in msg, (st, msg)
