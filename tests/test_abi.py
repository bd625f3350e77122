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
