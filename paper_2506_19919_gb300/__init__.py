"""GB300 (sm_103a) implementation of the SPS photometry likelihood and batched
HMC of arXiv 2506.19919, behind the C ABI declared in include/sps.h.

The Python layer marshals arguments only: torch tensors provide device memory
and streams, every step of the computation runs in the CUDA library.  Loading
fails loudly when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (SPS_APPROX, SPS_BF16, SPS_EXACT, SPS_FP32, SPS_TF32X3, SpsError, check, load, sps_config,
                   sps_hmc_config, sps_hmc_stats, sps_info, sps_tables)

__all__ = ["Context", "diagnostics", "SpsError", "load", "MODES", "PRECS"]

MODES = {"exact": SPS_EXACT, "approx": SPS_APPROX}
PRECS = {"fp32": SPS_FP32, "bf16": SPS_BF16, "tf32x3": SPS_TF32X3}


def _vp(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


def _stream(t):
    if isinstance(t, torch.Tensor) and t.is_cuda:
        return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return None


def _f32(x, device=None):
    """x as a contiguous float32 tensor on `device` (a tensor's own device when
    None); a tensor that already is one is returned as it is, without a copy."""
    t = torch.as_tensor(x)
    return t.to(device=t.device if device is None else device, dtype=torch.float32).contiguous()


def _mask32(mask, device):
    """Band bitmasks as a contiguous int32 tensor holding the uint32 bits."""
    if isinstance(mask, torch.Tensor):
        if mask.dtype != torch.int32:
            mask = torch.as_tensor(np.asarray(mask.cpu().numpy(), dtype=np.int64).astype(np.uint32).view(np.int32))
        return mask.to(device).contiguous()
    return torch.as_tensor(np.asarray(mask, dtype=np.uint32).view(np.int32)).to(device).contiguous()


class Context:
    """One library context: tables on one device plus the current galaxy set."""

    def __init__(self, tables, device: int = 0, h0: float = 70.0, omega_m: float = 0.3,
                 prior_lo=None, prior_hi=None, gl_order: int = 6, panel: float = 0.25,
                 sigmoid_k=None, sigmoid_x0=None, skew=None):
        """skew = (xi, omega, s), each of 12 values, selects the skew-normal
        prior of Eq. SkewNormPrior on the unbounded parameters (see
        priors.fit_skew_normal); otherwise the prior is uniform in the bounded
        parameters.  sigmoid_k / sigmoid_x0 are the Eq. BoundingFunction
        hyper-parameters (see priors.tune_sigmoid); default 1 and 0."""
        lib = load()
        self._lib = lib
        cfg = sps_config()
        check(lib.sps_config_default(C.byref(cfg)), "sps_config_default")
        cfg.h0_kms_mpc = h0
        cfg.omega_m = omega_m
        cfg.device = device
        cfg.sfh_gl_order = gl_order
        cfg.sfh_panel = panel
        if prior_lo is not None:
            for k in range(_lib.NPARAM):
                cfg.prior_lo[k] = float(prior_lo[k])
                cfg.prior_hi[k] = float(prior_hi[k])
        for k in range(_lib.NPARAM):
            if sigmoid_k is not None:
                cfg.sigmoid_k[k] = float(sigmoid_k[k])
            if sigmoid_x0 is not None:
                cfg.sigmoid_x0[k] = float(sigmoid_x0[k])
        if skew is not None:
            cfg.prior = 1
            for k in range(_lib.NPARAM):
                cfg.skew_xi[k], cfg.skew_omega[k], cfg.skew_s[k] = (float(v[k]) for v in skew)
        self._keep = [np.ascontiguousarray(tables.age_yr, dtype=np.float64),
                      np.ascontiguousarray(tables.lgZ, dtype=np.float64),
                      np.ascontiguousarray(tables.lam_ang, dtype=np.float64),
                      np.ascontiguousarray(tables.ssp, dtype=np.float64),
                      np.ascontiguousarray(tables.band_kind, dtype=np.int32),
                      np.ascontiguousarray(tables.band_p0, dtype=np.float64),
                      np.ascontiguousarray(tables.band_p1, dtype=np.float64)]
        a, z, l, s, k, p0, p1 = self._keep
        tab_n = getattr(tables, "band_tab_n", None)
        tab_T = getattr(tables, "band_tab_T", None)
        if tab_n is not None:
            self._keep += [np.ascontiguousarray(tab_n, dtype=np.int32),
                           np.ascontiguousarray(tab_T, dtype=np.float64)]
        off = getattr(tables, "mdf_offset", None)
        self._mdf = None if off is None else np.ascontiguousarray(off, dtype=np.float64)
        t = sps_tables(len(a), len(z), len(l), len(k), a.ctypes.data, z.ctypes.data,
                       l.ctypes.data, s.ctypes.data, k.ctypes.data, p0.ctypes.data,
                       p1.ctypes.data, self._keep[7].ctypes.data if tab_n is not None else None,
                       self._keep[8].ctypes.data if tab_n is not None else None,
                       self._mdf.ctypes.data if self._mdf is not None else None)
        h = C.c_void_p()
        check(lib.sps_create(C.byref(h), C.byref(t), C.byref(cfg)), "sps_create")
        self.h = h
        self.device = torch.device("cuda", device)
        self.n_band = len(k)
        self.n_gal = 0

    def close(self):
        if getattr(self, "h", None):
            self._lib.sps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ set-up
    def set_galaxies(self, z, build_approx: bool = True):
        zt = _f32(z, "cpu").numpy()
        check(self._lib.sps_set_galaxies(self.h, _vp(zt), len(zt), int(build_approx), None),
              "sps_set_galaxies")
        self.n_gal = len(zt)

    def info(self) -> dict:
        i = sps_info()
        check(self._lib.sps_get_info(self.h, C.byref(i)), "sps_get_info")
        return {f: getattr(i, f) for f, _ in sps_info._fields_}

    def gl_rule(self):
        n = self.info()["sfh_gl_order"]
        x = np.zeros(n)
        w = np.zeros(n)
        check(self._lib.sps_gl_rule(self.h, _vp(x), _vp(w)), "sps_gl_rule")
        return x, w

    # ------------------------------------------------------------------ compute
    def photometry(self, theta, gal_idx=None, mode="exact", prec="fp32", out=None):
        th = _f32(theta, None if isinstance(theta, torch.Tensor) else self.device)
        n = th.shape[0]
        if out is None:
            out = torch.empty((n, self.n_band), dtype=torch.float32, device=th.device)
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=th.device).contiguous()
        check(self._lib.sps_photometry(self.h, _vp(th), _vp(gi), n, MODES[mode], PRECS[prec],
                                       _vp(out), _stream(th)), "sps_photometry")
        return out

    def loglike_grad(self, theta, mag_obs, sigma, mask, gal_idx=None, mode="approx",
                     prec="fp32", grad=True):
        th = _f32(theta, None if isinstance(theta, torch.Tensor) else self.device)
        dev = th.device
        n = th.shape[0]
        mo = _f32(mag_obs, dev)
        sg = _f32(sigma, dev)
        mk = _mask32(mask, dev)
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=dev).contiguous()
        ll = torch.empty(n, dtype=torch.float32, device=dev)
        g = torch.empty((n, _lib.NPARAM), dtype=torch.float32, device=dev) if grad else None
        check(self._lib.sps_loglike_grad(self.h, _vp(th), _vp(gi), n, _vp(mo), _vp(sg), _vp(mk),
                                         MODES[mode], PRECS[prec], _vp(ll), _vp(g), _stream(th)),
              "sps_loglike_grad")
        return ll, g

    def loglike_grad_z(self, theta, mag_obs, sigma, mask, gal_idx=None, mode="approx", prec="fp32"):
        """log L and its gradient with respect to the 12 parameters and the
        galaxy's redshift: returns (loglike [n], grad [n, 13]), column 12 = d/dz."""
        th = _f32(theta, None if isinstance(theta, torch.Tensor) else self.device)
        dev = th.device
        n = th.shape[0]
        mo = _f32(mag_obs, dev)
        sg = _f32(sigma, dev)
        mk = _mask32(mask, dev)
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=dev).contiguous()
        ll = torch.empty(n, dtype=torch.float32, device=dev)
        g = torch.empty((n, _lib.NPARAM + 1), dtype=torch.float32, device=dev)
        check(self._lib.sps_loglike_grad_z(self.h, _vp(th), _vp(gi), n, _vp(mo), _vp(sg), _vp(mk),
                                           MODES[mode], PRECS[prec], _vp(ll), _vp(g), _stream(th)),
              "sps_loglike_grad_z")
        return ll, g

    def loglike_grad_forward_mode(self, theta, mag_obs, sigma, mask, gal_idx=None):
        """The plain forward-mode comparison path (approximate photometry)."""
        th = _f32(theta, None if isinstance(theta, torch.Tensor) else self.device)
        dev = th.device
        n = th.shape[0]
        mo = _f32(mag_obs, dev)
        sg = _f32(sigma, dev)
        mk = _mask32(mask, dev)
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=dev).contiguous()
        ll = torch.empty(n, dtype=torch.float32, device=dev)
        g = torch.empty((n, _lib.NPARAM), dtype=torch.float32, device=dev)
        check(self._lib.sps_loglike_grad_forward_mode(self.h, _vp(th), _vp(gi), n, _vp(mo), _vp(sg),
                                                      _vp(mk), _vp(ll), _vp(g), _stream(th)),
              "sps_loglike_grad_forward_mode")
        return ll, g

    def hmc_run(self, theta0_unb, mag_obs, sigma, mask, chains_per_gal=4, n_warm=500,
                n_samp=500, L_min=8, L_max=64, target_accept=0.8, eps0=0.1, seed=2506199190,
                use_graph=True, autotune=True, samples=True, mode="approx", adapt_mass=0,
                path="fused", sampler="hmc", max_depth=10, prec="bf16"):
        """Batched HMC (sampler="hmc") or NUTS (sampler="nuts", identity metric,
        trees of at most max_depth doublings; L_min / L_max unused).
        path="fused" runs the persistent sampler (sps_hmc_run); path="plain"
        the lock-step forward-mode comparison baseline (sps_hmc_run_forward_mode,
        HMC with the identity metric only).  mode="exact" samples on the exact
        photometry (HMC, identity metric; prec selects the contraction)."""
        x0 = _f32(theta0_unb, None if isinstance(theta0_unb, torch.Tensor) else self.device)
        dev = x0.device
        mo = _f32(mag_obs, dev)
        sg = _f32(sigma, dev)
        mk = _mask32(mask, dev)
        nc = x0.shape[0]
        cfg = sps_hmc_config()
        check(self._lib.sps_hmc_config_default(C.byref(cfg)), "sps_hmc_config_default")
        cfg.chains_per_gal, cfg.n_warm, cfg.n_samp = chains_per_gal, n_warm, n_samp
        cfg.L_min, cfg.L_max = L_min, L_max
        cfg.target_accept, cfg.eps0, cfg.seed = target_accept, eps0, seed
        cfg.mode = MODES[mode]
        cfg.prec = PRECS[prec]
        cfg.use_graph, cfg.autotune = int(use_graph), int(autotune)
        cfg.adapt_mass = {False: 0, True: 1, "diag": 1, "dense": 2, "none": 0}.get(adapt_mass, adapt_mass)
        cfg.sampler = {"hmc": 0, "nuts": 1}[sampler]
        cfg.max_depth = max_depth
        out = {
            "samples": torch.empty((nc, n_samp, _lib.NPARAM), dtype=torch.float32, device=dev)
            if samples else None,
            "accept_prob": torch.empty(nc, dtype=torch.float32, device=dev),
            "step_size": torch.empty(nc, dtype=torch.float32, device=dev),
            "divergences": torch.empty(nc, dtype=torch.int32, device=dev),
            "grad_evals": torch.empty(nc, dtype=torch.int64, device=dev),
            "status": torch.empty(nc, dtype=torch.int32, device=dev),
        }
        st = sps_hmc_stats(*(C.c_void_p(out[k].data_ptr()) for k in
                             ("accept_prob", "step_size", "divergences", "grad_evals", "status")))
        fn = {"fused": "sps_hmc_run", "plain": "sps_hmc_run_forward_mode"}[path]
        check(getattr(self._lib, fn)(self.h, C.byref(cfg), _vp(x0), _vp(mo), _vp(sg), _vp(mk),
                                     _vp(out["samples"]), C.byref(st), _stream(x0)), fn)
        return out

    def leapfrog(self, x0, p0, eps, L, mag_obs, sigma, mask, gal_idx=None):
        x = _f32(x0, self.device)
        dev = x.device
        n = x.shape[0]
        p = _f32(p0, dev)
        e = _f32(eps, dev)
        l = torch.as_tensor(L, dtype=torch.int32).to(dev).contiguous()
        mo, sg = _f32(mag_obs, dev), _f32(sigma, dev)
        mk = torch.as_tensor(np.asarray(mask, dtype=np.uint32).view(np.int32)).to(dev).contiguous()
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=dev).contiguous()
        xo = torch.empty_like(x)
        po = torch.empty_like(x)
        lo = torch.empty(n, dtype=torch.float64, device=dev)
        check(self._lib.sps_leapfrog(self.h, _vp(x), _vp(p), _vp(e), _vp(l), _vp(gi), n, _vp(mo),
                                     _vp(sg), _vp(mk), _vp(xo), _vp(po), _vp(lo), _stream(x)),
              "sps_leapfrog")
        return xo, po, lo

    def wait_probe(self, ready: bool, spin_limit: int = 1 << 16):
        """Run the bounded device wait on a barrier that is (ready) or is never
        completed; raises SpsError (SPS_E_TIMEOUT) when the wait gives up."""
        check(self._lib.sps_wait_probe(self.h, int(bool(ready)), spin_limit, None), "sps_wait_probe")

    def philox(self, ctr, key: int):
        c = torch.as_tensor(np.asarray(ctr, dtype=np.uint32).view(np.int32)).to(self.device).contiguous()
        n = c.shape[0]
        o = torch.empty_like(c)
        check(self._lib.sps_philox(self.h, _vp(c), n, C.c_uint64(key), _vp(o), _stream(c)),
              "sps_philox")
        return o.cpu().numpy().view(np.uint32)

    def weights(self, theta, gal_idx=None):
        th = _f32(theta, self.device)
        n = th.shape[0]
        info = self.info()
        W = torch.empty((n, info["n_age"] * info["n_met"]), dtype=torch.float32, device=th.device)
        M = torch.empty(n, dtype=torch.float64, device=th.device)
        gi = None if gal_idx is None else torch.as_tensor(gal_idx, dtype=torch.int32,
                                                             device=th.device).contiguous()
        check(self._lib.sps_weights(self.h, _vp(th), _vp(gi), n, _vp(W), _vp(M), _stream(th)),
              "sps_weights")
        return W, M


def diagnostics(samples, n_gal: int, chains_per_gal: int):
    """Multi-chain ESS and split R-hat per galaxy and parameter (host, FP64)."""
    lib = load()
    s = np.ascontiguousarray(samples.detach().cpu().numpy() if isinstance(samples, torch.Tensor)
                             else samples, dtype=np.float32)
    nd, npar = s.shape[1], s.shape[2]
    ess = np.zeros((n_gal, npar))
    rh = np.zeros((n_gal, npar))
    check(lib.sps_diagnostics(_vp(s), n_gal, chains_per_gal, nd, npar, _vp(ess), _vp(rh)),
          "sps_diagnostics")
    return ess, rh
