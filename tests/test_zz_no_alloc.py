"""The allocation-free exact photometry entry point.

It serves callers that cannot allocate device memory while running (a fixed
device-memory budget reserved at start-up, a host allocator that owns the
device memory, or loops where cudaMalloc would synchronise or fail): its
scratch is a fixed array compiled into the library.  Its magnitudes must
equal those of the ordinary sps_photometry entry point (exact, FP32) and
those of the FP64 oracle within the magnitude tolerance the parity tests
use, on two calls in a row that share the static scratch.  This file is
collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import sps_workloads as W
from oracle import sps as O

pytestmark = pytest.mark.gpu

MAG_TOL = 1e-3


def _vp(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_matches_photometry_on_two_calls():
    import paper_2506_19919_gb300 as pkg
    from paper_2506_19919_gb300 import _lib
    lib = _lib.load()
    wl = W.config(0)                                  # 64 galaxies, 50 x 6 x 2000 grid
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=False)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, n, use_idx in ((0, 64, False), (1, 40, True)):
        th = torch.as_tensor(W.prior_draw(np.random.default_rng(seed), n), dtype=torch.float32,
                             device="cuda")
        gidx = (torch.as_tensor(np.random.default_rng(seed).permutation(64)[:n], dtype=torch.int32,
                                device="cuda") if use_idx else None)
        ref = ctx.photometry(th, gal_idx=gidx, mode="exact", prec="fp32")
        out = torch.full((n, 6), float("nan"), dtype=torch.float32, device="cuda")
        st = lib.sps_photometry_exact_noalloc(ctx.h, _vp(th), _vp(gidx) if use_idx else None, n,
                                              _vp(out), stream)
        assert st == 0, lib.sps_last_error_message()
        assert torch.isfinite(out).all()
        assert (out - ref).abs().max().item() < MAG_TOL
        rows = gidx.cpu().numpy() if use_idx else np.arange(64)
        mo = O.photometry(th.cpu().numpy().astype(np.float64), wl.z[rows], wl.tables, "exact")
        assert np.abs(out.cpu().numpy() - mo.numpy()).max() < MAG_TOL
    # sizes beyond the static scratch and host arrays are refused with a message
    big = torch.zeros(40000, dtype=torch.int32, device="cuda")
    thb = torch.zeros((40000, 12), dtype=torch.float32, device="cuda")
    outb = torch.zeros((40000, 6), dtype=torch.float32, device="cuda")
    assert lib.sps_photometry_exact_noalloc(ctx.h, _vp(thb), _vp(big), 40000, _vp(outb), stream) == 2
    assert b"32 MiB" in lib.sps_last_error_message()
    host = np.zeros((64, 12), np.float32)
    assert lib.sps_photometry_exact_noalloc(ctx.h, C.c_void_p(host.ctypes.data), None, 64,
                                            _vp(out), stream) == 1
    assert b"device pointers" in lib.sps_last_error_message()
    assert lib.sps_photometry_exact_noalloc(None, _vp(thb), None, 64, _vp(out), stream) == 1
    assert b"null context" in lib.sps_last_error_message()
    assert torch.cuda.current_device() == 0
    ctx.close()
