"""Host logic of the Python binding, without a GPU: argument marshalling
(dtype, layout and bitmask handling) and the torch.autograd.Function around
the library's log L + gradient, driven by a stand-in context whose log L is
known in closed form (the library's own numbers are held to the oracle by
the GPU parity tests)."""
import numpy as np
import torch

import paper_2506_19919_gb300 as pkg
from paper_2506_19919_gb300 import autograd as AG


def test_f32_passes_float32_tensors_through_and_converts_the_rest():
    t = torch.randn(5, 12)
    assert pkg._f32(t) is t                                   # no copy, same pointer
    d = pkg._f32(t.double())
    assert d.dtype == torch.float32 and torch.equal(d, t)
    nc = torch.randn(12, 5).t()                               # non-contiguous view
    c = pkg._f32(nc)
    assert c.is_contiguous() and torch.equal(c, nc)
    a = pkg._f32(np.arange(6.0).reshape(2, 3), "cpu")
    assert a.dtype == torch.float32 and a.shape == (2, 3)


def test_mask32_keeps_the_32_bits():
    m = np.array([0, 1, 0x7FFFFFFF, 0x80000001, 0xFFFFFFFF], np.uint64)
    want = m.astype(np.uint32).view(np.int32)
    for src in (m.astype(np.uint32), torch.as_tensor(m.astype(np.int64)),
                torch.as_tensor(m.astype(np.uint32).view(np.int32))):
        got = pkg._mask32(src, "cpu")
        assert got.dtype == torch.int32 and got.is_contiguous()
        np.testing.assert_array_equal(got.numpy(), want)
    t = torch.as_tensor(want)
    assert pkg._mask32(t, "cpu") is t


class _StandIn:
    """loglike_grad with log L = -1/2 sum_k w_k (theta_k - c_k)^2 per row."""

    def __init__(self, c, w):
        self.c, self.w, self.calls = c, w, []

    def loglike_grad(self, theta, mag_obs, sigma, mask, gal_idx=None, mode="approx", prec="fp32",
                     grad=True):
        self.calls.append((theta.requires_grad, grad, mode, prec, gal_idx))
        r = theta - self.c
        return -0.5 * (self.w * r * r).sum(1), -(self.w * r)


def test_autograd_function_backpropagates_the_library_gradient():
    torch.manual_seed(0)
    c = torch.randn(12, dtype=torch.float64)
    w = torch.rand(12, dtype=torch.float64) + 0.5
    sps = _StandIn(c, w)
    theta = torch.randn(4, 12, dtype=torch.float64, requires_grad=True)
    f = lambda th: AG.loglike(th, sps, None, None, None, mode="exact", prec="bf16")
    assert torch.autograd.gradcheck(f, (theta,), eps=1e-6, atol=1e-8)   # central differences
    ll = f(theta)
    (gw,) = torch.autograd.grad((ll * torch.arange(1.0, 5.0, dtype=torch.float64)).sum(), theta)
    np.testing.assert_allclose(gw.numpy(), (-(w * (theta - c)) * torch.arange(1.0, 5.0)[:, None]).detach().numpy(),
                               rtol=1e-14)
    assert all(not rg and g and m == "exact" and p == "bf16" for rg, g, m, p, _ in sps.calls)
