"""The HMC team kernel's last wave run as one-chain teams (a second launch)
gives exactly the chains of one launch of two-chain teams: the draws come
from Philox counters per chain, and both kernels take the same arithmetic per
chain.  1,300 galaxies x 4 chains make 2,600 two-chain teams, more than the
resident warps of the default launch shape, with a partial last wave."""
import os

import numpy as np
import pytest
import torch

import sps_workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("use_graph", [False, True])
def test_split_last_wave_matches_one_launch(use_graph):
    """With and without graph capture (the bench's path: the side-stream fork
    and join captured into the graph)."""
    import paper_2506_19919_gb300 as pkg
    wl = W.config(3, n_gal=1300)
    dev = torch.device("cuda", 0)
    ctx = pkg.Context(wl.tables, device=0)
    ctx.set_galaxies(wl.z, build_approx=True)
    mt = ctx.photometry(torch.as_tensor(wl.theta_true, dtype=torch.float32, device=dev), mode="approx")
    mo = (mt + torch.as_tensor(wl.noise, dtype=torch.float32, device=dev)).contiguous()
    x0 = torch.as_tensor(wl.extra["theta0_unb"], dtype=torch.float32, device=dev)
    kw = dict(chains_per_gal=4, n_warm=4, n_samp=4, L_min=4, L_max=12, autotune=False, use_graph=use_graph)
    runs = {}
    for tail in ("1", "0"):
        os.environ["SPS_HMC_TAIL"] = tail
        try:
            o = ctx.hmc_run(x0, mo, wl.sigma, wl.mask, **kw)
            torch.cuda.synchronize()
        finally:
            os.environ.pop("SPS_HMC_TAIL", None)
        runs[tail] = ({k: v.cpu().numpy() for k, v in o.items() if v is not None}, ctx.info()["hmc_launches"])
    assert runs["1"][1] == 2 and runs["0"][1] == 1
    split, one = runs["1"][0], runs["0"][0]
    assert np.isfinite(one["samples"]).all()
    for k in one:
        np.testing.assert_array_equal(split[k], one[k], err_msg=k)
