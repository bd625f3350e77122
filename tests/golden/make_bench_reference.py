"""Writes bench_error_reference.json: FP64 oracle values on rows sampled from
the benchmark's workloads, which bench.py reads to report the error of every
path and precision against the oracle (magnitudes in mag, gradients as the
per-row max-component relative error) without running the oracle itself.

Only ``oracle/`` and the seeded input generator ``sps_workloads`` are called;
nothing here comes from the CUDA path.  The observed magnitudes of each case
are the oracle's own approximate photometry at the seeded truth plus the
workload's noise, so the record is self-contained.

    python tests/golden/make_bench_reference.py   # rewrites bench_error_reference.json
"""
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sps_workloads as W          # noqa: E402
from oracle import sps as O        # noqa: E402

OUT = os.path.join(HERE, "bench_error_reference.json")


def cases():
    """(name, tables, z, theta_true, theta_eval, sigma, mask, noise, modes) of
    the sampled rows: 32 of the 100,000-pair production-grid workload and 16
    galaxies of the HMC workload (evaluated at independent prior draws)."""
    out = []
    wl = W.config(2)
    idx = np.linspace(0, wl.n_gal - 1, 32).astype(np.int64)
    out.append((W.CONFIG_NAMES[2], wl.tables, wl.z[idx], wl.theta_true[idx], wl.theta[idx],
                wl.sigma[idx], wl.mask[idx], wl.noise[idx], ("approx", "exact"), idx))
    wl = W.config(3)
    idx = np.linspace(0, wl.n_gal - 1, 16).astype(np.int64)
    ev = W.prior_draw(np.random.default_rng(W.SEED_BASE + 800), len(idx))
    out.append((W.CONFIG_NAMES[3], wl.tables, wl.z[idx], wl.theta_true[idx], ev,
                wl.sigma[idx], wl.mask[idx], wl.noise[idx], ("approx",), idx))
    return out


def compute():
    rec = {}
    for name, tabs, z, truth, ev, sigma, mask, noise, modes, idx in cases():
        th_true = torch.as_tensor(truth, dtype=torch.float64)
        mobs = O.photometry(th_true, z, tabs, "approx").numpy() + noise
        r = {"rows": idx.tolist(), "z": z.tolist(), "theta": ev.tolist(), "mag_obs": mobs.tolist(),
             "sigma": sigma.tolist(), "mask": mask.astype(np.int64).tolist()}
        for mode in modes:
            r[f"mag_{mode}"] = O.photometry(ev, z, tabs, mode).numpy().tolist()
            ll, g, _ = O.loglike_and_grad(ev, z, tabs, mobs, sigma, mask, mode, wrt_z=True)
            r[f"loglike_{mode}"] = ll.numpy().tolist()
            r[f"grad_{mode}"] = g.numpy().tolist()
        rec[name] = r
    return rec


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=0)
        f.write("\n")
    print("wrote", OUT)
