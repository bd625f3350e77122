"""Writes oracle_regression.json: the FP64 oracle's outputs on a small seeded
case (tiny SSP grid, four galaxies), stored so that any later change to the
oracle's arithmetic shows up as a failing test and is made on purpose.

Only ``oracle/`` and the seeded input generator ``sps_workloads`` are called;
nothing here comes from the CUDA path.  These values are a regression record
of the oracle, not a pin of it: the pins (closed forms, invariants, brute
force, limits) are in tests/test_oracle_*.py.

    python tests/golden/make_golden.py        # rewrites oracle_regression.json
"""
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import sps_workloads as W          # noqa: E402
from oracle import hmc as OH       # noqa: E402
from oracle import nuts as ON      # noqa: E402
from oracle import sps as O        # noqa: E402

OUT = os.path.join(HERE, "oracle_regression.json")


def case():
    """The inputs: everything seeded, rounded to float32 like the workloads."""
    rng = np.random.default_rng(W.SEED_BASE + 700)
    tables = W.tiny_tables()
    G = 4
    theta = W.prior_draw(rng, G)
    z = np.round(rng.uniform(0.05, 2.0, G), 4).astype(np.float32).astype(np.float64)
    theta_eval = W.prior_draw(rng, G)
    sigma = np.full((G, tables.n_band), 0.05)
    mask = np.array([0b1111, 0b0111, 0b1101, 0b1011], np.uint32)
    noise = np.round(rng.normal(0.0, 0.05, (G, tables.n_band)), 4)
    return tables, theta, z, theta_eval, sigma, mask, noise


def compute():
    tables, theta, z, theta_eval, sigma, mask, noise = case()
    th = torch.as_tensor(theta, dtype=torch.float64)
    out = {"z": z.tolist(),
           "t_obs_gyr": [float(O.t_obs_gyr(float(v))) for v in z],
           "lum_dist_mpc": [float(O.lum_dist_mpc(float(v))) for v in z]}
    Wt, M, _, _ = O.ssp_weights(th, tables, O.t_obs_gyr(torch.as_tensor(z)))
    out["mass_formed"] = M.reshape(-1).tolist()
    out["weights_row0"] = Wt.reshape(len(z), -1)[0].tolist()
    for mode in ("exact", "approx"):
        out[f"mag_{mode}"] = O.photometry(th, z, tables, mode).numpy().tolist()
    mobs = O.photometry(th, z, tables, "exact").numpy() + noise
    out["mag_obs"] = mobs.tolist()
    for mode in ("exact", "approx"):
        ll, g, _ = O.loglike_and_grad(theta_eval, z, tables, mobs, sigma, mask, mode)
        out[f"loglike_{mode}"] = ll.numpy().tolist()
        out[f"grad_{mode}"] = g.numpy().tolist()
    # samplers: two chains on each of the first two galaxies, from the truth
    rows = np.repeat(np.arange(2), 2)
    x0 = W.unbounded_of(theta[rows]) + 0.01 * np.arange(1, 13)[None, :] * np.array([1, -1, 1, -1])[:, None]
    tgt = OH.ApproxTarget(tables, z[:2], mobs[:2], sigma[:2], mask[:2], W.PRIOR_LO, W.PRIOR_HI)
    h = OH.run_hmc(tgt, x0, rows, seed=11, n_warm=2, n_samp=2, L_min=4, L_max=8, eps0=0.02)
    out["hmc_samples"] = h["samples"].tolist()
    out["hmc_eps"] = h["eps"].tolist()
    n = ON.run_nuts(tgt, x0, rows, seed=13, n_warm=1, n_samp=2, eps0=0.02, max_depth=4)
    out["nuts_samples"] = n["samples"].tolist()
    out["nuts_grad_evals"] = np.asarray(n["grad_evals"]).tolist()
    return out


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(compute(), f, indent=0)
        f.write("\n")
    print("wrote", OUT)
