"""Regression record of the FP64 oracle (tests/golden/oracle_regression.json,
written by tests/golden/make_golden.py, which calls only the oracle and the
seeded input generator).  A failure means the oracle's arithmetic changed:
if the change is meant, rewrite the record and name, in the commit, the
passage of the paper that justifies it."""
import importlib.util
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden")


def _load_generator(name="make_golden"):
    spec = importlib.util.spec_from_file_location(name, os.path.join(GOLD, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_reproduces_its_regression_record():
    with open(os.path.join(GOLD, "oracle_regression.json")) as f:
        ref = json.load(f)
    got = _load_generator().compute()
    assert set(got) == set(ref)
    for key in ref:
        a, b = np.asarray(got[key], dtype=np.float64), np.asarray(ref[key], dtype=np.float64)
        assert a.shape == b.shape, key
        if key == "nuts_grad_evals":
            np.testing.assert_array_equal(a, b)
            continue
        # relative to each array's scale: BLAS and libm may round differently
        # across machines, and the samplers amplify that only mildly over a
        # few short trajectories
        tol = 1e-7 if key.startswith(("hmc", "nuts")) else 1e-9
        scale = np.abs(b).max() if b.size else 1.0
        np.testing.assert_allclose(a, b, rtol=tol, atol=tol * scale, err_msg=key)


def test_bench_error_reference_is_the_oracle():
    """bench_error_reference.json (the FP64 values bench.py reports its
    errors against) is what the oracle gives on those rows now."""
    with open(os.path.join(GOLD, "bench_error_reference.json")) as f:
        ref = json.load(f)
    got = _load_generator("make_bench_reference").compute()
    assert set(got) == set(ref)
    for case in ref:
        assert set(got[case]) == set(ref[case]), case
        for key in ref[case]:
            a = np.asarray(got[case][key], dtype=np.float64)
            b = np.asarray(ref[case][key], dtype=np.float64)
            assert a.shape == b.shape, (case, key)
            scale = np.abs(b).max() if b.size else 1.0
            np.testing.assert_allclose(a, b, rtol=1e-9, atol=1e-9 * scale, err_msg=f"{case} {key}")
