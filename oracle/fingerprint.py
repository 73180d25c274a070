"""Comparison of a solution with a stored oracle fingerprint (test
infrastructure, like the rest of this package).

tests/golden/make_oracle_fingerprint.py runs the oracle once on a workload too
large to store or re-solve in a test and keeps: ||x||_2, x at seeded sample
indices, and g_k . x for seeded Gaussian probe vectors g_k.  Given another
solution x' this module returns

  * sample_rel: ||x'[S] - x[S]||_2 / ||x[S]||_2 over the stored sample S
    (exact, not an estimate), and the largest entry difference over the
    largest sampled entry;
  * probe_rel: sqrt(mean_k (g_k . x' - g_k . x)^2) / ||x||_2, an unbiased
    estimate of ||x' - x||^2 / ||x||^2 under the square root (E[(g . e)^2] =
    ||e||^2 for standard normal g), with 16 probes its relative spread is
    about 18%; its floor is the FP64 rounding of the probe products,
    ~1e-13 relative.
"""
import json
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "tests", "golden")


def load(name):
    with open(os.path.join(GOLDEN, f"oracle_{name}.json")) as f:
        d = json.load(f)
    d["sample_idx"] = np.asarray(d["sample_idx"], dtype=np.int64)
    d["sample_x"] = np.asarray([float(v) for v in d["sample_x"]])
    d["probes"] = np.asarray([float(v) for v in d["probes"]])
    return d


def compare(x, fp):
    x = np.asarray(x, dtype=np.float64)
    n = int(fp["n"])
    assert x.shape == (n,), (x.shape, n)
    idx, xs = fp["sample_idx"], fp["sample_x"]
    d = x[idx] - xs
    out = dict(sample_rel=float(np.linalg.norm(d) / np.linalg.norm(xs)),
               sample_maxrel=float(np.abs(d).max() / np.abs(xs).max()),
               samples=int(len(idx)))
    diffs = []
    for k, pk in enumerate(fp["probes"]):
        g = np.random.default_rng(int(fp["probe_seed"]) + k).standard_normal(n)
        diffs.append(float(g @ x) - pk)
    out["probe_rel"] = float(np.sqrt(np.mean(np.square(diffs))) / fp["norm2"])
    out["probes"] = len(diffs)
    out["oracle_iters"] = int(fp["iters"])
    return out
