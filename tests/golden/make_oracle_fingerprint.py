"""Write the oracle's FGMRES solution fingerprint for a large workload.

The oracle's full solution of the 128x128x64 two-phase workload (5,342,147
unknowns) is too large to store and too slow to recompute inside a test or
the benchmark, so this script runs the oracle once (plain serial FP64, about
ten minutes) and stores what a comparison needs:

  * iterations, restarts-free true relative residual, ||x||_2, max |x_i|;
  * x at 4096 indices drawn with numpy default_rng(20240) (without
    replacement), printed with 17 significant digits;
  * p_k = g_k . x for 16 probe vectors g_k = default_rng(1000 + k)
    .standard_normal(n): E[(g . e)^2] = ||e||^2 for any fixed e, so the
    probes give an unbiased estimate of ||x_gpu - x_oracle||^2.

Only oracle/ and the seeded generator are used; nothing comes from the CUDA
path.  Usage:  python tests/golden/make_oracle_fingerprint.py two_phase_128x128x64
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1904_05960_gb300 import synth  # noqa: E402

NSAMPLE = 4096
NPROBE = 16
SAMPLE_SEED = 20240
PROBE_SEED = 1000


def sample_indices(n):
    return np.sort(np.random.default_rng(SAMPLE_SEED).choice(n, size=min(NSAMPLE, n), replace=False))


def probe(k, n):
    return np.random.default_rng(PROBE_SEED + k).standard_normal(n)


WORKLOADS = {
    # two-phase, 128x128x64 cells, lognormal k (sigma 2, correlation 16/16/2),
    # lognormal E (sigma 1.5): 5,342,147 unknowns
    "two_phase_128x128x64": lambda: synth.two_phase(128, 128, 64, seed=0, sigma=2.0, E_sigma=1.5),
}


def main(name):
    p = WORKLOADS[name]()
    t0 = time.perf_counter()
    o = oracle.Oracle(p)
    t1 = time.perf_counter()
    r = o.fgmres(p.rhs)
    t2 = time.perf_counter()
    x = r["x"]
    idx = sample_indices(p.n)
    out = dict(
        workload=name, n=p.n, nnz=p.nnz,
        iters=r["iters"], status=r["status"], relres=r["relres"],
        norm2=float(np.linalg.norm(x)), maxabs=float(np.abs(x).max()),
        oracle_setup_s=t1 - t0, oracle_solve_s=t2 - t1,
        sample_seed=SAMPLE_SEED, probe_seed=PROBE_SEED,
        sample_idx=[int(i) for i in idx], sample_x=[repr(float(v)) for v in x[idx]],
        probes=[repr(float(probe(k, p.n) @ x)) for k in range(NPROBE)])
    path = os.path.join(HERE, f"oracle_{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print(f"wrote {path}: iters {r['iters']}, relres {r['relres']:.3e}, "
          f"setup {t1 - t0:.1f} s, solve {t2 - t1:.1f} s")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "two_phase_128x128x64")
