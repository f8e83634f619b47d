"""Writes tests/golden/fullsize_box64x64x256_re2000_q4.json: the FP64 oracle's
solution of the 4,343,300-unknown tangent (64x64x256 hexes, Re 2000, four
quadrant outlets, seed 2) solved to the outer tolerance delta^r = 1e-12, far
below the 1e-8 of the benchmark, so that the oracle's own error is negligible
against the solution-error bars (1e-6 FP64, 1e-5 mixed precision).

Stored, for the GPU test to compare with (nothing here comes from the CUDA
library; the script calls only oracle/ and synth/):
  * the 2-norms and max-norms of x, x_v and x_p;
  * x at 8192 indices drawn uniformly from 0..4N-1 (numpy default_rng(1911));
  * the projections g_k . x for 8 standard normal vectors g_k
    (default_rng(1000 + k), k = 0..7), which bound the whole-vector error
    through |g.(x - x_o)| <= |g| |x - x_o|;
  * the oracle's true relative residual and iteration counts, and the
    relative difference between its own 1e-8 solution and the 1e-12 one.

Run from the repository root (about ten minutes on eight cores):
    python tests/golden/make_fullsize_golden.py
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_box64x64x256_re2000_q4.json")
N_SAMPLES = 8192
N_PROJ = 8


def sample_indices(n):
    return np.sort(np.random.default_rng(1911).choice(n, N_SAMPLES, replace=False))


def projection_vector(k, n):
    return np.random.default_rng(1000 + k).standard_normal(n)


def main():
    spec = synth.large_mixed(64)
    d = synth.generate(spec)
    n, nv = 4 * d["n_nodes"], 3 * d["n_nodes"]
    o = oracle.Oracle(d)
    t0 = time.perf_counter()
    o.setup()
    t1 = time.perf_counter()
    o.set_options(rtol=1e-8)
    x8, info8, rc8 = o.solve(d["b"])
    t2 = time.perf_counter()
    o.set_options(rtol=1e-12)
    x, info, rc = o.solve(d["b"])
    t3 = time.perf_counter()
    assert rc == 0, "the oracle did not reach 1e-12"
    r = d["b"] - o.apply_full(x)
    rel_true = float(np.linalg.norm(r) / np.linalg.norm(d["b"]))
    idx = sample_indices(n)
    out = {
        "_source": "tests/golden/make_fullsize_golden.py: FP64 oracle nested solve (Algorithms 2-3 inside "
                   "FGMRES, Sec. 3) of synth.large_mixed(64) to delta^r = 1e-12, default inner options",
        "workload": spec.name, "unknowns": n,
        "rtol": 1e-12, "rel_res_true": rel_true,
        "iters": {"outer": info.outer_iters, "A": info.A_iters, "S": info.S_iters, "I": info.I_iters},
        "norm2": float(np.linalg.norm(x)), "norm2_v": float(np.linalg.norm(x[:nv])),
        "norm2_p": float(np.linalg.norm(x[nv:])),
        "norminf": float(np.abs(x).max()), "norminf_v": float(np.abs(x[:nv]).max()),
        "norminf_p": float(np.abs(x[nv:]).max()),
        "sample_seed": 1911, "idx": [int(i) for i in idx], "x": [float(v) for v in x[idx]],
        "proj_seeds": [1000 + k for k in range(N_PROJ)],
        "proj": [float(projection_vector(k, n) @ x) for k in range(N_PROJ)],
        "oracle_1e8": {"rel_res_true": info8.rel_res_true,
                       "rel_err_vs_1e12": float(np.linalg.norm(x8 - x) / np.linalg.norm(x)),
                       "iters": {"outer": info8.outer_iters, "A": info8.A_iters, "S": info8.S_iters,
                                 "I": info8.I_iters}},
        "oracle_setup_s": t1 - t0, "oracle_solve_1e8_s": t2 - t1, "oracle_solve_1e12_s": t3 - t2,
        "threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=0)
    print(json.dumps({k: v for k, v in out.items() if k not in ("idx", "x")}))


if __name__ == "__main__":
    main()
