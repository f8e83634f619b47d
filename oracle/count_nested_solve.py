"""Iteration counts of the oracle's FP64 nested solve of the 4,343,300-unknown
box (64x64x256 hexes, Re 2000, 4 outlets, default options), written to
profiles/nested_solve_counts.json.  The benchmark's CPU reference arm times a
bounded sample of oracle iterations and scales it by these counts.

Run from the repository root:  python oracle/count_nested_solve.py
(minutes to an hour of one CPU core)."""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    spec = synth.large_mixed(64)
    d = synth.generate(spec)
    o = oracle.Oracle(d)
    t0 = time.perf_counter()
    o.setup()
    t1 = time.perf_counter()
    x, info, rc = o.solve(d["b"])
    t2 = time.perf_counter()
    out = {
        "_source": "oracle/count_nested_solve.py: the oracle's FP64 nested solve of the 64x64x256 box (Re 2000, "
                   "4 outlets), outer tol 1e-8, default options; the CPU reference arm scales its per-iteration "
                   "time by these counts",
        "fp64": {"outer_iters": info.outer_iters, "A_iters": info.A_iters, "S_iters": info.S_iters,
                 "I_iters": info.I_iters},
        "oracle_status": rc, "rel_res_true": info.rel_res_true,
        "oracle_setup_s": t1 - t0, "oracle_solve_s": t2 - t1,
    }
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles",
                        "nested_solve_counts.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
