"""The oracle's results do not depend on its thread count: every parallel
loop has independent iterations and every sum keeps one fixed order (inner
products summed per run of 4096 entries, the runs in ascending order).  A
nested solve on a box large enough for the parallel loops to run (more than
32768 entries per vector) is compared bit for bit at 1 and 4 threads."""
import numpy as np

import oracle
import synth


def test_nested_solve_is_bitwise_equal_at_one_and_four_threads():
    spec = synth.MeshSpec(16, 16, 64, Lz=4.0, Re=500.0, seed=9, R=(1e2, 1e3, 1e4, 1e5), name="box16x16x64_q4")
    d = synth.generate(spec)
    assert 3 * d["n_nodes"] > 32768
    before = oracle.threads()
    try:
        out = []
        for nt in (1, 4):
            assert oracle.threads(nt) == nt
            o = oracle.Oracle(d)
            x, info, _ = o.solve(d["b"])
            out.append((x, (info.outer_iters, info.A_iters, info.S_iters, info.I_iters), info.rel_res_true))
        (x1, c1, r1), (x4, c4, r4) = out
        assert c1 == c4
        assert r1 == r4
        assert np.array_equal(x1, x4)
    finally:
        oracle.threads(before)
