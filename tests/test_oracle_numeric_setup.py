"""Numeric re-setup of the oracle (or_setup_numeric): after new values on the
same patterns (a later Newton tangent, Sec. 2.5) the preconditioner is
rebuilt from the new values on the aggregates of the last full setup.  Pins:
unchanged values reproduce the full setup bit for bit; with changed values
the aggregates are the kept ones, every coarse operator is the Galerkin
triple product P^T A P of the new level above it (dense, with the indicator
P of the kept map), S_hat is D - C diag(A)^{-1} B of the new blocks, and the
nested solve still solves the new system (the outer FGMRES takes any
preconditioner, Sec. 3)."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny():
    d = synth.generate(synth.tiny())
    return d


def _levels(o):
    return o.amg_levels(0), o.amg_levels(1)


def test_unchanged_values_reproduce_the_full_setup(tiny):
    d = tiny
    o = oracle.Oracle(d)
    o.setup()
    x0, i0, _ = o.solve(d["b"])
    before = _levels(o)
    o.setup_numeric()
    x1, i1, _ = o.solve(d["b"])
    after = _levels(o)
    for h0, h1 in zip(before, after):
        assert len(h0) == len(h1)
        for a, b in zip(h0, h1):
            assert np.array_equal(a["rowptr"], b["rowptr"]) and np.array_equal(a["col"], b["col"])
            assert np.array_equal(a["val"], b["val"]) and a["rho"] == b["rho"]
    assert np.array_equal(x0, x1)
    assert (i0.outer_iters, i0.A_iters, i0.S_iters, i0.I_iters) == (i1.outer_iters, i1.A_iters, i1.S_iters, i1.I_iters)


def test_setup_numeric_before_setup_is_refused(tiny):
    o = oracle.Oracle(tiny)
    with pytest.raises(RuntimeError):
        o.setup_numeric()


def _perturbed(d, seed=4):
    rng = np.random.default_rng(seed)
    out = {}
    for k in ("A", "B", "C", "D"):
        v = np.asarray(d[k], dtype=np.float64)
        out[k] = v * rng.uniform(0.9, 1.1, v.shape)
    return out


def test_changed_values_keep_the_aggregates_and_rebuild_the_operators(tiny):
    d = tiny
    o = oracle.Oracle(d)
    o.setup()
    old = _levels(o)
    new = _perturbed(d)
    o.set_values(new["A"], new["B"], new["C"], new["D"])
    o.setup_numeric()
    cur = _levels(o)
    d2 = dict(d, **new)
    A, B, C, D, F = oracle.dense_system(d2)
    for which, bs in ((0, 3), (1, 1)):
        Lo, L = old[which], cur[which]
        assert len(Lo) == len(L)
        for l in range(len(L) - 1):
            assert np.array_equal(Lo[l]["agg"], L[l]["agg"])          # the kept map
            n0, n1 = len(L[l]["rowptr"]) - 1, len(L[l + 1]["rowptr"]) - 1
            A0 = oracle.dense_block(L[l]["rowptr"], L[l]["col"], L[l]["val"], bs, bs, n0, n0)
            A1 = oracle.dense_block(L[l + 1]["rowptr"], L[l + 1]["col"], L[l + 1]["val"], bs, bs, n1, n1)
            P = np.zeros((n0 * bs, n1 * bs))
            for i, I in enumerate(L[l]["agg"]):
                if I >= 0:
                    P[i * bs:(i + 1) * bs, I * bs:(I + 1) * bs] = np.eye(bs)
            assert np.abs(P.T @ A0 @ P - A1).max() <= 1e-13 * np.abs(A1).max()
    # level 0 of AMG(A) holds the new sparse A (no rank-one term), AMG(S_hat) the new S_hat
    N = d["n_nodes"]
    L0 = cur[0][0]
    Asp = oracle.dense_block(L0["rowptr"], L0["col"], L0["val"], 3, 3, N, N)
    Anew = oracle.dense_block(d["rowptr"], d["col"], new["A"].reshape(-1, 3, 3), 3, 3, N, N)
    assert np.array_equal(Asp, Anew)
    rp, ci, v = o.shat()
    Sh = oracle.dense_block(rp, ci, v, 1, 1, N, N)
    ref = D - C @ np.diag(1.0 / np.diag(A)) @ B
    assert np.abs(Sh - ref).max() <= 1e-13 * np.abs(ref).max()
    S0 = cur[1][0]
    assert np.array_equal(oracle.dense_block(S0["rowptr"], S0["col"], S0["val"], 1, 1, N, N), Sh)
    # the nested solve with the re-set-up preconditioner solves the new system
    o.set_options(rtol=1e-12)
    x, info, rc = o.solve(d["b"])
    assert rc == 0
    xd = np.linalg.solve(F, d["b"])
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
