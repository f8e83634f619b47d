"""Conditioning of the tangent and what a relative residual says about the
relative error (Sec. 3.1 stopping rule: relative residual delta^r).

On the 8x8x8 tangent (2,916 unknowns) the 2-norm condition number of the
block system is taken by a dense SVD (LAPACK).  It is large (~1.8e7): the
smallest singular vectors are pressure modes, nearly constant over the
domain, which the outlet coupling fixes only weakly.  So the textbook bound
rel.err <= kappa * rel.res does not turn the 1e-8 residual bar into a 1e-6
error bar by itself; the measured error of the oracle's solution stays within
a small factor of its residual, which these tests pin against the dense LU
solution."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def tiny_svd():
    d = synth.generate(synth.tiny())
    F = oracle.dense_system(d)[4]
    U, s, Vt = np.linalg.svd(F)
    return d, F, s, Vt


def test_condition_number_of_the_tiny_tangent(tiny_svd):
    d, F, s, Vt = tiny_svd
    kappa = s[0] / s[-1]
    assert 1e6 < kappa < 1e9            # 1.84e7 measured (dense SVD)
    # the two smallest singular vectors live on the pressure unknowns
    nv = 3 * d["n_nodes"]
    for v in Vt[-2:]:
        assert np.linalg.norm(v[nv:]) ** 2 > 0.999
    # the 1-norm condition number from the explicit inverse is of the same order
    k1 = np.linalg.norm(F, 1) * np.linalg.norm(np.linalg.inv(F), 1)
    assert 0.1 * kappa < k1 < 100 * kappa


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_error_follows_the_residual(tiny_svd, rtol):
    """rel.err <= kappa rel.res always (textbook bound); on this tangent the
    error of the nested solve stays within 20x its residual, far inside that
    bound, so the 1e-8 residual bar gives errors well below 1e-6."""
    d, F, s, Vt = tiny_svd
    kappa = s[0] / s[-1]
    x_lu = np.linalg.solve(F, d["b"])
    o = oracle.Oracle(d, rtol=rtol)
    o.setup()
    x, info, rc = o.solve(d["b"])
    assert rc == 0
    res = np.linalg.norm(d["b"] - F @ x) / np.linalg.norm(d["b"])
    err = np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu)
    assert res <= rtol
    assert err <= kappa * res
    assert err <= 20.0 * res
    assert err <= 100.0 * rtol


# ---------------------------------------------------------------- mid size
# A box shaped like the benchmark workload, 12 x 12 x 48 hexes (33,124
# unknowns, Re 2000, four outlets with resistances 1e2-1e5): too large
# for a dense SVD, so the 1-norm condition number is estimated (Higham and
# Tisseur's block estimator on the sparse LU factors) and the oracle's
# solutions are compared with the direct solution.

def _sparse_system(d):
    """The block tangent [[A + sum_k r_k a^k a^kT, B], [C, D]] as a sparse
    matrix, assembled here from the blocks and the outlet vectors."""
    import scipy.sparse as sp
    N, rp, col = d["n_nodes"], d["rowptr"], d["col"]
    A = sp.bsr_matrix((d["A"], col, rp), shape=(3 * N, 3 * N))
    B = sp.bsr_matrix((d["B"].reshape(-1, 3, 1), col, rp), shape=(3 * N, N))
    C = sp.bsr_matrix((d["C"].reshape(-1, 1, 3), col, rp), shape=(N, 3 * N))
    D = sp.csr_matrix((d["D"], col, rp), shape=(N, N))
    optr, oidx, oval = d["out_ptr"], d["out_idx"], d["out_val"]
    k_of = np.repeat(np.arange(len(optr) - 1), np.diff(optr))
    U = sp.csr_matrix((oval, (oidx, k_of)), shape=(3 * N, len(optr) - 1))
    A = A + U @ sp.diags(d["r"]) @ U.T
    return sp.bmat([[A, B], [C, D]]).tocsc()


@pytest.fixture(scope="module")
def mid_lu():
    spla = pytest.importorskip("scipy.sparse.linalg")
    spec = synth.MeshSpec(12, 12, 48, Lz=4.0, Re=2000.0, seed=11, R=(1e2, 1e3, 1e4, 1e5),
                          name="box12x12x48_re2000_q4")
    d = synth.generate(spec)
    F = _sparse_system(d)
    return d, F, spla.splu(F)


def test_mid_size_assembly_is_the_oracles_operator(mid_lu):
    d, F, _ = mid_lu
    x = np.random.default_rng(0).standard_normal(4 * d["n_nodes"])
    yo = oracle.Oracle(d).apply_full(x)
    assert np.abs(F @ x - yo).max() <= 1e-13 * np.abs(yo).max()


def test_mid_size_condition_estimate(mid_lu):
    """kappa_1 of the mid-size tangent is beyond 1e8 (estimated 5.8e9): the
    bound rel.err <= kappa rel.res says nothing at the 1e-8 bar."""
    import scipy.sparse.linalg as spla
    d, F, lu = mid_lu
    inv = spla.LinearOperator(F.shape, matvec=lu.solve, rmatvec=lambda v: lu.solve(v, trans="T"), dtype=float)
    np.random.seed(3)   # the estimator's random starting columns
    kappa1 = spla.norm(F, 1) * spla.onenormest(inv)
    assert kappa1 > 1e8


@pytest.mark.parametrize("rtol", [1e-6, 1e-8])
def test_mid_size_error_follows_the_residual(mid_lu, rtol):
    """The oracle's nested solve against the direct solution: the error stays
    within a small factor of the true relative residual for the whole vector
    and for the velocity and pressure parts separately (measured 0.1-1.1x)."""
    d, F, lu = mid_lu
    b = d["b"]
    x_lu = lu.solve(b)
    o = oracle.Oracle(d, rtol=rtol)
    o.setup()
    x, info, rc = o.solve(b)
    assert rc == 0
    res = np.linalg.norm(b - F @ x) / np.linalg.norm(b)
    assert res <= rtol
    nv = 3 * d["n_nodes"]
    for sl in (slice(None), slice(0, nv), slice(nv, None)):
        err = np.linalg.norm(x[sl] - x_lu[sl]) / np.linalg.norm(x_lu[sl])
        assert err <= 20.0 * res
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 100.0 * rtol
