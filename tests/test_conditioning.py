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
