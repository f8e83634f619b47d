"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a dense
textbook computation (numpy/LAPACK), a closed form, an invariant, or a
hand-derived special case.  Citations are to the paper's sections/algorithms.
"""
import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tiny():
    d = synth.generate(synth.tiny())
    dense = oracle.dense_system(d)
    return d, dense


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_default_options_follow_paper():
    """delta^a = 1e-50 and m = m_A = m_S = n_max = 200 (Sec. 3.1, last paragraphs)."""
    with open(os.path.join(GOLDEN, "paper_solver_settings.json")) as f:
        g = json.load(f)
    o = oracle.default_options()
    assert o.atol == g["delta_a"]
    assert o.m == o.m_A == o.m_S == g["m"]
    assert o.nmax == o.nmax_A == o.nmax_S == g["n_max"]


def test_apply_blocks_match_dense(tiny):
    """A = A_sp + sum_k r_k a^k a^kT (Sec. 2.5, K term) and the full block product."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    rng = np.random.default_rng(1)
    x = rng.standard_normal(4 * d["n_nodes"])
    nv = 3 * d["n_nodes"]
    assert _rel(o.apply_A(x[:nv]), A @ x[:nv]) < 1e-14
    assert _rel(o.apply_B(x[nv:]), B @ x[nv:]) < 1e-14
    assert _rel(o.apply_C(x[:nv]), C @ x[:nv]) < 1e-14
    assert _rel(o.apply_D(x[nv:]), D @ x[nv:]) < 1e-14
    assert _rel(o.apply_full(x), F @ x) < 1e-14


def test_diag_A_includes_rank_one_terms(tiny):
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    assert np.allclose(o.diag_A(), np.diag(A), rtol=1e-15, atol=0)


def test_nested_solve_matches_dense_lu(tiny):
    """x = A^{-1} b: FGMRES + P_SCR (Sec. 3, Algorithm 3) against LAPACK LU."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    o.setup()
    x, info, rc = o.solve(d["b"])
    assert rc == 0
    x_lu = np.linalg.solve(F, d["b"])
    assert np.linalg.norm(d["b"] - F @ x) / np.linalg.norm(d["b"]) <= 1e-8
    assert info.rel_res_true <= 1e-8
    assert _rel(x, x_lu) <= 1e-6
    assert 1 <= info.outer_iters <= 20
    # tighter outer tolerance drives the error further down
    o.set_options(rtol=1e-12)
    x2, info2, rc2 = o.solve(d["b"])
    assert rc2 == 0 and _rel(x2, x_lu) <= 1e-9


def test_exact_inner_solves_give_one_outer_iteration(tiny):
    """With exact A^{-1} and S^{-1}, Algorithm 3 is the exact inverse of the
    block LDU factorisation (Sec. 3.1), so FGMRES stops after one iteration."""
    d, _ = tiny
    o = oracle.Oracle(d, rtol_A=1e-13, rtol_S=1e-13, rtol_I=1e-13)
    o.setup()
    x, info, rc = o.solve(d["b"])
    assert rc == 0 and info.outer_iters == 1


def test_block_triangular_preconditioner_gives_two_iterations(tiny):
    """P = [[A, B], [0, S]] gives A P^{-1} = [[I, 0], [C A^{-1}, I]] (from the
    block LDU factorisation, Sec. 3.1): (A P^{-1} - I)^2 = 0, so GMRES needs
    exactly two iterations with exact inner solves."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d, rtol_A=1e-13, rtol_S=1e-13, rtol_I=1e-13, variant=1)
    o.setup()
    x, info, rc = o.solve(d["b"])
    assert rc == 0 and info.outer_iters == 2
    # the closed form itself, densely
    S = D - C @ np.linalg.solve(A, B)
    N = d["n_nodes"]
    P = np.block([[A, B], [np.zeros((N, 3 * N)), S]])
    E = F @ np.linalg.inv(P) - np.eye(4 * N)
    assert np.abs(E @ E).max() <= 1e-9 * max(1.0, np.abs(E).max())


def test_matrix_free_schur_matches_dense(tiny):
    """Algorithm 2 with an exact inner solve equals (D - C A^{-1} B) x."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d, rtol_I=1e-14)
    o.setup()
    S = D - C @ np.linalg.solve(A, B)
    rng = np.random.default_rng(2)
    for _ in range(3):
        xp = rng.standard_normal(d["n_nodes"])
        assert _rel(o.apply_S(xp), S @ xp) <= 1e-10


def test_pscr_with_exact_solves_is_inverse(tiny):
    """Algorithm 3 with exact intermediate/inner solves returns A^{-1} s."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d, rtol_A=1e-14, rtol_S=1e-14, rtol_I=1e-14)
    o.setup()
    s = np.random.default_rng(3).standard_normal(4 * d["n_nodes"])
    y = o.apply_pscr(s)
    assert _rel(F @ y, s) <= 1e-9


def test_shat_matches_dense_formula(tiny):
    """S_hat = D - C diag(A)^{-1} B with the scalar diagonal of A (Sec. 3.1)."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    o.setup()
    rp, ci, v = o.shat()
    N = d["n_nodes"]
    Sh = oracle.dense_block(rp, ci, v, 1, 1, N, N)
    ref = D - C @ np.diag(1.0 / np.diag(A)) @ B
    assert np.abs(Sh - ref).max() <= 1e-13 * np.abs(ref).max()
    # pattern: sorted rows, distance-2 graph of the node pattern
    for i in range(N):
        assert np.all(np.diff(ci[rp[i]:rp[i + 1]]) > 0)


def _path(n, w=1.0):
    rp, ci, v = [0], [], []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                ci.append(j)
                v.append(2.0 if i == j else -w)
        rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def test_aggregation_path_graph_closed_form():
    """Handshake matching on a uniform path: pass 1 pairs (0,1),(2,3),...
    (ties go to the smaller index), three passes give blocks of 8 consecutive
    nodes (golden fixture written by hand from the matching rule)."""
    with open(os.path.join(GOLDEN, "aggregation_path16.json")) as f:
        g = json.load(f)
    rp, ci, v = _path(16)
    nc, agg = oracle.aggregate(rp, ci, v, 1, 0.0064)
    assert nc == g["n_aggregates"]
    assert agg.tolist() == g["agg"]


def test_aggregation_isolated_and_weak():
    # diagonal matrix: every node isolated -> no aggregate
    n = 10
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    nc, agg = oracle.aggregate(rp, ci, np.ones(n), 1, 0.0064)
    assert nc == 0 and np.all(agg == -1)
    # weak couplings: sigma = w^2 / (2*2) = 0.0025 < theta -> isolated
    rp, ci, v = _path(8, w=0.1)
    nc, agg = oracle.aggregate(rp, ci, v, 1, 0.0064)
    assert nc == 0
    # strong couplings, then one decoupled node in the middle
    rp, ci, v = _path(8)
    v = v.copy()
    for i in (3, 4):
        for e in range(rp[i], rp[i + 1]):
            if (i == 3 and ci[e] == 4) or (i == 4 and ci[e] == 3):
                v[e] = 0.0
    nc, agg = oracle.aggregate(rp, ci, v, 1, 0.0064)
    assert set(agg[:4]) == {0} and set(agg[4:]) == {1}


def test_aggregation_invariants_on_tangent(tiny):
    d, _ = tiny
    o = oracle.Oracle(d)
    o.setup()
    for which in (0, 1):
        levels = o.amg_levels(which)
        for l in levels[:-1]:
            agg = l["agg"]
            nc = len(levels[levels.index(l) + 1]["rowptr"]) - 1
            used = agg[agg >= 0]
            sizes = np.bincount(used, minlength=nc)
            assert sizes.min() >= 1 and sizes.max() <= 8
            # numbering by smallest member
            first = np.array([np.min(np.nonzero(agg == I)[0]) for I in range(nc)])
            assert np.all(np.diff(first) > 0)


def test_galerkin_matches_dense_triple_product(tiny):
    d, _ = tiny
    o = oracle.Oracle(d)
    o.setup()
    for which, bs in ((0, 3), (1, 1)):
        L = o.amg_levels(which)
        n0 = len(L[0]["rowptr"]) - 1
        n1 = len(L[1]["rowptr"]) - 1
        A0 = oracle.dense_block(L[0]["rowptr"], L[0]["col"], L[0]["val"], bs, bs, n0, n0)
        A1 = oracle.dense_block(L[1]["rowptr"], L[1]["col"], L[1]["val"], bs, bs, n1, n1)
        P = np.zeros((n0 * bs, n1 * bs))
        for i, I in enumerate(L[0]["agg"]):
            if I >= 0:
                P[i * bs:(i + 1) * bs, I * bs:(I + 1) * bs] = np.eye(bs)
        assert np.abs(P.T @ A0 @ P - A1).max() <= 1e-14 * np.abs(A1).max()


def _cheb_closed_form(Ad, Dinv, rho, k, b, lodiv=10.0):
    """x = (I - q(D^{-1}A)) A^{-1} b, q(t) = T_k((theta - t)/delta) / T_k(theta/delta),
    interval [rho / lodiv, rho] (10 on AMG(A), 3 on AMG(S_hat))."""
    lmax, lmin = rho, rho / lodiv
    th, de = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    n = Ad.shape[0]
    X = (th * np.eye(n) - Dinv @ Ad) / de
    T0, T1 = np.eye(n), X
    for _ in range(k - 1):
        T0, T1 = T1, 2 * X @ T1 - T0
    s = th / de
    t0, t1 = 1.0, s
    for _ in range(k - 1):
        t0, t1 = t1, 2 * s * t1 - t0
    Q = (T1 if k >= 1 else T0) / (t1 if k >= 1 else t0)
    if b is None:                                       # the smoother as a matrix
        return (np.eye(n) - Q) @ np.linalg.inv(Ad)
    return (np.eye(n) - Q) @ np.linalg.solve(Ad, b)


def _spectral_norm(M):
    """||M||_2 from the largest eigenvalue of M^T M (LAPACK).  Every Ritz value
    of M (an eigenvalue of V^T M V, V orthonormal) lies in M's field of
    values, so its magnitude is at most the numerical radius <= ||M||_2."""
    return float(np.sqrt(np.linalg.eigvalsh(M.T @ M)[-1]))


def test_chebyshev_bound_covers_the_spectrum(tiny):
    """The Chebyshev interval's upper end lies above every eigenvalue
    magnitude of D_b^{-1} A (dense eigenvalues, LAPACK) on every smoothed
    level, and below the bounds its definition gives: on AMG(A) 1.1 x the
    largest Ritz value magnitude of 20 Arnoldi steps, capped by Gershgorin,
    hence at most 1.1 x the spectral norm ||D_b^{-1} A||_2 (LAPACK);
    on AMG(S_hat) exactly the Gershgorin bound (largest absolute row sum)."""
    d, _ = tiny
    o = oracle.Oracle(d)
    o.setup()
    for which, bs in ((0, 3), (1, 1)):
        L = o.amg_levels(which)
        for lev in L[:-1]:
            n = len(lev["rowptr"]) - 1
            Ad = oracle.dense_block(lev["rowptr"], lev["col"], lev["val"], bs, bs, n, n)
            Db = np.zeros_like(Ad)
            for i in range(n):
                Db[bs * i:bs * i + bs, bs * i:bs * i + bs] = Ad[bs * i:bs * i + bs, bs * i:bs * i + bs]
            DA = np.linalg.inv(Db) @ Ad
            lam = np.abs(np.linalg.eigvals(DA)).max()
            assert lev["rho"] >= lam
            gers = np.abs(DA).sum(axis=1).max()
            assert lev["rho"] <= gers * (1 + 1e-14)
            if which == 0:
                # 1.1 x the largest |Ritz value| (capped by Gershgorin): at most 1.1 ||DA||_2
                assert lev["rho"] <= 1.1 * _spectral_norm(DA) * (1 + 1e-12)
            else:
                assert np.isclose(lev["rho"], gers, rtol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_chebyshev_matches_closed_form(tiny, k):
    """Chebyshev smoother (Saad, Alg. 12.1) vs its residual polynomial."""
    d, _ = tiny
    o = oracle.Oracle(d)
    o.setup()
    L = o.amg_levels(0)
    n = len(L[0]["rowptr"]) - 1
    Ad = oracle.dense_block(L[0]["rowptr"], L[0]["col"], L[0]["val"], 3, 3, n, n)
    Db = np.zeros_like(Ad)
    for i in range(n):
        Db[3 * i:3 * i + 3, 3 * i:3 * i + 3] = Ad[3 * i:3 * i + 3, 3 * i:3 * i + 3]
    Dinv = np.linalg.inv(Db)
    b = np.random.default_rng(4).standard_normal(3 * n)
    x = oracle.chebyshev(L[0]["rowptr"], L[0]["col"], L[0]["val"], 3, L[0]["rho"], k, b)
    assert _rel(x, _cheb_closed_form(Ad, Dinv, L[0]["rho"], k, b)) <= 1e-10


def test_two_level_cycle_is_coarse_projection(tiny):
    """With no smoothing and an exact coarse solve, the cycle is P (P^T A P)^{-1} P^T."""
    d, _ = tiny
    o = oracle.Oracle(d, amg_max_levels=2, cheb_degree=0, amg_coarse_max=10)
    o.setup()
    L = o.amg_levels(0)
    assert len(L) == 2
    n0, n1 = len(L[0]["rowptr"]) - 1, len(L[1]["rowptr"]) - 1
    A0 = oracle.dense_block(L[0]["rowptr"], L[0]["col"], L[0]["val"], 3, 3, n0, n0)
    P = np.zeros((3 * n0, 3 * n1))
    for i, I in enumerate(L[0]["agg"]):
        if I >= 0:
            P[3 * i:3 * i + 3, 3 * I:3 * I + 3] = np.eye(3)
    b = np.random.default_rng(5).standard_normal(3 * n0)
    ref = P @ np.linalg.solve(P.T @ A0 @ P, P.T @ b)
    assert _rel(o.vcycle(0, b), ref) <= 1e-12


@pytest.mark.parametrize("deg", [1, 2])
def test_vcycle_error_propagation(tiny, deg):
    """Two-level V(1,1): E = (I - S A)(I - P A_c^{-1} P^T A)(I - S A), M^{-1} = (I - E) A^{-1},
    S the Chebyshev smoother of degree deg (1: the cycle of the inner A-solves of Algorithm 2)."""
    d, _ = tiny
    o = oracle.Oracle(d, amg_max_levels=2, amg_coarse_max=10, cheb_degree=deg)
    o.setup()
    L = o.amg_levels(0)
    n0, n1 = len(L[0]["rowptr"]) - 1, len(L[1]["rowptr"]) - 1
    A0 = oracle.dense_block(L[0]["rowptr"], L[0]["col"], L[0]["val"], 3, 3, n0, n0)
    Db = np.zeros_like(A0)
    for i in range(n0):
        Db[3 * i:3 * i + 3, 3 * i:3 * i + 3] = A0[3 * i:3 * i + 3, 3 * i:3 * i + 3]
    Dinv = np.linalg.inv(Db)
    n = 3 * n0
    # smoother as a matrix: x = S b from x0 = 0
    Sm = _cheb_closed_form(A0, Dinv, L[0]["rho"], deg, None)
    P = np.zeros((n, 3 * n1))
    for i, I in enumerate(L[0]["agg"]):
        if I >= 0:
            P[3 * i:3 * i + 3, 3 * I:3 * I + 3] = np.eye(3)
    CC = np.eye(n) - P @ np.linalg.solve(P.T @ A0 @ P, P.T @ A0)
    E = (np.eye(n) - Sm @ A0) @ CC @ (np.eye(n) - Sm @ A0)
    b = np.random.default_rng(6).standard_normal(n)
    ref = (np.eye(n) - E) @ np.linalg.solve(A0, b)
    assert _rel(o.vcycle(0, b), ref) <= 1e-9
    # and it contracts: the preconditioner is useful
    assert np.abs(np.linalg.eigvals(E)).max() < 0.9


def test_gmres_iterate_is_krylov_minimiser(tiny):
    """GMRES (Saad & Schultz) iterate k minimises ||b - A x|| over K_k(A, b):
    brute force by dense least squares on an orthonormalised Krylov basis."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    b = np.random.default_rng(7).standard_normal(3 * d["n_nodes"])
    for k in (1, 3, 6):
        x, its, rel, rc = o.gmres_A(b, 1e-30, 200, k, 0)
        assert its == k
        K = np.empty((len(b), k))
        v = b / np.linalg.norm(b)
        for j in range(k):
            K[:, j] = v
            v = A @ v
            for i in range(j + 1):          # re-orthonormalise for stability
                v -= (K[:, i] @ v) * K[:, i]
            v /= np.linalg.norm(v)
        Q, _ = np.linalg.qr(K)
        y, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
        x_ref = Q @ y
        assert _rel(x, x_ref) <= 1e-8
        # Givens residual estimate equals the true residual
        assert abs(rel - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) <= 1e-10


def test_restarted_gmres_is_cyclewise_minimiser(tiny):
    """GMRES(m) restarted (Saad & Schultz): each cycle of m steps minimises
    ||b - A x|| over x_c + K_m(A, b - A x_c) from the cycle's start x_c;
    brute force by dense least squares, cycle after cycle."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    b = np.random.default_rng(17).standard_normal(3 * d["n_nodes"])
    for m in (1, 2, 3):
        x, its, rel, rc = o.gmres_A(b, 1e-30, m, 6, 0)
        assert its == 6
        xr = np.zeros_like(b)
        for _ in range(6 // m):
            r = b - A @ xr
            K = np.empty((len(b), m))
            v = r / np.linalg.norm(r)
            for j in range(m):
                K[:, j] = v
                v = A @ v
                for i in range(j + 1):
                    v -= (K[:, i] @ v) * K[:, i]
                v /= np.linalg.norm(v)
            Q, _ = np.linalg.qr(K)
            y, *_ = np.linalg.lstsq(A @ Q, r, rcond=None)
            xr = xr + Q @ y
        assert _rel(x, xr) <= 1e-8
        assert abs(rel - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) <= 1e-10


@pytest.fixture(scope="module")
def tiny4():
    spec = synth.MeshSpec(8, 8, 8, Re=100.0, seed=0, R=(1e2, 1e3, 3e3, 1e4), name="cube8_re100_q4")
    d = synth.generate(spec)
    return d, oracle.dense_system(d)


def test_adjoint_matches_dense_and_finite_differences(tiny4):
    """lambda = A^{-T} g, dL/dr_k = -(lambda_v . a^k)(a^k . x_v) because
    dA/dr_k = [[a^k a^kT, 0], [0, 0]] (Sec. 2.5, K term); L = sum_k (a^k.u - q_k)^2.
    Four outlets: with one outlet and a prescribed inflow the outlet flux is
    fixed by continuity and dL/dr vanishes."""
    d, (A, B, C, D, F) = tiny4
    N = d["n_nodes"]
    nv = 3 * N
    n_out = len(d["out_ptr"]) - 1
    av = []
    for k in range(n_out):
        v = np.zeros(nv)
        v[d["out_idx"][d["out_ptr"][k]:d["out_ptr"][k + 1]]] = d["out_val"][d["out_ptr"][k]:d["out_ptr"][k + 1]]
        av.append(v)
    x = np.linalg.solve(F, d["b"])
    flux = np.array([a @ x[:nv] for a in av])
    q = (2 * synth.uniforms(44, n_out) - 1) * np.abs(flux).max()

    def loss(rv):
        dd = dict(d)
        dd["r"] = np.asarray(rv)
        *_, Fr = oracle.dense_system(dd)
        xr = np.linalg.solve(Fr, d["b"])
        return sum((av[k] @ xr[:nv] - q[k]) ** 2 for k in range(n_out))

    g = np.zeros(4 * N)
    for k in range(n_out):
        g[:nv] += 2 * (av[k] @ x[:nv] - q[k]) * av[k]
    lam, dLdr, info = oracle.adjoint(d, g, x, rtol=1e-12)
    lam_ref = np.linalg.solve(F.T, g)
    assert _rel(lam, lam_ref) <= 1e-6
    for k in range(n_out):
        e = np.zeros(n_out)
        e[k] = 1e-6 * d["r"][k]
        fd = (loss(d["r"] + e) - loss(d["r"] - e)) / (2 * e[k])
        assert abs(dLdr[k] - fd) <= 1e-5 * abs(fd)


def test_kcycle_is_two_step_minimal_residual(tiny):
    """K-cycle on AMG(S_hat): on level 1 the coarse correction is the element of
    span{z1, z2} with the least residual (two GCR steps), z1 = T b and
    z2 = T r1, T the two-grid cycle of level 1 and r1 the residual after the
    best multiple of z1.  Checked by dense least squares on a 3-level
    hierarchy, composed with the level-0 smoothing and transfers."""
    import scipy.linalg as sla
    d, _ = tiny
    o = oracle.Oracle(d, amg_max_levels=3, amg_coarse_max=10, amg_cycle=1, cheb_degree_S=2)
    o.setup()
    L = o.amg_levels(1)
    assert len(L) == 3
    mats, Ps = [], []
    for l in range(3):
        n = len(L[l]["rowptr"]) - 1
        mats.append(oracle.dense_block(L[l]["rowptr"], L[l]["col"], L[l]["val"], 1, 1, n, n))
    for l in range(2):
        n, nc = mats[l].shape[0], mats[l + 1].shape[0]
        P = np.zeros((n, nc))
        for i, I in enumerate(L[l]["agg"]):
            if I >= 0:
                P[i, I] = 1.0
        Ps.append(P)

    def smoother(l):
        A = mats[l]
        Dinv = np.diag(1.0 / np.diag(A))
        return _cheb_closed_form(A, Dinv, L[l]["rho"], 2, None, lodiv=3.0)

    def two_grid(l, b):
        A, P, S = mats[l], Ps[l], smoother(l)
        n = A.shape[0]
        CC = np.eye(n) - P @ np.linalg.solve(P.T @ A @ P, P.T @ A)
        E = (np.eye(n) - S @ A) @ CC @ (np.eye(n) - S @ A)
        return (np.eye(n) - E) @ np.linalg.solve(A, b)

    def kcycle(b):
        A1 = mats[1]
        z1 = two_grid(1, b)
        w1 = A1 @ z1
        a1 = sla.lstsq(w1[:, None], b)[0][0]
        z2 = two_grid(1, b - a1 * w1)
        Z = np.column_stack([z1, z2])
        y = sla.lstsq(A1 @ Z, b)[0]
        return Z @ y

    A0, P0, S0 = mats[0], Ps[0], smoother(0)
    b = np.random.default_rng(9).standard_normal(A0.shape[0])
    x = S0 @ b
    x = x + P0 @ kcycle(P0.T @ (b - A0 @ x))
    x = x + S0 @ (b - A0 @ x)
    assert _rel(o.vcycle(1, b), x) <= 1e-9


def test_simple_preconditioner_identity(tiny):
    """SIMPLE (Sec. 3.2): with exact solves its inverse is the inverse of
    [[A, A diag(A)^{-1} B], [C, D]] (the product of its three factors)."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d, variant=2, rtol_A=1e-14, rtol_S=1e-14)
    o.setup()
    N = d["n_nodes"]
    P = np.block([[A, A @ np.diag(1.0 / np.diag(A)) @ B], [C, D]])
    y = np.random.default_rng(12).standard_normal(4 * N)
    assert _rel(o.apply_pscr(P @ y), y) <= 1e-8
    # and the nested FGMRES with it still solves the system
    o.set_options(rtol_A=1e-3, rtol_S=1e-2)
    x, info, rc = o.solve(d["b"])
    assert rc == 0 and np.linalg.norm(d["b"] - F @ x) <= 1e-8 * np.linalg.norm(d["b"])


# ------------------------------------------------------------ RCR outlets
def _rcr_exact(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, T):
    """Closed form of one step of dPi/dt = -Pi/tau + Q(t)/C (tau = Rd C) with
    Q linear on [0, T]: Pi(T) = Pi_n e + (Q_n/C)(I0 - I1) + (Q_np1/C) I1,
    e = exp(-T/tau), I0 = tau (1 - e), I1 = tau - tau^2 (1 - e)/T; and
    dP/dQ_np1 = Rp + I1/C."""
    tau = Rd * C
    e = np.exp(-T / tau)
    I0 = tau * (1.0 - e)
    I1 = tau - tau * tau * (1.0 - e) / T
    Pi = Pi_n * e + Q_n / C * (I0 - I1) + Q_np1 / C * I1
    return Rp * Q_np1 + Pi + Pd, Pi, Rp + I1 / C


def test_rcr_step_fourth_order_to_the_exact_solution():
    """Algorithm 1 is a fourth-order Runge-Kutta scheme: against the closed
    form of the linear RCR ODE the error falls by ~2^4 per halving of h."""
    Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, T = 120.0, 1e-3, 1.0, 3.0, 5.0, 0.4, 0.9, 1e-3   # tau = T
    Pex, Piex, _ = _rcr_exact(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, T)
    errs = []
    for nts in (4, 8, 16, 32):   # h / tau = 1/4 .. 1/32 (asymptotic range)
        P, Pi, _ = oracle.rcr_step([Rp], [C], [Rd], [Pd], [Pi_n], [Q_n], [Q_np1], T, nts)
        assert abs(P[0] - Rp * Q_np1 - Pi[0] - Pd) <= 1e-12 * abs(P[0])
        errs.append(abs(Pi[0] - Piex))
    for a, b in zip(errs, errs[1:]):
        assert 15.0 <= a / b <= 19.0
    P, _, _ = oracle.rcr_step([Rp], [C], [Rd], [Pd], [Pi_n], [Q_n], [Q_np1], T, 64)
    assert abs(P[0] - Pex) <= 1e-10 * abs(Pex)


def test_rcr_stiffness_is_the_derivative_of_the_step():
    """The model is affine in Q_{n+1}, so the difference quotient of Sec. 2.5
    equals dP/dQ_{n+1} of the RK4 map for any eps, and tends to the exact
    Rp + I1/C as h -> 0."""
    rng = np.random.default_rng(31)
    n = 50
    Rp = 10 ** rng.uniform(1, 3, n); C = 10 ** rng.uniform(-5, -3, n); Rd = 10 ** rng.uniform(2, 4, n)
    Pd = rng.uniform(0, 10, n); Pi_n = rng.uniform(0, 100, n); Q_n = rng.uniform(-1, 1, n); Q_np1 = rng.uniform(-1, 1, n)
    T = 1e-3
    P, _, m = oracle.rcr_step(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, T, 64)
    _, _, m_big = oracle.rcr_step(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, T, 64, eps_abs=1e-2, eps_rel=0.0)
    exact = np.array([_rcr_exact(*a, T)[2] for a in zip(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1)])
    # a wide step: only the RK4 truncation (h / tau <= 0.013 here) is left
    assert np.max(np.abs(m_big - exact) / exact) <= 1e-9
    # the paper's step eps = max(1e-8, 1e-5 |Q|): plus the rounding of P over eps
    eps = np.maximum(1e-8, 1e-5 * np.abs(Q_np1))
    bound = 16 * np.finfo(float).eps * (np.abs(P) + np.abs(Rp * eps)) / eps + 1e-9 * exact
    assert np.all(np.abs(m - exact) <= bound)


def test_rcr_fixed_point_and_resistance_limit():
    """At the steady state Pi = Rd Q with constant Q nothing moves:
    P = (Rp + Rd) Q + Pd.  As C -> 0+ the RCR model reduces to a resistance
    Rp + Rd (Sec. 2.1), so m^k -> Rp + Rd."""
    Rp, Rd, Q, Pd = 200.0, 1800.0, 0.3, 7.0
    P, Pi, _ = oracle.rcr_step([Rp], [1e-3], [Rd], [Pd], [Rd * Q], [Q], [Q], 1e-3, 5)
    assert abs(P[0] - ((Rp + Rd) * Q + Pd)) <= 1e-13 * abs(P[0])
    assert abs(Pi[0] - Rd * Q) <= 1e-13 * Rd * Q
    # tau = 1e-6 s: h = dt / 4000 keeps explicit RK4 stable (h / tau = 0.25)
    _, _, m = oracle.rcr_step([Rp], [1e-9], [1000.0], [0.0], [0.0], [0.1], [0.2], 1e-3, 4000)
    assert abs(m[0] - (Rp + 1000.0)) <= 2e-3 * (Rp + 1000.0)


def test_many_outlet_patches_cover_the_outlet_face():
    """The many-outlet split (772 patches of consecutive outlet triangles,
    the patient-model outlet count of Sec. 4) partitions the outlet face:
    every patch is non-empty and the patch vectors sum to the whole-face
    outlet vector a = int N_A n dGamma."""
    many = synth.MeshSpec(32, 32, 16, R=tuple([1e3] * 772), name="box32_o772")
    one = synth.MeshSpec(32, 32, 16, R=(1e3,), name="box32_o1")
    ptr, idx, val = synth.outlets(many)
    assert np.all(np.diff(ptr) > 0)
    tot = np.zeros(3 * many.n_nodes)
    np.add.at(tot, idx, val)
    p1, i1, v1 = synth.outlets(one)
    whole = np.zeros(3 * one.n_nodes)
    whole[i1] = v1
    assert np.max(np.abs(tot - whole)) <= 1e-15 * np.max(np.abs(whole)) * 8
    # sparse outlet vectors equal the dense ones assembled with the tangent
    dense = synth.outlets_dense(synth.large_mixed(8))
    p4, i4, v4 = synth.outlets(synth.large_mixed(8))
    for k in range(4):
        nz = np.nonzero(dense[k])[0]
        assert np.array_equal(nz, i4[p4[k]:p4[k + 1]]) and np.array_equal(dense[k][nz], v4[p4[k]:p4[k + 1]])


def test_solve_without_explicit_setup_builds_the_hierarchies(tiny):
    """The oracle's solves need the AMG hierarchies; a solve called before
    setup() builds them instead of reading unbuilt data."""
    d, (A, B, C, D, F) = tiny
    o = oracle.Oracle(d)
    x, info, rc = o.solve(d["b"])
    assert rc == 0 and np.linalg.norm(d["b"] - F @ x) <= 1e-8 * np.linalg.norm(d["b"])


def test_schur_apply_inner_solve_uses_its_own_cycle_degree(tiny):
    """Algorithm 2's inner A-solve (line 3, tolerance rtol_I) is preconditioned
    by the AMG(A) cycle of degree cheb_degree_I, every other A-solve by that of
    cheb_degree: the S-apply equals D x_p - C y with y from an A-solve whose
    context has cheb_degree = cheb_degree_I, bit for bit, and differs from the
    one with the other degree."""
    d, _ = tiny
    xp = np.random.default_rng(23).standard_normal(d["n_nodes"])
    o1 = oracle.Oracle(d, cheb_degree=2, cheb_degree_I=1)
    o1.setup()
    y1 = o1.apply_S(xp)
    o2 = oracle.Oracle(d, cheb_degree=1)
    o2.setup()
    xt = o2.solve_A(o2.apply_B(xp), o2.options().rtol_I)[0]
    assert np.array_equal(y1, o2.apply_D(xp) - o2.apply_C(xt))
    o3 = oracle.Oracle(d, cheb_degree=2, cheb_degree_I=2)
    o3.setup()
    assert not np.array_equal(y1, o3.apply_S(xp))


def test_cycle_with_a_chosen_degree(tiny):
    """or_vcycle_degree: the AMG(A) cycle of degree k on a context built with
    another degree equals the cycle of a context built with degree k."""
    d, _ = tiny
    b = np.random.default_rng(29).standard_normal(3 * d["n_nodes"])
    o = oracle.Oracle(d)
    o.setup()
    o1 = oracle.Oracle(d, cheb_degree=1)
    o1.setup()
    assert np.array_equal(o.vcycle(0, b, degree=1), o1.vcycle(0, b))
    assert np.array_equal(o.vcycle(0, b, degree=2), o.vcycle(0, b))
