"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: integer work (aggregate maps) and the sequential-order setup
sums (Galerkin blocks, S_hat) are bit-exact; FP64 products agree to rounding
(1e-12 of the row scale); solves agree within the error bound of their
tolerances; FP32/BF16 inner modes are checked against the FP64 oracle at the
bars 1e-5 (solution) and 1e-8 (true residual)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


CASES = {
    "tiny": synth.tiny(),
    # several reduction chunks and a ragged tail; 4 outlets
    "box9x11x23_q4": synth.MeshSpec(9, 11, 23, Lz=2.0, Re=300.0, seed=5, R=(1e2, 1e3, 3e3, 1e4), name="box9x11x23_q4"),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    d = synth.generate(CASES[request.param])
    s = Solver(d)
    s.setup()
    o = oracle.Oracle(d)
    o.setup()
    yield request.param, d, s, o
    s.close()


def test_apply_A_fp64(case):
    _, d, s, o = case
    x = np.random.default_rng(0).standard_normal(3 * d["n_nodes"])
    y = s.apply_A(_t(x)).cpu().numpy()
    yo = o.apply_A(x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 2e-2)])
def test_apply_A_low_precision(prec, tol):
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, precision=prec)
    s.setup()
    o = oracle.Oracle(d)
    x = np.random.default_rng(1).standard_normal(3 * d["n_nodes"])
    y = s.apply_A(_t(x.astype(np.float32)), precision=prec).cpu().numpy().astype(np.float64)
    yo = o.apply_A(x.astype(np.float32).astype(np.float64))
    # bound: |A||x| row scale times the storage rounding of the values
    scale = np.abs(yo).max()
    assert np.abs(y - yo).max() <= tol * scale
    s.close()


def test_apply_full_fp64(case):
    _, d, s, o = case
    x = np.random.default_rng(2).standard_normal(4 * d["n_nodes"])
    y = s.apply_full(_t(x)).cpu().numpy()
    yo = o.apply_full(x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()


def test_amg_hierarchy_bit_exact(case):
    """Aggregate maps and Galerkin blocks equal the oracle's bit for bit."""
    _, d, s, o = case
    for which in (0, 1):
        G = s.amg_levels(which)
        O = o.amg_levels(which)
        assert len(G) == len(O)
        for lg, lo in zip(G, O):
            assert np.array_equal(lg["rowptr"], lo["rowptr"])
            assert np.array_equal(lg["col"], lo["col"])
            assert np.array_equal(lg["val"], lo["val"])
            if lo["agg"] is not None:   # smoothed levels: Chebyshev bounds (Arnoldi in FP64) to rounding
                assert np.array_equal(lg["agg"], lo["agg"])
                assert lg["rho"] == pytest.approx(lo["rho"], rel=1e-9)


def test_shat_bit_exact(case):
    _, d, s, o = case
    rp, ci, v = s.shat()
    rpo, cio, vo = o.shat()
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio)
    assert np.array_equal(v, vo)


def test_vcycle_fp64(case):
    _, d, s, o = case
    rng = np.random.default_rng(3)
    for which, n in ((0, 3 * d["n_nodes"]), (1, d["n_nodes"])):
        b = rng.standard_normal(n)
        x = s.vcycle(which, _t(b)).cpu().numpy()
        xo = o.vcycle(which, b)
        assert _rel(x, xo) <= 1e-10


def test_solve_A_tight(case):
    _, d, s, o = case
    b = np.random.default_rng(4).standard_normal(3 * d["n_nodes"])
    y, its = s.solve_A(_t(b), 1e-12)
    yo, itso, _ = o.solve_A(b, 1e-12)
    assert _rel(y.cpu().numpy(), yo) <= 1e-8
    assert abs(its - itso) <= 1


def test_matrix_free_schur():
    """Algorithm 2 on the device vs the oracle, both with a tight inner solve."""
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, rtol_I=1e-12)
    s.setup()
    o = oracle.Oracle(d, rtol_I=1e-12)
    o.setup()
    xp = np.random.default_rng(5).standard_normal(d["n_nodes"])
    y = s.apply_S(_t(xp)).cpu().numpy()
    assert _rel(y, o.apply_S(xp)) <= 1e-8
    s.close()


def test_nested_solve_fp64(case):
    name, d, s, o = case
    x, info = s.solve(_t(d["b"]))
    xh = x.cpu().numpy()
    r = d["b"] - o.apply_full(xh)
    assert np.linalg.norm(r) / np.linalg.norm(d["b"]) <= 1e-8
    assert info["rel_res_true"] <= 1e-8
    o.set_options(rtol=1e-12)
    xo, oinfo, rc = o.solve(d["b"])
    o.set_options(rtol=1e-8)
    assert rc == 0
    assert _rel(xh, xo) <= 1e-6
    if name == "tiny":
        *_, F = oracle.dense_system(d)
        assert _rel(xh, np.linalg.solve(F, d["b"])) <= 1e-6


def test_nested_solve_iteration_counts_match_oracle(case):
    _, d, s, o = case
    _, info = s.solve(_t(d["b"]))
    _, oinfo, _ = o.solve(d["b"])
    assert abs(info["outer_iters"] - oinfo.outer_iters) <= 1
    assert abs(info["S_iters"] - oinfo.S_iters) <= max(2, 0.1 * oinfo.S_iters)


@pytest.mark.parametrize("prec", [1, 2, 3, 4])
def test_nested_solve_mixed(prec):
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, precision=prec)
    s.setup()
    o = oracle.Oracle(d, rtol=1e-12)
    o.setup()
    x, info = s.solve(_t(d["b"]))
    xh = x.cpu().numpy()
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) / np.linalg.norm(d["b"]) <= 1e-8
    xo, _, _ = o.solve(d["b"])
    assert _rel(xh, xo) <= 1e-5
    s.close()


@pytest.mark.parametrize("prec,pc_A,variant", [(0, 0, 0), (1, 0, 0), (3, 0, 0), (4, 0, 0), (3, 1, 0), (3, 0, 1)])
def test_device_loop_matches_host_loop(prec, pc_A, variant):
    """The nested solve as one graph with device-driven WHILE loops against
    the host-driven loop: the same iteration counts (within one), solutions
    equal to far below the solve tolerance, the oracle's true residual
    <= 1e-8, and two device-loop solves in a row (one captured graph, two
    launches) bitwise equal."""
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, precision=prec, pc_A=pc_A, variant=variant)
    s.setup()
    b = _t(d["b"])
    x0, i0 = s.solve(b, device_loop=0)
    x1, i1 = s.solve(b, device_loop=1)
    x2, i2 = s.solve(b, device_loop=1)
    assert torch.equal(x1, x2)
    for k in ("outer_iters", "A_iters", "S_iters", "I_iters"):
        assert i1[k] == i2[k]
    assert abs(i1["outer_iters"] - i0["outer_iters"]) <= 1
    assert abs(i1["S_iters"] - i0["S_iters"]) <= max(2, 0.05 * i0["S_iters"])
    x0h, x1h = x0.cpu().numpy(), x1.cpu().numpy()
    assert _rel(x1h, x0h) <= 1e-6
    o = oracle.Oracle(d)
    assert np.linalg.norm(d["b"] - o.apply_full(x1h)) / np.linalg.norm(d["b"]) <= 1e-8
    assert i1["rel_res_true"] <= 1e-8
    s.close()


def test_device_loop_falls_back_when_inner_solves_restart():
    """With m_A < n_max_A an inner solve may restart, which the device loop
    does not do: the host-driven loop runs instead, with the same result."""
    d = synth.generate(synth.tiny())
    s = Solver(d, precision=1)
    s.setup()
    b = _t(d["b"])
    x0, i0 = s.solve(b, m_A=4, device_loop=0)
    x1, i1 = s.solve(b, m_A=4, device_loop=1)
    assert torch.equal(x0, x1)
    s.close()


def test_block_triangular_two_iterations():
    d = synth.generate(synth.tiny())
    s = Solver(d, variant=1, rtol_A=1e-13, rtol_S=1e-13, rtol_I=1e-13)
    s.setup()
    _, info = s.solve(_t(d["b"]))
    assert info["outer_iters"] == 2
    s.close()


@pytest.mark.parametrize("prec", [0, 3])
def test_adjoint_matches_oracle(prec):
    spec = CASES["box9x11x23_q4"]
    d = synth.generate(spec)
    s = Solver(d, rtol=1e-12, precision=prec)
    s.setup()
    x, _ = s.solve(_t(d["b"]))
    xh = x.cpu().numpy()
    nv = 3 * d["n_nodes"]
    g = np.zeros(4 * d["n_nodes"])
    rng = np.random.default_rng(6)
    g[:nv] = rng.standard_normal(nv)
    lam, dldr, info = s.adjoint(_t(g), x)
    lam_o, dldr_o, _ = oracle.adjoint(d, g, xh, rtol=1e-12)
    assert _rel(lam.cpu().numpy(), lam_o) <= (1e-6 if prec == 0 else 1e-5)
    assert np.allclose(dldr, dldr_o, rtol=1e-5, atol=0)
    s.close()


def test_repeatable_bitwise(case):
    _, d, s, o = case
    x1, _ = s.solve(_t(d["b"]))
    x2, _ = s.solve(_t(d["b"]))
    assert torch.equal(x1, x2)


def test_invalid_input_rejected():
    d = synth.generate(synth.tiny())
    bad = dict(d)
    col = d["col"].copy()
    col[5] = 10 ** 6
    bad["col"] = col
    from paper_1911_10814_gb300.nbp import NbpError
    with pytest.raises(NbpError):
        Solver(bad)


@pytest.mark.parametrize("cycle,kdepth", [(1, 1), (2, 1), (1, 3)])
def test_kcycle_vcycle_vs_oracle(cycle, kdepth):
    """K-cycle on the coarse levels (device coefficients, graph replay) vs the oracle."""
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, amg_coarse_max=10, amg_cycle=cycle, amg_kdepth=kdepth)
    s.setup()
    o = oracle.Oracle(d, amg_coarse_max=10, amg_cycle=cycle, amg_kdepth=kdepth)
    o.setup()
    rng = np.random.default_rng(8)
    for which, n in ((0, 3 * d["n_nodes"]), (1, d["n_nodes"])):
        assert len(s.amg_levels(which)) >= 3
        b = rng.standard_normal(n)
        for _ in range(2):   # second call replays the captured graph
            x = s.vcycle(which, _t(b)).cpu().numpy()
            assert _rel(x, o.vcycle(which, b)) <= 1e-10
    x, info = s.solve(_t(d["b"]))
    assert np.linalg.norm(d["b"] - o.apply_full(x.cpu().numpy())) / np.linalg.norm(d["b"]) <= 1e-8
    s.close()


@pytest.mark.parametrize("prec", [0, 3])
def test_restarted_solves_match_oracle(prec):
    """GMRES(4) at every level (outer, A and S solves all restart) on a context
    whose Krylov spaces were first sized by a GMRES(200) solve: the smaller
    restart length reuses the larger allocation."""
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, precision=prec)
    s.setup()
    s.solve(_t(d["b"]))
    x, info = s.solve(_t(d["b"]), m=4, m_A=4, m_S=4)
    xh = x.cpu().numpy()
    o = oracle.Oracle(d, m=4, m_A=4, m_S=4)
    o.setup()
    xo, oinfo, rc = o.solve(d["b"])
    assert rc == 0 and oinfo.outer_iters > 4 and oinfo.A_iters > 4 * oinfo.n_A_solves
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) / np.linalg.norm(d["b"]) <= 1e-8
    assert info["rel_res_true"] <= 1e-8
    if prec == 0:
        assert abs(info["outer_iters"] - oinfo.outer_iters) <= 1
        assert abs(info["S_iters"] - oinfo.S_iters) <= max(2, 0.1 * oinfo.S_iters)
    o.set_options(rtol=1e-12)
    xt, _, _ = o.solve(d["b"])
    assert _rel(xh, xt) <= 1e-5
    s.close()


def test_simple_variant_solves_and_matches_oracle():
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, variant=2)
    s.setup()
    o = oracle.Oracle(d, variant=2)
    o.setup()
    x, info = s.solve(_t(d["b"]))
    xh = x.cpu().numpy()
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) / np.linalg.norm(d["b"]) <= 1e-8
    sv = np.random.default_rng(13).standard_normal(4 * d["n_nodes"])
    o2 = oracle.Oracle(d, variant=2, rtol_A=1e-12, rtol_S=1e-12)
    o2.setup()
    s2 = Solver(d, variant=2, rtol_A=1e-12, rtol_S=1e-12)
    s2.setup()
    assert _rel(s2.apply_pscr(_t(sv)).cpu().numpy(), o2.apply_pscr(sv)) <= 1e-7
    s.close()
    s2.close()


def test_zero_rhs_gives_zero_solution():
    """b = 0: the nested solve returns x = 0 at once (||b|| = 0 meets every
    tolerance) in every precision mode."""
    d = synth.generate(synth.tiny())
    s = Solver(d, precision=3)
    s.setup()
    b = torch.zeros(4 * d["n_nodes"], dtype=torch.float64, device=DEV)
    for prec in (0, 1, 3, 4):
        x, info = s.solve(b, precision=prec)
        assert float(torch.abs(x).max()) == 0.0 and info["outer_iters"] == 0
    s.close()


@pytest.mark.parametrize("prec", [0, 2])
def test_no_outlets(prec):
    """A tangent without outlet coupling (n_out = 0, no rank-one term): the
    A product, S_hat and the nested solve against the oracle."""
    spec = synth.MeshSpec(7, 9, 13, Lz=2.0, Re=200.0, seed=8, R=(), name="box7x9x13_o0")
    d = synth.generate(spec)
    assert len(d["out_ptr"]) == 1
    s = Solver(d, precision=prec)
    s.setup()
    o = oracle.Oracle(d, rtol=1e-12)
    x = np.random.default_rng(2).standard_normal(3 * d["n_nodes"])
    y = s.apply_A(_t(x)).cpu().numpy()
    yo = o.apply_A(x)
    assert np.max(np.abs(y - yo)) <= 1e-12 * np.max(np.abs(yo))
    xs, info = s.solve(_t(d["b"]))
    xh = xs.cpu().numpy()
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) <= 1e-8 * np.linalg.norm(d["b"])
    xo, _, _ = o.solve(d["b"])
    assert _rel(xh, xo) <= (1e-6 if prec == 0 else 1e-5)
    s.close()


@pytest.mark.parametrize("deg,gs", [(1, 1), (2, 1), (1, 2)])
def test_inner_cycle_degree_matches_oracle(deg, gs):
    """Algorithm 2's inner A-solves preconditioned by the AMG(A) cycle of
    degree cheb_degree_I (1 by default, 2 the degree of the other A-solves),
    with gs Gram-Schmidt passes per Arnoldi step (the oracle's modified
    Gram-Schmidt is the same process in exact arithmetic): FP64 solve, the
    oracle's iteration counts and solution."""
    d = synth.generate(CASES["box9x11x23_q4"])
    s = Solver(d, cheb_degree_I=deg, gs_passes_I=gs)
    s.setup()
    o = oracle.Oracle(d, cheb_degree_I=deg)
    o.setup()
    x, info = s.solve(_t(d["b"]))
    xo, oi, rc = o.solve(d["b"])
    assert rc == 0 and info["rel_res_true"] <= 1e-8
    assert info["outer_iters"] == oi.outer_iters
    assert abs(info["I_iters"] - oi.I_iters) <= max(2, 0.05 * oi.I_iters)
    assert _rel(x.cpu().numpy(), xo) <= 1e-6
    s.close()
