"""Parity of the on-device VMS residual, tangent and Newton time step
(Sec. 2.3-2.5) with the oracle, through the C ABI.

Tolerances: FP64 residual and FP64 tangent agree with the oracle to
rounding (1e-12 of each array's largest entry; both sum the same terms in a
different order).  The FP32 tangent: every entry is a sum of O(10^2) FP32
products and sums of terms no larger than the block's largest entry, so its
error is below 10^2 x 2^-24 ~ 6e-6 of that entry; the bar is 2e-5.  Newton
steps: both sides solve each tangent system to a relative residual 1e-10,
so the accepted states agree to well below the stopping tolerance; bar 1e-7."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver, Vms  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _maxrel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SPEC = synth.MeshSpec(5, 4, 7, Lz=1.5, Re=400.0, seed=11, R=(1e3, 3e3, 1e4), name="box5x4x7_o3")


@pytest.fixture(scope="module")
def case():
    d = synth.generate(SPEC)
    m = synth.mesh(SPEC)
    ph = oracle.vms_phys(SPEC)
    return d, m, ph


def _state(d, seed):
    rng = np.random.default_rng(seed)
    N = d["n_nodes"]
    v = d["vel"] * (1.0 + 0.3 * rng.standard_normal(3 * N))
    vd = 40.0 * rng.standard_normal(3 * N)
    p = 80.0 * rng.standard_normal(N)
    P = 1e3 * rng.uniform(0.5, 1.5, SPEC.n_out)
    return vd, v, p, P


def _vms(d, m, fp32, **opts):
    s = Solver(d, **opts)
    vm = Vms(s, m, SPEC.rho, SPEC.mu, SPEC.dt, SPEC.rho_inf, tangent_fp32=fp32)
    return s, vm


def test_residual_matches_oracle(case):
    d, m, ph = case
    s, vm = _vms(d, m, False)
    N = d["n_nodes"]
    for seed in (1, 2):
        vd, v, p, P = _state(d, seed)
        ref = oracle.vms_assemble(m, d, ph, vd, v, p, P, tangent=False)["R"]
        got = vm.residual(_t(vd), _t(v), _t(p), _t(P)).cpu().numpy()
        assert _maxrel(got, ref) <= 1e-12
    # frozen tau at another velocity
    vd, v, p, P = _state(d, 3)
    vt = d["vel"]
    ref = oracle.vms_assemble(m, d, ph, vd, v, p, P, vtau=vt, tangent=False)["R"]
    got = vm.residual(_t(vd), _t(v), _t(p), _t(P), vtau=_t(vt)).cpu().numpy()
    assert _maxrel(got, ref) <= 1e-12
    # bitwise repeatable
    again = vm.residual(_t(vd), _t(v), _t(p), _t(P), vtau=_t(vt)).cpu().numpy()
    assert np.array_equal(got, again)
    assert N == len(got) // 4
    vm.close()
    s.close()


@pytest.mark.parametrize("fp32,tol", [(False, 1e-12), (True, 2e-5)])
def test_tangent_matches_oracle(case, fp32, tol):
    d, m, ph = case
    s, vm = _vms(d, m, fp32)
    nnz = len(d["col"])
    vd, v, p, P = _state(d, 4)
    ref = oracle.vms_assemble(m, d, ph, vd, v, p, P, residual=False)
    got = vm.tangent(_t(vd), _t(v), _t(p), nnz)
    for k in "ABCD":
        assert _maxrel(got[k].cpu().numpy(), ref[k]) <= tol, k
    vm.close()
    s.close()


def test_tangent_equals_generator_tangent(case):
    """At the generator's state (vdot = 0, p = 0) the device tangent is the
    generator's A, B, C, D."""
    d, m, ph = case
    s, vm = _vms(d, m, False)
    N, nnz = d["n_nodes"], len(d["col"])
    got = vm.tangent(_t(np.zeros(3 * N)), _t(d["vel"]), _t(np.zeros(N)), nnz)
    for k in "ABCD":
        assert _maxrel(got[k].cpu().numpy(), d[k]) <= 1e-12, k
    vm.close()
    s.close()


def test_set_values_then_solve(case):
    """New tangent values in place, new setup, nested solve: the solution of
    the new system (checked with the oracle's operator)."""
    d, m, ph = case
    vd, v, p, P = _state(d, 5)
    T = oracle.vms_assemble(m, d, ph, vd, v, p, P, residual=False)
    s = Solver(d)
    s.setup()
    s.set_values(*(_t(np.ravel(T[k])) for k in "ABCD"))
    with pytest.raises(Exception):
        s.solve(_t(d["b"]))             # setup is stale
    s.setup()
    x, info = s.solve(_t(d["b"]))
    d2 = dict(d, A=T["A"], B=T["B"], C=T["C"], D=T["D"])
    o = oracle.Oracle(d2)
    r = d["b"] - o.apply_full(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(d["b"]) <= 1e-8
    s.close()


def _rcr(seed=7):
    R = np.asarray(SPEC.R)
    rng = np.random.default_rng(seed)
    return dict(Rp=0.1 * R, Rd=0.9 * R, C=1e-1 / R, Pd=np.full(len(R), 5.0),
                Pi=rng.uniform(10.0, 50.0, len(R)), nts=10)


@pytest.mark.parametrize("fp32", [False, True])
def test_newton_step_matches_oracle(case, fp32):
    d, m, ph = case
    N = d["n_nodes"]
    am, af, gm = oracle.gen_alpha(ph.rho_inf)
    rng = np.random.default_rng(9)
    y_n = np.concatenate([d["vel"], 10.0 * rng.standard_normal(N)])
    yd_n = np.concatenate([rng.standard_normal(3 * N) * np.repeat(m["dir"] == 0, 3), rng.standard_normal(N)])
    rc = _rcr()
    ref = oracle.newton_step(m, d, ph, y_n, yd_n, rc, tol_R=1e-8, tol_A=1e-12, rtol=1e-10)
    s, vm = _vms(d, m, fp32, rtol=1e-10)
    rct = {k: _t(rc[k]) for k in ("Rp", "C", "Rd", "Pd", "Pi")}
    y, yd, Pi, info = vm.newton_step(_t(y_n), _t(yd_n), rct, tol_R=1e-8, tol_A=1e-12, nts=rc["nts"])
    y, yd, Pi = y.cpu().numpy(), yd.cpu().numpy(), Pi.cpu().numpy()
    assert info["converged"] == 1
    if not fp32:
        assert info["iters"] == ref["iters"]
        assert abs(info["res0"] - ref["res"][0]) <= 1e-12 * ref["res"][0]
    assert _maxrel(y, ref["y"]) <= 1e-7
    assert _maxrel(yd, ref["yd"]) <= 1e-7 * max(1.0, np.abs(ref["yd"]).max() / np.abs(yd_n).max())
    assert _maxrel(Pi, ref["Pi"]) <= 1e-9
    # generalized-alpha relation and Dirichlet values
    lhs = y - y_n - ph.dt * yd_n - gm * ph.dt * (yd - yd_n)
    assert np.abs(lhs).max() <= 1e-12 * np.abs(y_n).max()
    dm = np.repeat(m["dir"] == 1, 3)
    assert np.array_equal(y[:3 * N][dm], y_n[:3 * N][dm])
    vm.close()
    s.close()


@pytest.mark.parametrize("lag", [2, 3, 4])
def test_lagged_preconditioner_matches_oracle(case, lag):
    """Two time steps with a preconditioner other than a build per tangent
    (pc_rebuild 2: built from the first tangent, kept for every later one;
    3: rebuilt numerically on the first build's aggregates from every
    tangent; 4: the same once per step, kept within it): the same corrector
    counts, builds and accepted states as the oracle's steps in that mode,
    and the same corrector counts as a build per tangent (pc_rebuild 0)."""
    d, m, ph = case
    N = d["n_nodes"]
    rng = np.random.default_rng(9)
    y_n = np.concatenate([d["vel"], 10.0 * rng.standard_normal(N)])
    yd_n = np.concatenate([rng.standard_normal(3 * N) * np.repeat(m["dir"] == 0, 3), rng.standard_normal(N)])
    rc = _rcr()
    iters = {}
    for mode in (0, lag):
        s, vm = _vms(d, m, False, rtol=1e-10)
        pc = {}
        y, yd, Pi_h, rch = _t(y_n), _t(yd_n), rc["Pi"], dict(rc)
        yo, ydo = y_n, yd_n
        iters[mode] = []
        for step in range(2):
            rct = {k: _t(rch[k]) for k in ("Rp", "C", "Rd", "Pd")}
            rct["Pi"] = _t(Pi_h)
            y, yd, Pi, info = vm.newton_step(y, yd, rct, tol_R=1e-8, tol_A=1e-12, nts=rc["nts"], pc_rebuild=mode)
            assert info["converged"] == 1
            iters[mode].append(info["iters"])
            ref = oracle.newton_step(m, d, ph, yo, ydo, dict(rch, Pi=Pi_h), tol_R=1e-8, tol_A=1e-12, rtol=1e-10,
                                     pc_rebuild=mode, pc=pc)
            assert info["iters"] == ref["iters"]
            assert info["setups"] == ref["setups"]
            assert info["numeric_setups"] == ref["numeric"]
            if mode in (2, 3, 4):
                assert info["setups"] == (1 if step == 0 else 0)
            assert _maxrel(y.cpu().numpy(), ref["y"]) <= 1e-7
            Pi_h = Pi.cpu().numpy()
            yo, ydo = ref["y"], ref["yd"]
            y, yd = _t(yo), _t(ydo)
        vm.close()
        s.close()
    assert iters[0] == iters[lag]


def test_newton_without_outlets():
    sp = synth.MeshSpec(4, 4, 5, Re=200.0, seed=2, R=(), name="box4_no_outlets")
    d, m = synth.generate(sp), synth.mesh(sp)
    ph = oracle.vms_phys(sp)
    N = d["n_nodes"]
    y_n = np.concatenate([d["vel"], np.zeros(N)])
    yd_n = np.zeros(4 * N)
    ref = oracle.newton_step(m, d, ph, y_n, yd_n, dict(Rp=[], C=[], Rd=[], Pd=[], Pi=[], nts=1), tol_R=1e-8,
                             tol_A=1e-12, rtol=1e-10)
    s = Solver(d, rtol=1e-10)
    vm = Vms(s, m, sp.rho, sp.mu, sp.dt, sp.rho_inf, tangent_fp32=False)
    y, yd, Pi, info = vm.newton_step(_t(y_n), _t(yd_n), None, tol_R=1e-8, tol_A=1e-12)
    assert info["iters"] == ref["iters"]
    assert _maxrel(y.cpu().numpy(), ref["y"]) <= 1e-7
    vm.close()
    s.close()


def test_pattern_mismatch_rejected(case):
    d, m, ph = case
    s = Solver(d)
    bad = dict(m, tets=np.vstack([m["tets"], [[0, 1, 2, d["n_nodes"] - 1]]]).astype(np.int32))
    with pytest.raises(Exception):
        Vms(s, bad, SPEC.rho, SPEC.mu, SPEC.dt, SPEC.rho_inf)
    s.close()


def test_degenerate_elements_rejected(case):
    """A tet with a repeated vertex (zero volume) or a collinear outlet triangle
    is refused when the mesh is bound (its node pairs are in the pattern, so
    only the degeneracy check can refuse it)."""
    d, m, ph = case
    s = Solver(d)
    t = m["tets"][0]
    flat = dict(m, tets=np.vstack([m["tets"], [[t[0], t[1], t[2], t[0]]]]).astype(np.int32))
    with pytest.raises(Exception):
        Vms(s, flat, SPEC.rho, SPEC.mu, SPEC.dt, SPEC.rho_inf)
    f = m["tris"][0]
    line = dict(m, tris=np.vstack([m["tris"], [[f[0], f[1], f[1]]]]).astype(np.int32))
    with pytest.raises(Exception):
        Vms(s, line, SPEC.rho, SPEC.mu, SPEC.dt, SPEC.rho_inf)
    vm = Vms(s, m, SPEC.rho, SPEC.mu, SPEC.dt, SPEC.rho_inf)   # the mesh itself binds
    vm.close()
    s.close()


def test_set_values_refuses_non_finite(case):
    """A NaN in the new values is refused before anything is replaced: the
    context keeps its values and its setup, and solves as before."""
    d, m, ph = case
    s = Solver(d)
    s.setup()
    x0, _ = s.solve(_t(d["b"]))
    A = np.ravel(d["A"]).copy()
    A[7] = np.nan
    with pytest.raises(Exception):
        s.set_values(_t(A), _t(np.ravel(d["B"])), _t(np.ravel(d["C"])), _t(np.ravel(d["D"])))
    x1, _ = s.solve(_t(d["b"]))
    assert torch.equal(x0, x1)
    s.close()
