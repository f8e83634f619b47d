"""RCR outlets on the GPU (Sec. 2.1 model, Algorithm 1, the difference-quotient
stiffness of Sec. 2.5) through the C ABI, against the FP64 oracle; and the
many-outlet stress case (772 outlet patches) of the nested solve.

Tolerances: the RCR step is FP64 arithmetic in the same order on both sides,
so P and Pi agree to rounding (1e-13 relative); m^k is a difference quotient
whose rounding grows as (size of the recurrence's terms) / eps, so it is held
to that bound, and to 1e-10 with a wide difference step; solves are
held to the true residual 1e-8 and the oracle's solution at 1e-6 (FP64) or
1e-5 (mixed)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import NbpError, Solver, rcr_step  # noqa: E402
from paper_1911_10814_gb300 import nbp as _nbp  # noqa: E402

DEV = "cuda:0"


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _params(n, seed):
    rng = np.random.default_rng(seed)
    return dict(Rp=10 ** rng.uniform(1, 3, n), C=10 ** rng.uniform(-5, -3, n), Rd=10 ** rng.uniform(2, 4, n),
                Pd=rng.uniform(0, 10, n), Pi_n=rng.uniform(0, 100, n), Q_n=rng.uniform(-1, 1, n))


def _m_bound(p, Q1, P, dt, nts):
    """Rounding bound of the central difference (P+ - P-) / eps when the two
    sides round differently: each P is an nts-step recurrence whose terms
    are of size S = |Rp Q1| + |Pi_n| + |Pd| + |P| + dt (|Q_n| + |Q1|) / C."""
    eps = np.maximum(1e-8, 1e-5 * np.abs(Q1))
    S = (np.abs(p["Rp"] * Q1) + np.abs(p["Pi_n"]) + np.abs(p["Pd"]) + np.abs(P)
         + dt * (np.abs(p["Q_n"]) + np.abs(Q1)) / p["C"])
    return 16 * (nts + 1) * np.finfo(float).eps * S / eps


@pytest.mark.parametrize("nts", [1, 10])
def test_rcr_step_matches_oracle_772_outlets(nts):
    n = 772
    p = _params(n, 41)
    Q1 = np.random.default_rng(42).uniform(-1, 1, n)
    dt = 1e-3
    P, Pi, m = rcr_step(*[_t(p[k]) for k in ("Rp", "C", "Rd", "Pd", "Pi_n", "Q_n")], _t(Q1), dt, nts)
    torch.cuda.synchronize()
    Po, Pio, mo = oracle.rcr_step(p["Rp"], p["C"], p["Rd"], p["Pd"], p["Pi_n"], p["Q_n"], Q1, dt, nts)
    P, Pi, m = P.cpu().numpy(), Pi.cpu().numpy(), m.cpu().numpy()
    assert np.max(np.abs(P - Po) / np.abs(Po)) <= 1e-13
    assert np.max(np.abs(Pi - Pio) / np.abs(Pio)) <= 1e-13
    assert np.all(np.abs(m - mo) <= _m_bound(p, Q1, Po, dt, nts))
    # with a wide difference step the quotient's rounding vanishes
    _, _, mw = rcr_step(*[_t(p[k]) for k in ("Rp", "C", "Rd", "Pd", "Pi_n", "Q_n")], _t(Q1), dt, nts, eps_abs=1e-2,
                        eps_rel=0.0)
    _, _, mwo = oracle.rcr_step(p["Rp"], p["C"], p["Rd"], p["Pd"], p["Pi_n"], p["Q_n"], Q1, dt, nts, eps_abs=1e-2,
                                eps_rel=0.0)
    assert np.max(np.abs(mw.cpu().numpy() - mwo) / np.abs(mwo)) <= 1e-10


def test_rcr_step_rejects_bad_arguments():
    lib = _nbp.load()
    p = _params(4, 1)
    ts = {k: _t(v) for k, v in p.items()}
    par = _nbp.rcr_params(ts["Rp"], ts["C"], ts["Rd"], ts["Pd"], ts["Pi_n"], ts["Q_n"])
    q = _t(np.zeros(4))
    out = _t(np.zeros(4))
    import ctypes
    args = (ctypes.byref(par), ctypes.c_void_p(q.data_ptr()))
    o = ctypes.c_void_p(out.data_ptr())
    assert lib.nbp_rcr_step(4, *args, 1e-3, 0, o, o, o, None) == 1          # nts < 1
    assert lib.nbp_rcr_step(4, *args, 0.0, 5, o, o, o, None) == 1          # dt <= 0
    assert lib.nbp_rcr_step(-1, *args, 1e-3, 5, o, o, o, None) == 1        # n_out < 0
    bad = _nbp.rcr_params(ts["Rp"], ts["C"], ts["Rd"], ts["Pd"], ts["Pi_n"], ts["Q_n"], eps_abs=0.0, eps_rel=0.0)
    assert lib.nbp_rcr_step(4, ctypes.byref(bad), ctypes.c_void_p(q.data_ptr()), 1e-3, 5, o, o, o, None) == 1


@pytest.fixture(scope="module")
def q4():
    spec = synth.MeshSpec(9, 11, 23, Lz=2.0, Re=300.0, seed=5, R=(1e2, 1e3, 3e3, 1e4), name="box9x11x23_q4")
    return spec, synth.generate(spec)


def test_outlet_flows_match_oracle(q4):
    _, d = q4
    s = Solver(d)
    v = np.random.default_rng(5).standard_normal(3 * d["n_nodes"])
    Q = s.outlet_flows(_t(v)).cpu().numpy()
    Qo = oracle.outlet_flows(d, v)
    assert np.max(np.abs(Q - Qo)) <= 1e-13 * np.max(np.abs(Qo))
    s.close()


def test_rcr_update_feeds_the_solve(q4):
    """The Newton-step coupling: Q from the velocity, the RCR step, r_k =
    alpha_f gamma dt m^k installed on the device; the next nested solve is
    the oracle's solve with those weights."""
    spec, d = q4
    n = spec.n_out
    p = _params(n, 7)
    s = Solver(d)
    s.setup()
    v = np.asarray(d["vel"]) * 10.0
    scale = spec.alpha_f_gamma_dt
    out = s.rcr_update({k: _t(p[k]) for k in p}, _t(v), spec.dt, 8, scale)
    Q = out["Q"].cpu().numpy()
    Qo = oracle.outlet_flows(d, v)
    assert np.max(np.abs(Q - Qo)) <= 1e-13 * np.max(np.abs(Qo))
    Po, Pio, mo = oracle.rcr_step(p["Rp"], p["C"], p["Rd"], p["Pd"], p["Pi_n"], p["Q_n"], Q, spec.dt, 8)
    m = out["m"].cpu().numpy()
    assert np.all(np.abs(m - mo) <= _m_bound(p, Q, Po, spec.dt, 8))
    assert np.max(np.abs(out["P"].cpu().numpy() - Po) / np.abs(Po)) <= 1e-13
    # the solve uses r = scale m (the GPU's m); the oracle gets the same weights
    d2 = dict(d)
    d2["r"] = scale * m
    x, info = s.solve(_t(d["b"]), rtol=1e-10)
    o = oracle.Oracle(d2, rtol=1e-12)
    xo, _, _ = o.solve(d["b"])
    xh = x.cpu().numpy()
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) <= 1e-8 * np.linalg.norm(d["b"])
    assert _rel(xh, xo) <= 1e-6
    s.close()


def test_rcr_update_non_finite_stiffness_is_reported(q4):
    """A zero compliance gives an infinite rate: NBP_ERR_NAN, the weights stay
    as they were, and the context keeps working."""
    spec, d = q4
    n = spec.n_out
    p = _params(n, 8)
    p["C"] = np.zeros(n)
    s = Solver(d, rtol=1e-10)
    s.setup()
    with pytest.raises(NbpError) as e:
        s.rcr_update({k: _t(p[k]) for k in p}, _t(np.asarray(d["vel"])), spec.dt, 4, spec.alpha_f_gamma_dt)
    assert e.value.status == 6
    x, _ = s.solve(_t(d["b"]))
    o = oracle.Oracle(d)
    assert np.linalg.norm(d["b"] - o.apply_full(x.cpu().numpy())) <= 1e-8 * np.linalg.norm(d["b"])
    s.close()


@pytest.fixture(scope="module")
def many():
    u = synth.uniforms(7 ^ 0x5EED, 772)
    R = tuple(float(10.0 ** (2.0 + 3.0 * x)) for x in u)
    spec = synth.MeshSpec(32, 32, 16, Lz=0.5, Re=300.0, seed=7, R=R, name="box32x32x16_o772")
    d = synth.generate(spec)
    o = oracle.Oracle(d, rtol=1e-12)
    xo, _, _ = o.solve(d["b"])
    return d, o, xo


@pytest.mark.parametrize("prec", [0, 3])
def test_many_outlet_nested_solve(many, prec):
    """772 outlet patches: 772 rank-one terms in every A product (per-outlet
    inner products, per-row epilogue lists) and in diag(A) for S_hat."""
    d, o, xo = many
    s = Solver(d, precision=prec)
    s.setup()
    x, info = s.solve(_t(d["b"]))
    xh = x.cpu().numpy()
    assert np.linalg.norm(d["b"] - o.apply_full(xh)) <= 1e-8 * np.linalg.norm(d["b"])
    assert _rel(xh, xo) <= (1e-6 if prec == 0 else 1e-5)
    # the A product with its 772 rank-one terms, row by row
    v = np.random.default_rng(3).standard_normal(3 * d["n_nodes"])
    y = s.apply_A(_t(v)).cpu().numpy()
    yo = o.apply_A(v)
    assert np.max(np.abs(y - yo)) <= 1e-12 * np.max(np.abs(yo))
    s.close()
