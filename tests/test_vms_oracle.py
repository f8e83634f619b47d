"""Pins of the oracle's VMS residual / tangent and of its predictor
multi-corrector (Sec. 2.3-2.5) against what the mathematics fixes: P1
closed forms, an independently derived tangent, finite differences, the
divergence theorem, the node-order invariance the metric M provides, and
the generalized-alpha update identity."""
import itertools

import numpy as np
import pytest

import oracle
import synth


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.fixture(scope="module")
def small():
    sp = synth.MeshSpec(3, 3, 4, Lz=2.0, Re=300.0, seed=3, R=(1e3, 1e4), name="box3x3x4")
    return sp, synth.generate(sp), synth.mesh(sp), oracle.vms_phys(sp)


def test_tangent_equals_generator_tangent(small):
    """At the generator's linearisation state (vdot = 0, p = 0, tau frozen) the
    dual-number tangent equals the generator's hand-derived A, B, C, D
    (a separate derivation of Sec. 2.5, backflow and Dirichlet rows included)."""
    sp, d, m, ph = small
    N = d["n_nodes"]
    T = oracle.vms_assemble(m, d, ph, np.zeros(3 * N), d["vel"], np.zeros(N), residual=False)
    for k in "ABCD":
        assert np.abs(T[k] - d[k]).max() <= 1e-13 * np.abs(d[k]).max()


def _one_tet(X):
    """A one-element mesh with the all-pairs pattern and no Dirichlet nodes."""
    rp = np.arange(0, 17, 4, dtype=np.int32)
    col = np.tile(np.arange(4, dtype=np.int32), 4)
    mesh = dict(X=np.asarray(X, float), tets=np.array([[0, 1, 2, 3]], np.int32), tris=np.zeros((0, 3), np.int32),
                dir=np.zeros(4, np.uint8))
    sysd = dict(n_nodes=4, rowptr=rp, col=col, out_ptr=np.zeros(1, np.int32), out_idx=np.zeros(0, np.int32),
                out_val=np.zeros(0))
    return mesh, sysd


def test_single_element_closed_forms():
    """Zero state on one tet: the tangent blocks are the P1 consistent mass,
    viscous and grad-div stiffness, divergence/gradient and PSPG Laplacian
    matrices (exact under the degree-2 rule), with tau_M, tau_C from Sec. 2.3
    at zero velocity."""
    rng = np.random.default_rng(0)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.3 + 0.05 * rng.standard_normal((4, 3))
    mesh, sysd = _one_tet(X)
    ph = oracle.VmsPhys(1.06, 0.04, 1e-3, 0.5, 0.2, 36.0, 4.0)
    am, af, gm = oracle.gen_alpha(ph.rho_inf)
    c = af * gm * ph.dt
    T = oracle.vms_assemble(mesh, sysd, ph, np.zeros(12), np.zeros(12), np.zeros(4), residual=True)
    assert np.abs(T["R"]).max() == 0.0
    # independent geometry: grad N from the inverse of [1 x y z] (P1 interpolation)
    V = np.hstack([np.ones((4, 1)), X])
    coef = np.linalg.inv(V)                # N_a(x) = coef[0, a] + coef[1:, a] . x
    g = coef[1:, :].T                      # g[a] = grad N_a
    vol = abs(np.linalg.det(X[1:] - X[0])) / 6.0
    Jinv = np.linalg.inv((X[1:] - X[0]).T)   # d xi / d x with xi_k = N_{k+1}
    M = 2 ** (1 / 3) / 2 * (np.ones((3, 3)) + np.eye(3))
    G = Jinv.T @ M @ Jinv
    tauM = 1.0 / (ph.rho * np.sqrt(ph.CT / ph.dt ** 2 + ph.CI * (ph.mu / ph.rho) ** 2 * np.sum(G * G)))
    tauC = 1.0 / (tauM * np.trace(G))
    A = T["A"].reshape(4, 4, 3, 3)
    B = T["B"].reshape(4, 4, 3)
    C = T["C"].reshape(4, 4, 3)
    D = T["D"].reshape(4, 4)
    for a, b in itertools.product(range(4), range(4)):
        mass = vol / 20.0 * (2.0 if a == b else 1.0)
        Aref = am * ph.rho * mass * np.eye(3) + c * (
            ph.mu * vol * (g[a] @ g[b] * np.eye(3) + np.outer(g[b], g[a])) + tauC * vol * np.outer(g[a], g[b]))
        assert np.allclose(A[a, b], Aref, rtol=1e-12, atol=1e-14 * np.abs(Aref).max())
        assert np.allclose(B[a, b], -c * vol / 4.0 * g[a], rtol=1e-12, atol=1e-18)
        Cref = am * tauM * ph.rho * vol / 4.0 * g[a] + c * vol / 4.0 * g[b]
        assert np.allclose(C[a, b], Cref, rtol=1e-12, atol=1e-18)
        assert np.isclose(D[a, b], c * tauM * vol * (g[a] @ g[b]), rtol=1e-12)


def _state(d, seed):
    rng = np.random.default_rng(seed)
    N = d["n_nodes"]
    v = d["vel"] * (1.0 + 0.2 * rng.standard_normal(3 * N))
    vd = 50.0 * rng.standard_normal(3 * N)
    p = 100.0 * rng.standard_normal(N)
    P = 1e3 * rng.uniform(0.5, 1.5, len(d["out_ptr"]) - 1)
    return vd, v, p, P


def test_tangent_is_derivative_of_residual(small):
    """Central differences of the residual (tau frozen at the base state) along
    random directions of (vdot_{n+1}, pdot_{n+1}) -- which move vdot_{n+alpha_m}
    by alpha_m and (v, p)_{n+alpha_f} by alpha_f gamma dt -- equal the tangent
    applied to the direction, on the non-Dirichlet rows."""
    sp, d, m, ph = small
    N = d["n_nodes"]
    am, af, gm = oracle.gen_alpha(ph.rho_inf)
    c = af * gm * ph.dt
    vd, v, p, P = _state(d, 1)
    T = oracle.vms_assemble(m, d, ph, vd, v, p, P, vtau=v)
    K = oracle.dense_system(dict(d, A=T["A"], B=T["B"], C=T["C"], D=T["D"], r=np.zeros_like(d["r"])))[-1]
    free = np.concatenate([np.repeat(m["dir"] == 0, 3), np.ones(N, bool)])
    rng = np.random.default_rng(2)
    for _ in range(3):
        du = rng.standard_normal(4 * N) * free
        h = 1e-4
        def R(s):
            return oracle.vms_assemble(m, d, ph, vd + s * am * du[:3 * N], v + s * c * du[:3 * N],
                                       p + s * c * du[3 * N:], P, vtau=v, tangent=False)["R"]
        fd = (R(h) - R(-h)) / (2 * h)
        assert _rel(fd[free], (K @ du)[free]) <= 1e-6


def _boundary_flux(mesh, v):
    """int_{boundary} v . n from the boundary faces of the tets (faces that
    belong to one tet), n pointing away from that tet's fourth node: exact
    for P1 v (mean of the vertex values times area)."""
    X, tets = mesh["X"], mesh["tets"]
    faces = {}
    for e, t in enumerate(tets):
        for drop in range(4):
            f = tuple(sorted(np.delete(t, drop)))
            faces.setdefault(f, []).append(t[drop])
    flux = 0.0
    V = v.reshape(-1, 3)
    for f, opp in faces.items():
        if len(opp) != 1:
            continue
        a, b, cc = X[list(f)]
        n = np.cross(b - a, cc - a)
        if n @ (X[opp[0]] - a) > 0:
            n = -n
        flux += 0.5 * n @ V[list(f)].mean(axis=0)   # |n| = 2 area
    return flux


def test_continuity_rows_sum_to_boundary_flux(small):
    """Sum over A of R_p,A = int div v (the PSPG term drops out: sum_A grad N_A
    = 0) = the outward flux of v through the boundary (divergence theorem)."""
    sp, d, m, ph = small
    N = d["n_nodes"]
    vd, v, p, P = _state(d, 3)
    R = oracle.vms_assemble(m, d, ph, vd, v, p, P, tangent=False)["R"]
    flux = _boundary_flux(m, v)
    assert abs(R[3 * N:].sum() - flux) <= 1e-12 * np.abs(R[3 * N:]).sum()


def test_element_node_order_invariance(small):
    """The metric M makes G, hence tau_M and tau_C, independent of which
    vertex of a tet is the parent-domain origin (Sec. 2.3 remark): relabelling
    every tet's vertices leaves the residual and the tangent unchanged."""
    sp, d, m, ph = small
    vd, v, p, P = _state(d, 4)
    T0 = oracle.vms_assemble(m, d, ph, vd, v, p, P)
    rng = np.random.default_rng(5)
    tets = np.array([t[rng.permutation(4)] for t in m["tets"]], dtype=np.int32)
    T1 = oracle.vms_assemble(dict(m, tets=tets), d, ph, vd, v, p, P)
    for k in ("R", "A", "B", "C", "D"):
        assert np.abs(T1[k] - T0[k]).max() <= 1e-12 * np.abs(T0[k]).max()


def test_outlet_traction_enters_as_P_times_a(small):
    """R_m^bc = sum_k P_k a^k: the residual is affine in the outlet pressures
    with the outlet vectors as coefficients."""
    sp, d, m, ph = small
    N = d["n_nodes"]
    vd, v, p, P = _state(d, 6)
    R0 = oracle.vms_assemble(m, d, ph, vd, v, p, np.zeros_like(P), tangent=False)["R"]
    R1 = oracle.vms_assemble(m, d, ph, vd, v, p, P, tangent=False)["R"]
    ref = np.zeros(4 * N)
    for k in range(len(P)):
        for q in range(d["out_ptr"][k], d["out_ptr"][k + 1]):
            ref[d["out_idx"][q]] += P[k] * d["out_val"][q]
    assert np.abs((R1 - R0) - ref).max() <= 1e-12 * np.abs(ref).max()


def _rcr(d, seed=7):
    R = np.asarray(d["spec"].R)
    rng = np.random.default_rng(seed)
    return dict(Rp=0.1 * R, Rd=0.9 * R, C=1e-4 / R * 1e3, Pd=np.zeros(len(R)),
                Pi=rng.uniform(10.0, 50.0, len(R)), nts=10)


def test_newton_step_update_identity_and_convergence(small):
    """The accepted state satisfies the generalized-alpha relation
    y_{n+1} = y_n + dt ydot_n + gamma dt (ydot_{n+1} - ydot_n) (Sec. 2.4), its
    residual met the stopping rule, and the corrector contracts."""
    sp, d, m, ph = small
    N = d["n_nodes"]
    am, af, gm = oracle.gen_alpha(ph.rho_inf)
    rng = np.random.default_rng(8)
    y_n = np.concatenate([d["vel"], 10.0 * rng.standard_normal(N)])
    yd_n = np.concatenate([rng.standard_normal(3 * N) * np.repeat(m["dir"] == 0, 3), rng.standard_normal(N)])
    rc = _rcr(d)
    out = oracle.newton_step(m, d, ph, y_n, yd_n, rc, tol_R=1e-6, tol_A=1e-12, rtol=1e-10)
    lhs = out["y"] - y_n - ph.dt * yd_n - gm * ph.dt * (out["yd"] - yd_n)
    assert np.abs(lhs).max() <= 1e-12 * max(np.abs(y_n).max(), 1.0)
    assert out["iters"] >= 1
    assert out["res"][-1] <= 1e-6 * out["res"][0]
    # each corrector step reduces the residual at least tenfold
    assert all(b <= 0.1 * a for a, b in zip(out["res"], out["res"][1:]))
    # Dirichlet velocities keep their prescribed values
    dm = np.repeat(m["dir"] == 1, 3)
    assert np.array_equal(out["y"][:3 * N][dm], y_n[:3 * N][dm])


def test_newton_quadratic_from_consistent_start():
    """From a consistent start (outlet model at rest, uniform pressure equal
    to the outlet pressure, smooth Poiseuille velocity) each corrector
    roughly squares the relative residual, as Newton's method with the
    exact Jacobian of the residual does (tau held fixed: it moves little
    between correctors here), over successive time steps."""
    sp = synth.MeshSpec(4, 4, 12, Lz=3.0, Re=500.0, seed=2, R=(1e3,) * 4, pert=0.0, name="box4x4x12_eq")
    d, m, ph = synth.generate(sp), synth.mesh(sp), oracle.vms_phys(sp)
    N = d["n_nodes"]
    R = np.asarray(sp.R)
    Q0 = oracle.outlet_flows(d, d["vel"])
    rc = dict(Rp=0.1 * R, Rd=0.9 * R, C=0.1 / R, Pd=np.zeros(4), Pi=0.9 * R * Q0, nts=10)
    y = np.concatenate([d["vel"], np.full(N, float(np.mean(R * Q0)))])
    yd = np.zeros(4 * N)
    for _ in range(3):
        out = oracle.newton_step(m, d, ph, y, yd, rc, tol_R=1e-9, tol_A=1e-14, rtol=1e-12)
        res = np.asarray(out["res"])
        assert 2 <= out["iters"] <= 4
        rate = res[1:] / res[:-1]
        # a linearly convergent iteration keeps its rate; Newton's rate falls
        # with the residual itself (rate_{l+1} ~ K res_l / res_0; here by about
        # 1e-2 per corrector): at least tenfold
        for a, b in zip(rate[:-1], rate[1:]):
            assert b <= 0.1 * a
        y, yd, rc = out["y"], out["yd"], dict(rc, Pi=out["Pi"])


def test_lagged_preconditioner_keeps_the_newton_iterates():
    """A preconditioner built from an earlier tangent changes only the path of
    each nested solve, not its solution (Sec. 3: the outer FGMRES takes any
    preconditioner): over three time steps from a consistent start, one build
    for all steps (pc_rebuild 2) gives the same corrector counts and the same
    states, to the solve tolerance, as a build per tangent (pc_rebuild 0)."""
    sp = synth.MeshSpec(4, 4, 12, Lz=3.0, Re=500.0, seed=2, R=(1e3,) * 4, pert=0.0, name="box4x4x12_eq")
    d, m, ph = synth.generate(sp), synth.mesh(sp), oracle.vms_phys(sp)
    N = d["n_nodes"]
    R = np.asarray(sp.R)
    Q0 = oracle.outlet_flows(d, d["vel"])
    rc0 = dict(Rp=0.1 * R, Rd=0.9 * R, C=0.1 / R, Pd=np.zeros(4), Pi=0.9 * R * Q0, nts=10)
    y0 = np.concatenate([d["vel"], np.full(N, float(np.mean(R * Q0)))])
    runs = {}
    for mode in (0, 2):
        y, yd, rc, pc = y0.copy(), np.zeros(4 * N), dict(rc0), {}
        iters, setups = [], 0
        for _ in range(3):
            out = oracle.newton_step(m, d, ph, y, yd, rc, tol_R=1e-9, tol_A=1e-14, rtol=1e-12, pc_rebuild=mode, pc=pc)
            iters.append(out["iters"])
            setups += out["setups"]
            y, yd, rc = out["y"], out["yd"], dict(rc, Pi=out["Pi"])
        runs[mode] = (iters, setups, y, yd)
    assert runs[0][0] == runs[2][0]
    assert runs[2][1] == 1 and runs[0][1] == sum(runs[0][0])
    for a, b in zip(runs[0][2:], runs[2][2:]):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()


def test_numeric_resetup_keeps_the_newton_iterates():
    """A preconditioner rebuilt from each new tangent on the aggregates of the
    first build (pc_rebuild 3, every tangent; 4, the first tangent of each
    step) gives the same corrector counts and states, to the solve
    tolerance, as a full build per tangent (pc_rebuild 0); one full build in
    all, the rest numeric."""
    sp = synth.MeshSpec(4, 4, 12, Lz=3.0, Re=500.0, seed=2, R=(1e3,) * 4, pert=0.0, name="box4x4x12_eq")
    d, m, ph = synth.generate(sp), synth.mesh(sp), oracle.vms_phys(sp)
    N = d["n_nodes"]
    R = np.asarray(sp.R)
    Q0 = oracle.outlet_flows(d, d["vel"])
    rc0 = dict(Rp=0.1 * R, Rd=0.9 * R, C=0.1 / R, Pd=np.zeros(4), Pi=0.9 * R * Q0, nts=10)
    y0 = np.concatenate([d["vel"], np.full(N, float(np.mean(R * Q0)))])
    runs = {}
    for mode in (0, 3, 4):
        y, yd, rc, pc = y0.copy(), np.zeros(4 * N), dict(rc0), {}
        iters, setups, numeric = [], 0, 0
        for _ in range(3):
            out = oracle.newton_step(m, d, ph, y, yd, rc, tol_R=1e-9, tol_A=1e-14, rtol=1e-12, pc_rebuild=mode, pc=pc)
            iters.append(out["iters"])
            setups += out["setups"]
            numeric += out["numeric"]
            y, yd, rc = out["y"], out["yd"], dict(rc, Pi=out["Pi"])
        runs[mode] = (iters, setups, numeric, y, yd)
    assert runs[0][0] == runs[3][0] == runs[4][0]
    assert runs[3][1] == 1 and runs[3][2] == sum(runs[3][0]) - 1
    assert runs[4][1] == 1 and runs[4][2] == len(runs[4][0]) - 1
    for mode in (3, 4):
        for a, b in zip(runs[0][3:], runs[mode][3:]):
            assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()
