"""Input generator checks: mesh sizes of the workloads and the tangent against
central finite differences of the VMS element residual (paper Sec. 2.3, 2.5).

These pin the *inputs*; the generator holds none of the solver's arithmetic."""
import numpy as np
import pytest

import synth


def _residual(spec, X, vel0, vdot, v, p):
    """Momentum (4x3) and continuity (4) residual of one P1 tet with tau_M,
    tau_C frozen at the state vel0 (paper Sec. 2.3, B_m^vol and B_p)."""
    rho, mu, dt = spec.rho, spec.mu, spec.dt
    J = (X[1:] - X[0]).T
    inv = np.linalg.inv(J)
    dN = np.vstack([-inv.sum(axis=0), inv])          # (4, 3): grad N_b
    vol = abs(np.linalg.det(J)) / 6.0
    M = 2 ** (1 / 3) / 2 * (np.ones((3, 3)) + np.eye(3))
    G = inv.T @ M @ inv
    qa, qb = 0.5854101966249685, 0.1381966011250105
    Rm = np.zeros((4, 3), dtype=v.dtype)
    Rp = np.zeros(4, dtype=v.dtype)
    gv = v.T @ dN                                    # (3,3): d v_i / d x_j
    divv = np.trace(gv)
    gp = dN.T @ p
    for q in range(4):
        N = np.full(4, qb); N[q] = qa
        w = vol / 4
        a0 = N @ vel0
        tauM = 1.0 / (rho * np.sqrt(4.0 / dt**2 + a0 @ G @ a0 + 36.0 * (mu / rho) ** 2 * np.sum(G * G)))
        tauC = 1.0 / (tauM * np.trace(G))
        vq = N @ v
        vdq = N @ vdot
        pq = N @ p
        conv = gv @ vq                                # (v . grad) v
        vp = -tauM * (rho * vdq + rho * conv + gp)
        for a in range(4):
            for i in range(3):
                t = rho * N[a] * (vdq[i] + conv[i]) - dN[a, i] * pq
                t += mu * (dN[a] @ gv[i] + dN[a] @ gv[:, i])
                t += -rho * (vq @ dN[a]) * vp[i] + rho * N[a] * (gv[i] @ vp) - rho * (vp @ dN[a]) * vp[i]
                t += tauC * dN[a, i] * divv
                Rm[a, i] += w * t
            Rp[a] += w * (N[a] * divv - dN[a] @ vp)
    return Rm, Rp


def test_element_tangent_matches_fd_of_residual():
    spec = synth.MeshSpec(4, 4, 4, Re=300.0)
    rng = np.random.default_rng(7)
    X = np.array([[0, 0, 0], [0.3, 0.05, 0], [0.02, 0.25, 0.04], [0.05, 0.07, 0.28]]) + rng.uniform(0, 0.02, (4, 3))
    vel0 = rng.uniform(-2, 2, (4, 3))
    K = synth.element_tangent(spec, X, vel0)
    af = 1 / (1 + spec.rho_inf)
    am = 0.5 * (3 - spec.rho_inf) / (1 + spec.rho_inf)
    c = af * af * spec.dt
    h = 1e-4  # residual is a polynomial of degree 4 in v: rounding dominates below this
    Kfd = np.zeros((16, 16))
    zero3 = np.zeros((4, 3)); zero1 = np.zeros(4)
    for b in range(4):
        for j in range(4):
            col = 4 * b + j
            def R(vd, v, p):
                Rm, Rp = _residual(spec, X, vel0, vd, v, p)
                return np.concatenate([np.hstack([Rm, Rp[:, None]]).reshape(-1)])
            if j < 3:
                E = np.zeros((4, 3)); E[b, j] = h
                dv = (R(zero3, vel0 + E, zero1) - R(zero3, vel0 - E, zero1)) / (2 * h)
                dvd = (R(E, vel0, zero1) - R(-E, vel0, zero1)) / (2 * h)
                Kfd[:, col] = am * dvd + c * dv
            else:
                E = np.zeros(4); E[b] = h
                Kfd[:, col] = c * (R(zero3, vel0, E) - R(zero3, vel0, -E)) / (2 * h)
    # rows: (a, d) with d<3 momentum, d=3 continuity -- same layout as K
    scale = np.abs(Kfd).max()
    assert np.abs(K - Kfd).max() <= 1e-7 * scale


def test_backflow_tangent_matches_fd():
    spec = synth.MeshSpec(4, 4, 4)
    X = np.array([[0, 0, 1.0], [0.25, 0, 1.0], [0.25, 0.25, 1.0]])
    vel0 = np.array([[0.1, -0.2, -0.5], [0.0, 0.1, -0.3], [0.2, 0.0, -0.1]])  # inflow: a.n < 0
    K = synth.backflow_tangent(spec, X, vel0)
    c = (1 / (1 + spec.rho_inf)) ** 2 * spec.dt

    def Rbf(v):
        e1, e2 = X[1] - X[0], X[2] - X[0]
        area = 0.5 * np.linalg.norm(np.cross(e1, e2))
        out = np.zeros((3, 3))
        for q in range(3):
            N = np.full(3, 1 / 6); N[q] = 2 / 3
            vq = N @ v
            vn = vq[2]
            neg = 0.5 * (vn - abs(vn))
            for a in range(3):
                out[a] += area / 3 * (-spec.rho * 0.2 * neg * N[a] * vq)
        return out.reshape(-1)
    h = 1e-5
    Kfd = np.zeros((9, 9))
    for col in range(9):
        E = np.zeros(9); E[col] = h
        Kfd[:, col] = c * (Rbf(vel0 + E.reshape(3, 3)) - Rbf(vel0 - E.reshape(3, 3))) / (2 * h)
    assert np.abs(K - Kfd).max() <= 1e-7 * np.abs(Kfd).max()


def test_workload_sizes():
    assert synth.tiny().n_nodes == 729
    assert 4 * synth.tiny().n_nodes == 2916
    big = synth.large_fp64()
    assert big.n_nodes == 65 * 65 * 257 == 1_085_825
    assert 4 * big.n_nodes == 4_343_300
    assert synth.adjoint_case().n_nodes == 33 * 33 * 129
    sizes = [s.nx for s in synth.batch()]
    assert len(sizes) == 48 and min(sizes) >= 12 and max(sizes) <= 40


def test_tiny_tangent_structure():
    d = synth.generate(synth.tiny())
    N = d["n_nodes"]
    rp, col = d["rowptr"], d["col"]
    deg = np.diff(rp)
    assert deg.max() == 15 and deg.min() >= 4
    # interior node has 15 blocks; pattern symmetric and sorted
    S = set()
    for i in range(N):
        cols = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(cols) > 0)
        S.update((i, int(j)) for j in cols)
    assert all((j, i) in S for (i, j) in S)
    assert d["out_ptr"][-1] == 7 * 7  # interior outlet nodes of the 9x9 top face
    assert np.all(np.isfinite(d["A"])) and np.all(np.isfinite(d["b"]))
    assert np.all(np.abs(d["b"]) <= 1.0)


def test_no_outlet_spec():
    """A spec without outlets gives empty outlet arrays (and no stray writes)."""
    d = synth.generate(synth.MeshSpec(5, 6, 7, R=(), name="box5x6x7_o0"))
    assert list(d["out_ptr"]) == [0] and len(d["out_idx"]) == 0 and len(d["r"]) == 0
