"""FP64 CPU oracle of the nested block preconditioned solve (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.

``nbp_oracle.c`` is plain C: its own block-sparse products, flexible GMRES
with modified Gram-Schmidt and Givens rotations, Algorithm 2 (matrix-free
Schur product), Algorithm 3 (P_SCR^{-1}), S_hat = D - C diag(A)^{-1} B, an
aggregation AMG and a dense LU.  ``dense_*`` helpers below build the same
operators as dense numpy arrays for the pins on tiny cases.

``vms_oracle.c`` is the residual of the VMS / generalized-alpha P1-P1
discretisation (Sec. 2.3-2.4) and its consistent tangent (Sec. 2.5), the
tangent taken exactly by dual numbers; ``newton_step`` below is the
predictor multi-corrector of Sec. 2.5 around the oracle's nested solve.

Parity status per function (see the pins in tests/test_oracle.py and
tests/test_vms_oracle.py):
  apply_A/apply_full .... pinned (dense products)
  solve (FGMRES+P_SCR) .. pinned (dense LU solve; exact-inner 1-iteration and
                          block-triangular 2-iteration closed forms)
  apply_S (Alg. 2) ...... pinned (dense D - C A^{-1} B)
  S_hat ................. pinned (dense formula)
  AMG aggregation ....... pinned (invariants: partition, size <= 8, strong
                          pairs; brute-force handshake on tiny graphs)
  Galerkin .............. pinned (dense P^T A P)
  Chebyshev ............. pinned (dense polynomial in D^{-1}A)
  V-cycle ............... pinned (two-level exact-coarse identity)
  VMS residual/tangent .. pinned (P1 mass/stiffness/divergence closed forms on
                          one element; the generator's analytic tangent;
                          central differences; the divergence theorem; node
                          order invariance of the metric G)
  newton_step ........... pinned (generalized-alpha update identity; the
                          residual of the accepted state below tolerance)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nbp_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "vms_oracle.c")]
_LIB_PATH = os.path.join(_HERE, "_nbp_oracle.so")
_lib = None


class Options(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double), ("rtol_A", ctypes.c_double), ("rtol_S", ctypes.c_double),
        ("rtol_I", ctypes.c_double), ("atol", ctypes.c_double),
        ("m", ctypes.c_int), ("m_A", ctypes.c_int), ("m_S", ctypes.c_int),
        ("nmax", ctypes.c_int), ("nmax_A", ctypes.c_int), ("nmax_S", ctypes.c_int),
        ("pc_A", ctypes.c_int), ("pc_S", ctypes.c_int), ("variant", ctypes.c_int),
        ("amg_max_levels", ctypes.c_int), ("amg_coarse_max", ctypes.c_int), ("cheb_degree", ctypes.c_int),
        ("theta", ctypes.c_double), ("amg_cycle", ctypes.c_int), ("amg_kdepth", ctypes.c_int),
        ("cheb_degree_S", ctypes.c_int), ("cheb_degree_I", ctypes.c_int),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("outer_iters", ctypes.c_int),
        ("A_iters", ctypes.c_longlong), ("S_iters", ctypes.c_longlong), ("I_iters", ctypes.c_longlong),
        ("n_A_solves", ctypes.c_longlong), ("n_I_solves", ctypes.c_longlong), ("n_S_solves", ctypes.c_longlong),
        ("rel_res_est", ctypes.c_double), ("rel_res_true", ctypes.c_double), ("status", ctypes.c_int),
    ]


class VmsPhys(ctypes.Structure):
    """Physical and stabilisation constants of the VMS residual (Sec. 2.3-2.4)."""
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
                ("rho_inf", ctypes.c_double), ("beta", ctypes.c_double), ("CI", ctypes.c_double),
                ("CT", ctypes.c_double)]


def vms_phys(spec, beta: float = 0.2) -> VmsPhys:
    """Constants of a generator spec: backflow beta = 0.2, C_I = 36, C_T = 4 (Sec. 2.3)."""
    return VmsPhys(spec.rho, spec.mu, spec.dt, spec.rho_inf, beta, 36.0, 4.0)


def gen_alpha(rho_inf: float):
    """(alpha_m, alpha_f, gamma) from rho_inf (Sec. 2.4.1)."""
    return 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf), 1.0 / (1.0 + rho_inf), 1.0 / (1.0 + rho_inf)


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no fused multiply-add; OpenMP over independent loops only, so
    results do not depend on the thread count)."""
    stale = not os.path.exists(_LIB_PATH) or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(f) for f in _SRCS)
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               *_SRCS, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        vp = ctypes.c_void_p
        lib.or_create.restype = vp
        lib.or_create.argtypes = [ctypes.c_int] + [_ip, _ip, _dp] * 4 + [ctypes.c_int, _ip, _ip, _dp, _dp]
        for name, args in [
            ("or_apply_A", [vp, _dp, _dp]), ("or_apply_B", [vp, _dp, _dp]), ("or_apply_C", [vp, _dp, _dp]),
            ("or_apply_D", [vp, _dp, _dp]), ("or_apply_full", [vp, _dp, _dp]), ("or_apply_S", [vp, _dp, _dp]),
            ("or_apply_pscr", [vp, _dp, _dp]), ("or_vcycle", [vp, ctypes.c_int, _dp, _dp]),
            ("or_vcycle_degree", [vp, ctypes.c_int, ctypes.c_int, _dp, _dp]),
            ("or_set_options", [vp, ctypes.POINTER(Options)]), ("or_get_options", [vp, ctypes.POINTER(Options)]),
            ("or_set_values", [vp, _dp, _dp, _dp, _dp]),
            ("or_default_options", [ctypes.POINTER(Options)]), ("or_set_resistances", [vp, _dp]),
            ("or_amg_level_get", [vp, ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, _ip]),
            ("or_shat_get", [vp, _ip, _ip, _dp]), ("or_diag_A", [vp, _dp]),
            ("or_get_info", [vp, ctypes.POINTER(Info)]), ("or_destroy", [vp]),
            ("or_chebyshev", [ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                              _dp, _dp, ctypes.c_int]),
            ("or_rcr_step", [ctypes.c_int] + [_dp] * 7 + [ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                                          ctypes.c_double, _dp, _dp, _dp]),
        ]:
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = None
        for name, args, rt in [
            ("or_setup", [vp], ctypes.c_int),
            ("or_setup_numeric", [vp], ctypes.c_int),
            ("or_solve", [vp, _dp, _dp, ctypes.POINTER(Info)], ctypes.c_int),
            ("or_solve_A", [vp, _dp, _dp, ctypes.c_double, _ip], ctypes.c_int),
            ("or_gmres_A", [vp, _dp, _dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _dp],
             ctypes.c_int),
            ("or_amg_nlev", [vp, ctypes.c_int], ctypes.c_int),
            ("or_amg_level_rows", [vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            ("or_amg_level_nnz", [vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
            ("or_amg_level_rho", [vp, ctypes.c_int, ctypes.c_int], ctypes.c_double),
            ("or_shat_nnz", [vp], ctypes.c_int),
            ("or_threads", [ctypes.c_int], ctypes.c_int),
            ("or_strength_and_aggregate", [ctypes.c_int, ctypes.c_int, _ip, _ip, _dp, ctypes.c_double, _ip],
             ctypes.c_int),
            ("or_vms_assemble", [ctypes.c_int, _dp, ctypes.c_int, _ip, ctypes.c_int, _ip, ctypes.c_void_p,
                                 ctypes.POINTER(VmsPhys), _dp, _dp, _dp, _dp, ctypes.c_int, _ip, _ip, _dp, _dp, _ip, _ip,
                                 _dp, _dp, _dp, _dp, _dp], ctypes.c_int),
        ]:
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = rt
        _lib = lib
    return _lib


def threads(n: int = 0) -> int:
    """Set the oracle's thread count when n > 0 (timing only: every result is
    the same at any count); returns the count in use."""
    return int(_load().or_threads(int(n)))


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _pd(a):
    return a.ctypes.data_as(_dp)


def _pi(a):
    return a.ctypes.data_as(_ip)


def default_options(**kw) -> Options:
    o = Options()
    _load().or_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Oracle:
    """FP64 CPU reference of the nested solve for one tangent (see module doc)."""

    def __init__(self, sysd: dict, **opts):
        lib = _load()
        self.lib = lib
        self.N = int(sysd["n_nodes"])
        N = self.N
        rp, col = _i(sysd["rowptr"]), _i(sysd["col"])
        pats = {}
        for key in ("A", "B", "C", "D"):
            pats[key] = (_i(sysd.get(key + "_rowptr", rp)), _i(sysd.get(key + "_col", col)), _d(sysd[key]).reshape(-1))
        self._keep = [pats, _i(sysd["out_ptr"]), _i(sysd["out_idx"]), _d(sysd["out_val"]), _d(sysd["r"])]
        optr, oidx, oval, r = self._keep[1:]
        self.n_out = len(optr) - 1
        args = [N]
        for key in ("A", "B", "C", "D"):
            a, b, c = pats[key]
            args += [_pi(a), _pi(b), _pd(c)]
        args += [self.n_out, _pi(optr), _pi(oidx), _pd(oval), _pd(r)]
        self.ctx = lib.or_create(*args)
        self._ready = False   # hierarchies built (setup) -- the solves need them
        self.set_options(**opts)

    def __del__(self):
        try:
            if getattr(self, "ctx", None):
                self.lib.or_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    # -- options / setup
    def options(self) -> Options:
        o = Options()
        self.lib.or_get_options(self.ctx, ctypes.byref(o))
        return o

    def set_options(self, **kw):
        o = self.options()
        for k, v in kw.items():
            setattr(o, k, v)
        self.lib.or_set_options(self.ctx, ctypes.byref(o))

    def set_resistances(self, r):
        r = _d(r)
        self.lib.or_set_resistances(self.ctx, _pd(r))

    def set_values(self, A, B, C, D):
        """New values of the tangent blocks on the same patterns; the built
        preconditioner is kept (a lagged preconditioner, see newton_step)."""
        vals = [_d(np.asarray(M).reshape(-1)) for M in (A, B, C, D)]
        self.lib.or_set_values(self.ctx, *[_pd(v) for v in vals])

    def setup(self):
        self.lib.or_setup(self.ctx)
        self._ready = True

    def setup_numeric(self):
        """Rebuild the preconditioner from the current values on the
        aggregates of the last setup() (numeric re-setup)."""
        if not self._ready or self.lib.or_setup_numeric(self.ctx) != 0:
            raise RuntimeError("setup_numeric needs an earlier setup()")

    def _ensure_setup(self):
        # the solves and cycles use the AMG hierarchies; building them on
        # first use keeps a forgotten setup() from reaching unbuilt data
        if not self._ready:
            self.setup()

    # -- operators
    def _apply(self, fn, x, n_out):
        x = _d(x)
        y = np.zeros(n_out)
        fn(self.ctx, _pd(x), _pd(y))
        return y

    def apply_A(self, x):
        return self._apply(self.lib.or_apply_A, x, 3 * self.N)

    def apply_B(self, x):
        return self._apply(self.lib.or_apply_B, x, 3 * self.N)

    def apply_C(self, x):
        return self._apply(self.lib.or_apply_C, x, self.N)

    def apply_D(self, x):
        return self._apply(self.lib.or_apply_D, x, self.N)

    def apply_full(self, x):
        return self._apply(self.lib.or_apply_full, x, 4 * self.N)

    def apply_S(self, x):
        """Algorithm 2 (builds the hierarchies first if setup() was not called)."""
        self._ensure_setup()
        return self._apply(self.lib.or_apply_S, x, self.N)

    def apply_pscr(self, s):
        """Algorithm 3 (builds the hierarchies first if setup() was not called)."""
        self._ensure_setup()
        return self._apply(self.lib.or_apply_pscr, s, 4 * self.N)

    def vcycle(self, which, b, degree=None):
        """One AMG cycle (0: AMG(A), 1: AMG(S_hat)); degree: its Chebyshev
        degree instead of the hierarchy's own."""
        self._ensure_setup()
        b = _d(b)
        x = np.zeros_like(b)
        if degree is None:
            self.lib.or_vcycle(self.ctx, which, _pd(b), _pd(x))
        else:
            self.lib.or_vcycle_degree(self.ctx, which, int(degree), _pd(b), _pd(x))
        return x

    def solve_A(self, b, rtol):
        self._ensure_setup()
        b = _d(b)
        x = np.zeros_like(b)
        its = ctypes.c_int(0)
        rc = self.lib.or_solve_A(self.ctx, _pd(b), _pd(x), rtol, ctypes.byref(its))
        return x, its.value, rc

    def gmres_A(self, b, rtol, m, nmax, use_pc):
        if use_pc:
            self._ensure_setup()
        b = _d(b)
        x = np.zeros_like(b)
        its = ctypes.c_int(0)
        rel = ctypes.c_double(0)
        rc = self.lib.or_gmres_A(self.ctx, _pd(b), _pd(x), rtol, m, nmax, int(use_pc), ctypes.byref(its),
                                 ctypes.byref(rel))
        return x, its.value, rel.value, rc

    def solve(self, b):
        self._ensure_setup()
        b = _d(b)
        x = np.zeros_like(b)
        info = Info()
        rc = self.lib.or_solve(self.ctx, _pd(b), _pd(x), ctypes.byref(info))
        return x, info, rc

    def info(self) -> Info:
        i = Info()
        self.lib.or_get_info(self.ctx, ctypes.byref(i))
        return i

    # -- introspection
    def diag_A(self):
        out = np.zeros(3 * self.N)
        self.lib.or_diag_A(self.ctx, _pd(out))
        return out

    def amg_levels(self, which=0):
        """List of dicts per level: rowptr, col, val (blocks), agg (to next level) and rho."""
        lib = self.lib
        out = []
        nl = lib.or_amg_nlev(self.ctx, which)
        bs = 3 if which == 0 else 1
        for l in range(nl):
            n = lib.or_amg_level_rows(self.ctx, which, l)
            nnz = lib.or_amg_level_nnz(self.ctx, which, l)
            rp = np.zeros(n + 1, np.int32)
            ci = np.zeros(nnz, np.int32)
            v = np.zeros(nnz * bs * bs)
            agg = np.full(n, -1, np.int32)
            lib.or_amg_level_get(self.ctx, which, l, _pi(rp), _pi(ci), _pd(v), _pi(agg))
            out.append(dict(rowptr=rp, col=ci, val=v.reshape(nnz, bs, bs) if bs > 1 else v,
                            agg=agg if l + 1 < nl else None, rho=lib.or_amg_level_rho(self.ctx, which, l)))
        return out

    def shat(self):
        nnz = self.lib.or_shat_nnz(self.ctx)
        rp = np.zeros(self.N + 1, np.int32)
        ci = np.zeros(nnz, np.int32)
        v = np.zeros(nnz)
        self.lib.or_shat_get(self.ctx, _pi(rp), _pi(ci), _pd(v))
        return rp, ci, v


def aggregate(rowptr, col, val, bs, theta):
    """Aggregation (3 handshake passes) of a block matrix; returns (n_agg, agg map)."""
    lib = _load()
    rp, ci, v = _i(rowptr), _i(col), _d(val).reshape(-1)
    n = len(rp) - 1
    agg = np.zeros(n, np.int32)
    nc = lib.or_strength_and_aggregate(n, bs, _pi(rp), _pi(ci), _pd(v), theta, _pi(agg))
    return nc, agg


def chebyshev(rowptr, col, val, bs, rho, k, b, x0=None, lodiv=10.0):
    """k Chebyshev steps on D_b^{-1} A over [rho / lodiv, rho]."""
    lib = _load()
    rp, ci, v = _i(rowptr), _i(col), _d(val).reshape(-1)
    n = len(rp) - 1
    b = _d(b)
    x = np.zeros(n * bs) if x0 is None else _d(x0).copy()
    lib.or_chebyshev(n, bs, _pi(rp), _pi(ci), _pd(v), rho, float(lodiv), k, _pd(b), _pd(x), int(x0 is None))
    return x


def rcr_step(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, dt, nts, eps_abs=1e-8, eps_rel=1e-5):
    """RCR outlets, one time step (Algorithm 1) and the difference-quotient
    stiffness m^k (Sec. 2.5).  Arrays of n_out values; returns
    (P_np1, Pi_np1, m)."""
    lib = _load()
    arrs = [_d(np.atleast_1d(a)) for a in (Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1)]
    n = len(arrs[0])
    assert all(len(a) == n for a in arrs)
    P, Pi, m = np.zeros(n), np.zeros(n), np.zeros(n)
    lib.or_rcr_step(n, *[_pd(a) for a in arrs], float(dt), int(nts), float(eps_abs), float(eps_rel), _pd(P), _pd(Pi),
                    _pd(m))
    return P, Pi, m


def outlet_flows(sysd: dict, v):
    """Q^k = a^k . v (the flow rate through outlet k, Sec. 2.5), v the 3N velocity dofs."""
    ptr, idx, val = sysd["out_ptr"], sysd["out_idx"], sysd["out_val"]
    v = _d(v)
    return np.array([float(np.dot(val[ptr[k]:ptr[k + 1]], v[idx[ptr[k]:ptr[k + 1]]])) for k in range(len(ptr) - 1)])


# --------------------------------------------------------------- dense forms
def dense_block(rowptr, col, val, br, bc, nbr, nbc):
    """Dense matrix of a block-sparse matrix (for tiny cases)."""
    M = np.zeros((nbr * br, nbc * bc))
    val = np.asarray(val).reshape(len(col), br, bc)
    for i in range(nbr):
        for e in range(rowptr[i], rowptr[i + 1]):
            j = col[e]
            M[i * br:(i + 1) * br, j * bc:(j + 1) * bc] += val[e]
    return M


def dense_system(sysd: dict):
    """Dense A (incl. rank-one terms), B, C, D and the full tangent (tiny cases only)."""
    N = int(sysd["n_nodes"])
    rp, col = sysd["rowptr"], sysd["col"]
    A = dense_block(sysd.get("A_rowptr", rp), sysd.get("A_col", col), sysd["A"], 3, 3, N, N)
    B = dense_block(sysd.get("B_rowptr", rp), sysd.get("B_col", col), sysd["B"], 3, 1, N, N)
    C = dense_block(sysd.get("C_rowptr", rp), sysd.get("C_col", col), sysd["C"], 1, 3, N, N)
    D = dense_block(sysd.get("D_rowptr", rp), sysd.get("D_col", col), sysd["D"], 1, 1, N, N)
    optr, oidx, oval, r = sysd["out_ptr"], sysd["out_idx"], sysd["out_val"], sysd["r"]
    for k in range(len(optr) - 1):
        v = np.zeros(3 * N)
        v[oidx[optr[k]:optr[k + 1]]] = oval[optr[k]:optr[k + 1]]
        A += r[k] * np.outer(v, v)
    full = np.block([[A, B], [C, D]])
    return A, B, C, D, full


def transpose_system(sysd: dict) -> dict:
    """The transposed tangent [[A^T, C^T], [B^T, D^T]] in the same input format
    (pattern per block), for the adjoint solve lambda = A^{-T} g."""
    N = int(sysd["n_nodes"])
    rp, col = sysd["rowptr"], sysd["col"]

    def tr_blocks(key, br, bc):
        r_ = np.asarray(sysd.get(key + "_rowptr", rp))
        c_ = np.asarray(sysd.get(key + "_col", col))
        data = np.asarray(sysd[key]).reshape(len(c_), br, bc)
        rows = np.repeat(np.arange(N), np.diff(r_))
        order = np.lexsort((rows, c_))          # new row = old col, then new col = old row
        new_rows = c_[order]
        new_cols = rows[order].astype(np.int32)
        new_data = np.transpose(data[order], (0, 2, 1)).copy()
        new_rp = np.zeros(N + 1, np.int32)
        np.add.at(new_rp, new_rows + 1, 1)
        new_rp = np.cumsum(new_rp).astype(np.int32)
        return new_rp, new_cols, new_data

    At = tr_blocks("A", 3, 3)
    Bt = tr_blocks("B", 3, 1)   # B^T: N x N blocks 1x3 -> plays C
    Ct = tr_blocks("C", 1, 3)   # C^T: blocks 3x1 -> plays B
    Dt = tr_blocks("D", 1, 1)
    t = dict(sysd)
    t["A_rowptr"], t["A_col"], t["A"] = At[0], At[1], At[2]
    t["B_rowptr"], t["B_col"], t["B"] = Ct[0], Ct[1], Ct[2].reshape(-1, 3)
    t["C_rowptr"], t["C_col"], t["C"] = Bt[0], Bt[1], Bt[2].reshape(-1, 3)
    t["D_rowptr"], t["D_col"], t["D"] = Dt[0], Dt[1], Dt[2].reshape(-1)
    return t


def adjoint(sysd: dict, g, x, **opts):
    """Adjoint of the nested solve: lambda = A^{-T} g by the same nested method
    on the transposed tangent [[A^T, C^T], [B^T, D^T]] (its Schur complement is
    S^T = D^T - B^T A^{-T} C^T, so Algorithms 2 and 3 apply unchanged), then
    dL/db = lambda and dL/dr_k = -(lambda_v . a^k)(a^k . x_v) since
    dA/dr_k = [[a^k a^kT, 0], [0, 0]] (Sec. 2.5, K term).
    Returns (lambda, dL/dr, info)."""
    t = transpose_system(sysd)
    o = Oracle(t, **opts)
    o.setup()
    lam, info, rc = o.solve(np.asarray(g, dtype=np.float64))
    N = int(sysd["n_nodes"])
    nv = 3 * N
    optr, oidx, oval = sysd["out_ptr"], sysd["out_idx"], sysd["out_val"]
    dLdr = np.zeros(len(optr) - 1)
    for k in range(len(optr) - 1):
        idx = oidx[optr[k]:optr[k + 1]]
        val = oval[optr[k]:optr[k + 1]]
        dLdr[k] = -(lam[:nv][idx] @ val) * (np.asarray(x)[:nv][idx] @ val)
    return lam, dLdr, info


# ------------------------------------------------- VMS residual and Newton step
def vms_assemble(mesh: dict, sysd: dict, phys: VmsPhys, vd, v, p, P=None, vtau=None, residual=True, tangent=True):
    """Residual R (4N) and/or tangent blocks at (vdot_{n+alpha_m}, v_{n+alpha_f},
    p_{n+alpha_f}) with outlet pressures P (P^k_{n+alpha_f}); tau at vtau (default v).
    Returns dict(R=..., A=(nnz,3,3), B=(nnz,3), C=(nnz,3), D=(nnz,))."""
    lib = _load()
    N = sysd["n_nodes"]
    rp, col = _i(sysd["rowptr"]), _i(sysd["col"])
    nnz = int(rp[N])
    X, tets, tris = _d(mesh["X"]).reshape(-1), _i(mesh["tets"]).reshape(-1), _i(mesh["tris"]).reshape(-1)
    dirn = np.ascontiguousarray(mesh["dir"], dtype=np.uint8)
    vd, v, p = _d(vd), _d(v), _d(p)
    vt = _d(vtau) if vtau is not None else None
    optr, oidx, oval = _i(sysd["out_ptr"]), _i(sysd["out_idx"]), _d(sysd["out_val"])
    n_out = len(optr) - 1
    Pk = _d(P) if P is not None else np.zeros(max(n_out, 1))
    out = {}
    R = np.zeros(4 * N) if residual else None
    A = np.zeros((nnz, 3, 3)) if tangent else None
    B = np.zeros((nnz, 3)) if tangent else None
    C = np.zeros((nnz, 3)) if tangent else None
    D = np.zeros(nnz) if tangent else None
    nul = ctypes.POINTER(ctypes.c_double)()
    rc = lib.or_vms_assemble(N, _pd(X), len(mesh["tets"]), _pi(tets), len(mesh["tris"]), _pi(tris),
                             dirn.ctypes.data_as(ctypes.c_void_p), ctypes.byref(phys), _pd(vd), _pd(v), _pd(p),
                             _pd(vt) if vt is not None else nul, n_out, _pi(optr), _pi(oidx), _pd(oval), _pd(Pk),
                             _pi(rp), _pi(col), _pd(R) if residual else nul, _pd(A) if tangent else nul,
                             _pd(B) if tangent else nul, _pd(C) if tangent else nul, _pd(D) if tangent else nul)
    if rc != 0:
        raise RuntimeError("or_vms_assemble: element couples nodes absent from the pattern")
    if residual:
        out["R"] = R
    if tangent:
        out.update(A=A, B=B, C=C, D=D)
    return out


def newton_step(mesh: dict, sysd: dict, phys: VmsPhys, y_n, yd_n, rcr: dict, tol_R=1e-6, tol_A=1e-6, l_max=20,
                pc_rebuild=0, pc=None, **solve_opts):
    """One time step by the predictor multi-corrector of Sec. 2.5 around the
    oracle's nested solve.  y = [v (3N); p (N)], yd its time derivative;
    rcr = dict(Rp, C, Rd, Pd, Pi, nts) per outlet (Pi = Pi^k_n).
    Readings: ||R_(0)|| is the residual at the predictor (the first residual
    evaluated); velocity increments at Dirichlet nodes are set to zero.
    Preconditioner of the nested solves (AMG(A), S_hat, AMG(S_hat)):
    pc_rebuild 0 builds it from every tangent; 1 from the first tangent of
    this step only; 2 keeps the one held in the caller's dict `pc` (key
    "oracle", from an earlier step) and builds one only if there is none; 3
    rebuilds it numerically (setup_numeric: new values on the held
    aggregates) from every tangent; 4 numerically from the first tangent of
    this step only.  Modes 2-4 build one in full when none is held.  A kept
    preconditioner is applied to the new tangent's operators (a lagged
    preconditioner: only the path of the solve changes, not its solution).
    Returns dict(y, yd, Pi, P, iters (linear solves), res (residual norms),
    setups (full preconditioner builds), numeric (numeric re-setups))."""
    N = sysd["n_nodes"]
    am, af, gm = gen_alpha(phys.rho_inf)
    dt = phys.dt
    y_n, yd_n = _d(y_n), _d(yd_n)
    dmask = np.repeat(np.asarray(mesh["dir"], dtype=bool), 3)
    y1 = y_n.copy()
    yd1 = (gm - 1.0) / gm * yd_n                                   # predictor
    n_out = len(sysd["out_ptr"]) - 1
    Rp, Cc, Rd, Pd = (np.asarray(rcr[k], dtype=np.float64) for k in ("Rp", "C", "Rd", "Pd"))
    Pi_n = np.asarray(rcr["Pi"], dtype=np.float64)
    Q_n = outlet_flows(sysd, y_n[:3 * N]) if n_out else np.zeros(0)
    P_n = Rp * Q_n + Pi_n + Pd
    res, r0, lin = [], None, []
    setups = numeric = 0
    held = pc if pc is not None else {}
    P1 = Pi1 = np.zeros(n_out)
    for l in range(1, l_max + 1):
        Q1 = outlet_flows(sysd, y1[:3 * N]) if n_out else np.zeros(0)                   # step 1
        if n_out:
            P1, Pi1, m = rcr_step(Rp, Cc, Rd, Pd, Pi_n, Q_n, Q1, dt, int(rcr["nts"]))   # steps 2-3
        else:
            m = np.zeros(0)
        yaf = y_n + af * (y1 - y_n)                                                      # step 4
        ydam = yd_n + am * (yd1 - yd_n)
        Paf = (1.0 - af) * P_n + af * P1                                                 # step 5
        R = vms_assemble(mesh, sysd, phys, ydam[:3 * N], yaf[:3 * N], yaf[3 * N:], Paf, tangent=False)["R"]  # 6
        nr = float(np.linalg.norm(R))
        res.append(nr)
        if r0 is None:
            r0 = nr
        if (r0 > 0 and nr / r0 <= tol_R) or nr <= tol_A:                                 # step 7
            return dict(y=y1, yd=yd1, Pi=Pi1, P=P1, iters=l - 1, res=res, lin=lin, setups=setups, numeric=numeric)
        T = vms_assemble(mesh, sysd, phys, ydam[:3 * N], yaf[:3 * N], yaf[3 * N:], Paf, residual=False)  # step 8
        r_k = af * gm * dt * m
        if pc_rebuild not in (0, 1, 2, 3, 4):
            raise ValueError("pc_rebuild must be 0-4")
        rebuild = pc_rebuild == 0 or (pc_rebuild == 1 and l == 1) or "oracle" not in held
        if rebuild:
            o = Oracle(dict(sysd, A=T["A"], B=T["B"], C=T["C"], D=T["D"], r=r_k), **solve_opts)
            o.setup()
            held["oracle"] = o
            setups += 1
        else:                                         # new operators on the held context
            o = held["oracle"]
            o.set_values(T["A"], T["B"], T["C"], T["D"])
            if n_out:
                o.set_resistances(r_k)
            if pc_rebuild == 3 or (pc_rebuild == 4 and l == 1):
                o.setup_numeric()                     # new values on the held aggregates
                numeric += 1
        dx, info, rc = o.solve(-R)                                                       # step 9
        if rc != 0:
            raise RuntimeError(f"newton_step: nested solve failed (status {rc})")
        lin.append(info.outer_iters)
        dx[:3 * N][dmask] = 0.0
        yd1 = yd1 + dx                                                                   # step 10
        y1 = y1 + gm * dt * dx
    raise RuntimeError("newton_step: no convergence in l_max corrector iterations")
