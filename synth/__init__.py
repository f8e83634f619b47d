"""Seeded synthetic inputs for the nested block solve (input data only).

The tangent [[A, B], [C, D]] of the P1-P1 residual-based VMS / generalized-alpha
discretisation (paper Sec. 2.3-2.5, definitions of A, B, C, D and of the
rank-one resistance term K = alpha_f gamma dt sum_k m^k a^k a^kT) is assembled
in C (``synth.c``) on a hex-to-tet box mesh and returned as numpy arrays:

    rowptr, col     shared node-graph pattern (int32), N rows
    A               (nnz, 3, 3) float64 row-major blocks (velocity-velocity)
    B               (nnz, 3)    float64 (velocity row dofs x pressure column)
    C               (nnz, 3)    float64 (pressure row x velocity column dofs)
    D               (nnz,)      float64
    out_ptr/out_idx/out_val     sparse outlet vectors a^k over velocity dofs
    r               (n_out,)    weights r_k = alpha_f gamma dt R_k multiplying
                                a^k a^kT in A (paper Sec. 2.5, the K term)
    b               (4N,)       right-hand side, uniform [-1, 1]

Unknown ordering: x = [x_v; x_p] with x_v node-interleaved (u, v, w per node),
which matches the 3x3 blocks of A.

This module holds none of the solver's arithmetic; the oracle and the CUDA path
both read its output.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB_PATH = os.path.join(_HERE, "_synth.so")
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("Re", ctypes.c_double), ("rho", ctypes.c_double), ("mu", ctypes.c_double),
        ("dt", ctypes.c_double), ("rho_inf", ctypes.c_double), ("pert", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("n_out", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile synth.c into an in-tree shared library (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.synth_num_nodes.argtypes = [P]; lib.synth_num_nodes.restype = ctypes.c_long
        lib.synth_pattern.argtypes = [P, ip, ip]; lib.synth_pattern.restype = ctypes.c_long
        lib.synth_state.argtypes = [P, dp]; lib.synth_state.restype = None
        lib.synth_assemble.argtypes = [P, dp, ip, ip, dp, dp, dp, dp, dp]; lib.synth_assemble.restype = ctypes.c_int
        lib.synth_rhs.argtypes = [P, dp]; lib.synth_rhs.restype = None
        lib.synth_outlets.argtypes = [P, ip, ip, dp]; lib.synth_outlets.restype = ctypes.c_long
        lib.synth_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_long, dp]; lib.synth_uniforms.restype = None
        lib.synth_element_tangent.argtypes = [P, dp, dp, dp]; lib.synth_element_tangent.restype = None
        lib.synth_backflow_tangent.argtypes = [P, dp, dp, dp]; lib.synth_backflow_tangent.restype = None
        u8 = ctypes.POINTER(ctypes.c_uint8)
        lib.synth_mesh.argtypes = [P, dp, ip, ip, ip, u8]; lib.synth_mesh.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


@dataclass
class MeshSpec:
    """One synthetic tangent: box mesh, flow parameters, outlets, seed."""
    nx: int
    ny: int
    nz: int
    Lx: float = 1.0
    Ly: float = 1.0
    Lz: float = 1.0
    Re: float = 100.0
    rho: float = 1.06
    mu: float = 0.04
    dt: float = 1e-3
    rho_inf: float = 0.5
    pert: float = 0.05
    seed: int = 0
    R: tuple = (1e3,)            # physical outlet resistances R^k
    name: str = ""

    @property
    def n_out(self) -> int:
        return len(self.R)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    def params(self) -> _Params:
        return _Params(self.nx, self.ny, self.nz, self.Lx, self.Ly, self.Lz, self.Re, self.rho,
                       self.mu, self.dt, self.rho_inf, self.pert, self.seed & (2**64 - 1), self.n_out)

    @property
    def alpha_f_gamma_dt(self) -> float:
        af = 1.0 / (1.0 + self.rho_inf)
        return af * af * self.dt


def uniforms(seed: int, n: int) -> np.ndarray:
    """n SplitMix64 uniforms in [0, 1) from `seed` (same generator as synth.c)."""
    out = np.empty(n, dtype=np.float64)
    _load().synth_uniforms(ctypes.c_uint64(seed & (2**64 - 1)), n, _dp(out))
    return out


def generate(spec: MeshSpec) -> dict:
    """Assemble the tangent, outlet vectors and right-hand side for `spec`."""
    lib = _load()
    p = spec.params()
    N = lib.synth_num_nodes(ctypes.byref(p))
    nnz = lib.synth_pattern(ctypes.byref(p), None, None)
    rowptr = np.empty(N + 1, dtype=np.int32)
    col = np.empty(nnz, dtype=np.int32)
    lib.synth_pattern(ctypes.byref(p), _ip(rowptr), _ip(col))
    vel = np.empty(3 * N, dtype=np.float64)
    lib.synth_state(ctypes.byref(p), _dp(vel))
    A = np.empty((nnz, 3, 3), dtype=np.float64)
    B = np.empty((nnz, 3), dtype=np.float64)
    C = np.empty((nnz, 3), dtype=np.float64)
    D = np.empty(nnz, dtype=np.float64)
    rc = lib.synth_assemble(ctypes.byref(p), _dp(vel), _ip(rowptr), _ip(col), _dp(A), _dp(B), _dp(C), _dp(D), None)
    if rc != 0:
        raise RuntimeError("synth_assemble: element node missing from pattern")
    b = np.empty(4 * N, dtype=np.float64)
    lib.synth_rhs(ctypes.byref(p), _dp(b))
    out_ptr, out_idx, out_val = outlets(spec)
    r = np.asarray(spec.R, dtype=np.float64) * spec.alpha_f_gamma_dt
    return dict(
        spec=spec, n_nodes=N, rowptr=rowptr, col=col, A=A, B=B, C=C, D=D, vel=vel,
        out_ptr=out_ptr, out_idx=out_idx, out_val=out_val, r=r, b=b,
    )


def mesh(spec: MeshSpec) -> dict:
    """Explicit mesh arrays of the box: X (N, 3) coordinates, tets (E, 4) node
    ids, outlet triangles tris (T, 3) on z = Lz (outward +e_z orientation) with
    their outlet piece tri_out (T,), and the Dirichlet flag dir (N,) of every
    node (walls and inlet: velocity prescribed)."""
    lib = _load()
    p = spec.params()
    N = spec.n_nodes
    E = 6 * spec.nx * spec.ny * spec.nz
    T = 2 * spec.nx * spec.ny
    X = np.empty((N, 3), dtype=np.float64)
    tets = np.empty((E, 4), dtype=np.int32)
    tris = np.empty((T, 3), dtype=np.int32)
    tri_out = np.empty(T, dtype=np.int32)
    dirn = np.empty(N, dtype=np.uint8)
    lib.synth_mesh(ctypes.byref(p), _dp(X), _ip(tets), _ip(tris), _ip(tri_out),
                   dirn.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return dict(X=X, tets=tets, tris=tris, tri_out=tri_out, dir=dirn)


def outlets(spec: MeshSpec):
    """Sparse outlet vectors a^k (out_ptr, out_idx, out_val) of `spec`."""
    lib = _load()
    p = spec.params()
    out_ptr = np.zeros(spec.n_out + 1, dtype=np.int32)
    cnt = lib.synth_outlets(ctypes.byref(p), _ip(out_ptr), None, None)
    if cnt < 0:
        raise ValueError("synth_outlets: more outlets than outlet triangles")
    out_idx = np.zeros(cnt, dtype=np.int32)
    out_val = np.zeros(cnt, dtype=np.float64)
    lib.synth_outlets(ctypes.byref(p), _ip(out_ptr), _ip(out_idx), _dp(out_val))
    return out_ptr, out_idx, out_val


def outlets_dense(spec: MeshSpec) -> np.ndarray:
    """Dense outlet vectors (n_out, 3N) as assembled with the tangent (tests)."""
    lib = _load()
    p = spec.params()
    N = lib.synth_num_nodes(ctypes.byref(p))
    nnz = lib.synth_pattern(ctypes.byref(p), None, None)
    rowptr = np.empty(N + 1, dtype=np.int32)
    col = np.empty(nnz, dtype=np.int32)
    lib.synth_pattern(ctypes.byref(p), _ip(rowptr), _ip(col))
    vel = np.empty(3 * N, dtype=np.float64)
    lib.synth_state(ctypes.byref(p), _dp(vel))
    A = np.empty((nnz, 3, 3)); B = np.empty((nnz, 3)); C = np.empty((nnz, 3)); D = np.empty(nnz)
    avec = np.empty((max(spec.n_out, 1), 3 * N), dtype=np.float64)
    lib.synth_assemble(ctypes.byref(p), _dp(vel), _ip(rowptr), _ip(col), _dp(A), _dp(B), _dp(C), _dp(D), _dp(avec))
    return avec[:spec.n_out]


def element_tangent(spec: MeshSpec, X: np.ndarray, vel: np.ndarray) -> np.ndarray:
    """16x16 tangent of one tet (dofs ordered node-major, u v w p)."""
    K = np.empty(256, dtype=np.float64)
    p = spec.params()
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(12)
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(12)
    _load().synth_element_tangent(ctypes.byref(p), _dp(X), _dp(vel), _dp(K))
    return K.reshape(16, 16)


def backflow_tangent(spec: MeshSpec, X: np.ndarray, vel: np.ndarray) -> np.ndarray:
    """9x9 backflow tangent of one outlet triangle (n = +e_z)."""
    K = np.empty(81, dtype=np.float64)
    p = spec.params()
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(9)
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(9)
    _load().synth_backflow_tangent(ctypes.byref(p), _dp(X), _dp(vel), _dp(K))
    return K.reshape(9, 9)


# ----------------------------------------------------------------- workloads
def tiny(seed: int = 0) -> MeshSpec:
    """Unit cube, 8x8x8 hexes x 6 tets (729 nodes, 2916 unknowns), Re 100, one outlet R = 1e3."""
    return MeshSpec(8, 8, 8, Re=100.0, seed=seed, R=(1e3,), name="cube8_re100")


def large_fp64(scale: int = 64) -> MeshSpec:
    """Box 1x1x4, 64x64x256 hexes (1,085,825 nodes, 4,343,300 unknowns), Re 500, one outlet R = 1e3."""
    return MeshSpec(scale, scale, 4 * scale, Lz=4.0, Re=500.0, seed=1, R=(1e3,), name=f"box{scale}x{scale}x{4*scale}_re500")


def large_mixed(scale: int = 64) -> MeshSpec:
    """Same 4.34M-unknown box at Re 2000 with 4 quadrant outlets, R_k log-uniform in [1e2, 1e5]."""
    u = uniforms(2 ^ 0x5EED, 4)
    R = tuple(float(10.0 ** (2.0 + 3.0 * x)) for x in u)
    return MeshSpec(scale, scale, 4 * scale, Lz=4.0, Re=2000.0, seed=2, R=R, name=f"box{scale}x{scale}x{4*scale}_re2000_q4")


def adjoint_case(scale: int = 32) -> MeshSpec:
    """Box 1x1x4, 32x32x128 hexes (140,481 nodes), Re 300, 4 outlets, R_k log-uniform in [1e2, 1e4]."""
    u = uniforms(4 ^ 0x5EED, 4)
    R = tuple(float(10.0 ** (2.0 + 2.0 * x)) for x in u)
    return MeshSpec(scale, scale, 4 * scale, Lz=4.0, Re=300.0, seed=4, R=R, name=f"box{scale}x{scale}x{4*scale}_re300_q4")


def batch(count: int = 48, seed: int = 3, smin: int = 12, smax: int = 40) -> list:
    """`count` unit cubes with s^3 hexes, s = smin + floor((smax-smin+1) u), Re ~ U[100, 1000],
    n_out ~ U{1..4}, R_k log-uniform in [1e2, 1e4]."""
    u = uniforms(seed ^ 0x5EED, 8 * count)
    out = []
    for i in range(count):
        s = smin + int((smax - smin + 1) * u[8 * i])
        s = min(s, smax)
        Re = 100.0 + 900.0 * u[8 * i + 1]
        n_out = 1 + min(3, int(4 * u[8 * i + 2]))
        R = tuple(float(10.0 ** (2.0 + 2.0 * u[8 * i + 3 + k])) for k in range(n_out))
        out.append(MeshSpec(s, s, s, Re=Re, seed=seed * 1000 + i, R=R, name=f"cube{s}_re{Re:.0f}_o{n_out}"))
    return out
