"""ctypes binding of libnbp (include/nbp.h): argument marshalling only.

Every function of the C ABI is exposed under its own name; ``Solver`` wraps
one context for a tangent given as numpy arrays (the format of the ``synth``
package: shared or per-block patterns, outlet vectors, weights r_k) and moves
them to device memory with PyTorch.  All arithmetic of the method runs in the
library's CUDA kernels; there is no fallback: without the built library or a
CUDA device every call raises.
"""
from __future__ import annotations

import ctypes
import os
import weakref

import numpy as np

from . import build as _build

_lib = None


class nbp_system(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32)] + [
        (f"{b}_{f}", t) for b in "abcd" for f, t in (("rowptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
                                                     ("val", ctypes.c_void_p))
    ] + [("n_out", ctypes.c_int32), ("out_ptr", ctypes.c_void_p), ("out_idx", ctypes.c_void_p),
         ("out_val", ctypes.c_void_p), ("r", ctypes.c_void_p)]


class nbp_options(ctypes.Structure):
    _fields_ = [
        ("rtol", ctypes.c_double), ("rtol_A", ctypes.c_double), ("rtol_S", ctypes.c_double),
        ("rtol_I", ctypes.c_double), ("atol", ctypes.c_double),
        ("m", ctypes.c_int32), ("m_A", ctypes.c_int32), ("m_S", ctypes.c_int32),
        ("nmax", ctypes.c_int32), ("nmax_A", ctypes.c_int32), ("nmax_S", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("pc_A", ctypes.c_int32), ("pc_S", ctypes.c_int32),
        ("variant", ctypes.c_int32), ("amg_max_levels", ctypes.c_int32), ("amg_coarse_max", ctypes.c_int32),
        ("cheb_degree", ctypes.c_int32), ("theta", ctypes.c_double), ("amg_cycle", ctypes.c_int32),
        ("amg_kdepth", ctypes.c_int32), ("cheb_degree_S", ctypes.c_int32), ("device_loop", ctypes.c_int32),
        ("cheb_degree_I", ctypes.c_int32), ("gs_passes_I", ctypes.c_int32),
    ]


class nbp_info(ctypes.Structure):
    _fields_ = [
        ("outer_iters", ctypes.c_int32),
        ("A_iters", ctypes.c_int64), ("S_iters", ctypes.c_int64), ("I_iters", ctypes.c_int64),
        ("n_A_solves", ctypes.c_int64), ("n_I_solves", ctypes.c_int64), ("n_S_solves", ctypes.c_int64),
        ("rel_res_est", ctypes.c_double), ("rel_res_true", ctypes.c_double),
        ("setup_s", ctypes.c_double), ("solve_s", ctypes.c_double), ("status", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nbp_profile_info(ctypes.Structure):
    _fields_ = [
        ("spmv_ms", ctypes.c_double), ("spmv_bytes", ctypes.c_double),
        ("arnoldi_ms", ctypes.c_double), ("arnoldi_bytes", ctypes.c_double),
        ("a0_ms", ctypes.c_double), ("a0_bytes", ctypes.c_double),
        ("cheb0_ms", ctypes.c_double), ("cheb0_bytes", ctypes.c_double),
        ("vcycle_ms", ctypes.c_double),
        ("spmv_launches", ctypes.c_int64), ("arnoldi_launches", ctypes.c_int64), ("a0_launches", ctypes.c_int64),
        ("cheb0_launches", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("host_wait_s", ctypes.c_double), ("host_syncs", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class nbp_rcr(ctypes.Structure):
    _fields_ = [("Rp", ctypes.c_void_p), ("C", ctypes.c_void_p), ("Rd", ctypes.c_void_p), ("Pd", ctypes.c_void_p),
                ("Pi_n", ctypes.c_void_p), ("Q_n", ctypes.c_void_p), ("eps_abs", ctypes.c_double),
                ("eps_rel", ctypes.c_double)]


class nbp_mesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("n_tets", ctypes.c_int32), ("n_tris", ctypes.c_int32),
                ("X", ctypes.c_void_p), ("tets", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("dir", ctypes.c_void_p)]


class nbp_vms_params(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
                ("rho_inf", ctypes.c_double), ("beta", ctypes.c_double), ("CI", ctypes.c_double),
                ("CT", ctypes.c_double), ("tangent_fp32", ctypes.c_int32)]


class nbp_newton_opts(ctypes.Structure):
    _fields_ = [("tol_R", ctypes.c_double), ("tol_A", ctypes.c_double), ("l_max", ctypes.c_int32),
                ("nts", ctypes.c_int32), ("pc_rebuild", ctypes.c_int32)]


class nbp_newton_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("unconverged_solves", ctypes.c_int32),
                ("res0", ctypes.c_double), ("res", ctypes.c_double),
                ("outer_iters", ctypes.c_int64), ("A_iters", ctypes.c_int64), ("S_iters", ctypes.c_int64),
                ("I_iters", ctypes.c_int64), ("residual_s", ctypes.c_double), ("tangent_s", ctypes.c_double),
                ("setup_s", ctypes.c_double), ("solve_s", ctypes.c_double), ("total_s", ctypes.c_double),
                ("setups", ctypes.c_int32), ("numeric_setups", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


STATUS = {0: "NBP_OK", 1: "NBP_ERR_INVALID", 2: "NBP_ERR_CUDA", 3: "NBP_ERR_OOM", 4: "NBP_NOT_CONVERGED",
          5: "NBP_ERR_BREAKDOWN", 6: "NBP_ERR_NAN", 7: "NBP_ERR_TIMEOUT", 8: "NBP_ERR_STATE"}

# name -> (restype, argtypes)
_vp, _i32, _i64, _d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
SIGNATURES = {
    "nbp_default_options": (None, [ctypes.POINTER(nbp_options)]),
    "nbp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(nbp_system), ctypes.POINTER(nbp_options), _vp]),
    "nbp_setup": (ctypes.c_int, [_vp]),
    "nbp_setup_numeric": (ctypes.c_int, [_vp]),
    "nbp_set_resistances": (ctypes.c_int, [_vp, ctypes.POINTER(_d)]),
    "nbp_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(nbp_options), ctypes.POINTER(nbp_info)]),
    "nbp_solve_host": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(nbp_options), ctypes.POINTER(nbp_info)]),
    "nbp_adjoint": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(_d), ctypes.POINTER(nbp_info)]),
    "nbp_destroy": (ctypes.c_int, [_vp]),
    "nbp_last_error": (ctypes.c_char_p, [_vp]),
    "nbp_apply_A": (ctypes.c_int, [_vp, _vp, _vp, _i32]),
    "nbp_apply_full": (ctypes.c_int, [_vp, _vp, _vp]),
    "nbp_apply_S": (ctypes.c_int, [_vp, _vp, _vp]),
    "nbp_apply_pscr": (ctypes.c_int, [_vp, _vp, _vp]),
    "nbp_solve_A": (ctypes.c_int, [_vp, _vp, _vp, _d, ctypes.POINTER(_i32)]),
    "nbp_vcycle": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "nbp_amg_level_sizes": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i64), _i32]),
    "nbp_amg_level_get": (ctypes.c_int, [_vp, _i32, _i32, _vp, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "nbp_shat_nnz": (_i64, [_vp]),
    "nbp_shat_get": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "nbp_profile": (ctypes.c_int, [_vp, _i32]),
    "nbp_profile_get": (ctypes.c_int, [_vp, ctypes.POINTER(nbp_profile_info)]),
    "nbp_profile_report": (ctypes.c_char_p, [_vp]),
    "nbp_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(nbp_system), ctypes.POINTER(nbp_options)]),
    "nbp_batch_setup": (ctypes.c_int, [_vp]),
    "nbp_batch_solve": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(nbp_options),
                                       ctypes.POINTER(nbp_info)]),
    "nbp_batch_size": (_i32, [_vp]),
    "nbp_batch_destroy": (ctypes.c_int, [_vp]),
    "nbp_batch_last_error": (ctypes.c_char_p, [_vp]),
    "nbp_apply_A_noalloc": (ctypes.c_int, [_i32, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "nbp_rcr_step": (ctypes.c_int, [_i32, ctypes.POINTER(nbp_rcr), _vp, _d, _i32, _vp, _vp, _vp, _vp]),
    "nbp_outlet_flows": (ctypes.c_int, [_vp, _vp, _vp]),
    "nbp_rcr_update": (ctypes.c_int, [_vp, ctypes.POINTER(nbp_rcr), _vp, _d, _i32, _d, _vp, _vp, _vp, _vp]),
    "nbp_set_values": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "nbp_vms_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, ctypes.POINTER(nbp_mesh), ctypes.POINTER(nbp_vms_params)]),
    "nbp_vms_destroy": (ctypes.c_int, [_vp]),
    "nbp_vms_maps": (ctypes.c_int, [_i32, _vp, _vp, _i32, _i32, _vp, _vp, _vp, _vp, _vp]),
    "nbp_vms_residual": (ctypes.c_int, [_vp] * 7),
    "nbp_vms_tangent": (ctypes.c_int, [_vp] * 9),
    "nbp_newton_step": (ctypes.c_int, [_vp, ctypes.POINTER(nbp_rcr), _vp, _vp, _vp, _vp, _vp,
                                       ctypes.POINTER(nbp_newton_opts), ctypes.POINTER(nbp_newton_info)]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libnbp.so (building it in-tree when missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libnbp.so is not built; run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (rt, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = rt
            f.argtypes = args
        _lib = lib
    return _lib


class NbpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def default_options(**kw) -> nbp_options:
    o = nbp_options()
    load().nbp_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _optr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def rcr_params(Rp, C, Rd, Pd, Pi_n, Q_n, eps_abs=1e-8, eps_rel=1e-5) -> nbp_rcr:
    """nbp_rcr over CUDA float64 tensors (n_out each); keep the tensors alive
    while the structure is used."""
    p = nbp_rcr()
    p.Rp, p.C, p.Rd, p.Pd, p.Pi_n, p.Q_n = (t.data_ptr() for t in (Rp, C, Rd, Pd, Pi_n, Q_n))
    p.eps_abs, p.eps_rel = float(eps_abs), float(eps_rel)
    return p


def rcr_step(Rp, C, Rd, Pd, Pi_n, Q_n, Q_np1, dt, nts, eps_abs=1e-8, eps_rel=1e-5, stream=None):
    """One RCR time step of n_out outlets on the GPU (nbp_rcr_step); CUDA
    float64 tensors in, (P_np1, Pi_np1, m) out (stream-ordered, not synchronised)."""
    import torch
    n = Q_np1.numel()
    P, Pi, m = (torch.empty(n, dtype=torch.float64, device=Q_np1.device) for _ in range(3))
    p = rcr_params(Rp, C, Rd, Pd, Pi_n, Q_n, eps_abs, eps_rel)
    s = stream if stream is not None else torch.cuda.current_stream(Q_np1.device)
    st = load().nbp_rcr_step(n, ctypes.byref(p), _ptr(Q_np1), float(dt), int(nts), _ptr(P), _ptr(Pi), _ptr(m),
                             ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise NbpError(st, "nbp_rcr_step failed")
    return P, Pi, m


def _system(sysd, dev, keep):
    """nbp_system for a tangent in the synth format; device copies appended to keep."""
    import torch

    def put(a, dt):
        t = torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(dev)
        keep.append(t)
        return t

    rp, col = sysd["rowptr"], sysd["col"]
    s = nbp_system()
    s.n_nodes = int(sysd["n_nodes"])
    for key in "ABCD":
        k = key.lower()
        setattr(s, f"{k}_rowptr", put(sysd.get(key + "_rowptr", rp), torch.int32).data_ptr())
        setattr(s, f"{k}_col", put(sysd.get(key + "_col", col), torch.int32).data_ptr())
        setattr(s, f"{k}_val", put(np.asarray(sysd[key]).reshape(-1), torch.float64).data_ptr())
    n_out = len(sysd["out_ptr"]) - 1
    s.n_out = n_out
    s.out_ptr = put(sysd["out_ptr"], torch.int32).data_ptr()
    s.out_idx = put(sysd["out_idx"], torch.int32).data_ptr() if len(sysd["out_idx"]) else None
    s.out_val = put(sysd["out_val"], torch.float64).data_ptr() if len(sysd["out_val"]) else None
    r = np.ascontiguousarray(sysd["r"], dtype=np.float64)
    keep.append(r)
    s.r = r.ctypes.data if n_out else None
    return s


class BatchSolver:
    """Many independent tangents solved concurrently (nbp_batch_*)."""

    def __init__(self, systems, device: int = 0, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("nbp.BatchSolver needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load()
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        keep = []
        arr = (nbp_system * len(systems))(*[_system(d, self.dev, keep) for d in systems])
        self.sizes = [4 * int(d["n_nodes"]) for d in systems]
        self.opts = default_options(**opts)
        h = ctypes.c_void_p()
        torch.cuda.synchronize(self.dev)
        st = self.lib.nbp_batch_create(ctypes.byref(h), len(systems), arr, ctypes.byref(self.opts))
        if st != 0:
            raise NbpError(st, "nbp_batch_create failed (see stderr)")
        self.h = h
        del keep

    def _check(self, st, ok=(0,)):
        if st not in ok:
            raise NbpError(st, self.lib.nbp_batch_last_error(self.h).decode())
        return st

    def setup(self):
        self._check(self.lib.nbp_batch_setup(self.h))

    def solve(self, bs, xs=None, **kw):
        """bs: list of CUDA float64 tensors; returns (xs, list of info dicts)."""
        n = len(bs)
        if xs is None:
            xs = [self.torch.zeros(m, dtype=self.torch.float64, device=self.dev) for m in self.sizes]
        bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        infos = (nbp_info * n)()
        o = default_options()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(self.opts), ctypes.sizeof(o))
        for k, v in kw.items():
            setattr(o, k, v)
        self._check(self.lib.nbp_batch_solve(self.h, bp, xp, ctypes.byref(o), infos))
        return xs, [i.as_dict() for i in infos]

    def close(self):
        if getattr(self, "h", None):
            self.lib.nbp_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One library context for a tangent (numpy arrays in the synth format)."""

    def __init__(self, sysd: dict, device: int = 0, stream=None, **opts):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("nbp.Solver needs a CUDA device (no CPU fallback)")
        self.torch = torch
        self.lib = load()
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.N = int(sysd["n_nodes"])
        self.n_out = len(sysd["out_ptr"]) - 1
        rp, col = sysd["rowptr"], sysd["col"]
        self.nnz = len(col)   # entries of the shared pattern (the time-step tangent's layout)
        keep = []

        def dev(a, dt):
            t = torch.as_tensor(np.ascontiguousarray(a), dtype=dt).to(self.dev)
            keep.append(t)
            return t

        s = nbp_system()
        s.n_nodes = self.N
        for key in "ABCD":
            k = key.lower()
            r_ = dev(sysd.get(key + "_rowptr", rp), torch.int32)
            c_ = dev(sysd.get(key + "_col", col), torch.int32)
            v_ = dev(np.asarray(sysd[key]).reshape(-1), torch.float64)
            setattr(s, f"{k}_rowptr", r_.data_ptr())
            setattr(s, f"{k}_col", c_.data_ptr())
            setattr(s, f"{k}_val", v_.data_ptr())
        s.n_out = self.n_out
        s.out_ptr = dev(sysd["out_ptr"], torch.int32).data_ptr()
        s.out_idx = dev(sysd["out_idx"], torch.int32).data_ptr() if len(sysd["out_idx"]) else None
        s.out_val = dev(sysd["out_val"], torch.float64).data_ptr() if len(sysd["out_val"]) else None
        self._r = np.ascontiguousarray(sysd["r"], dtype=np.float64)
        s.r = self._r.ctypes.data if self.n_out else None
        self.opts = default_options(**opts)
        ctx = ctypes.c_void_p()
        st = self.lib.nbp_create(ctypes.byref(ctx), ctypes.byref(s), ctypes.byref(self.opts),
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise NbpError(st, "nbp_create failed (see stderr)")
        self.ctx = ctx
        torch.cuda.synchronize(self.dev)
        del keep   # the library copied everything during nbp_create

    # ---------------------------------------------------------------- api
    def _check(self, st, ok=(0,)):
        if st not in ok:
            raise NbpError(st, self.lib.nbp_last_error(self.ctx).decode())
        return st

    def close(self):
        # handles bound to this context (Vms) go first: they hold its pointer
        for child in list(getattr(self, "_children", ())):
            child.close()
        if getattr(self, "ctx", None):
            self.lib.nbp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def setup(self, numeric=False):
        """Build the preconditioner (nbp_setup); numeric=True rebuilds it from
        the current values on the aggregates of the last full setup
        (nbp_setup_numeric)."""
        self._check((self.lib.nbp_setup_numeric if numeric else self.lib.nbp_setup)(self.ctx))

    def set_resistances(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        self._check(self.lib.nbp_set_resistances(self.ctx, r.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def options(self, **kw) -> nbp_options:
        o = nbp_options()
        ctypes.memmove(ctypes.byref(o), ctypes.byref(self.opts), ctypes.sizeof(o))
        for k, v in kw.items():
            setattr(o, k, v)
        return o

    def zeros(self, n, dtype=None):
        return self.torch.zeros(n, dtype=dtype or self.torch.float64, device=self.dev)

    def solve(self, b, x=None, allow_not_converged=False, **kw):
        """b: CUDA float64 tensor (4N). Returns (x, info dict)."""
        x = self.zeros(4 * self.N) if x is None else x
        info = nbp_info()
        o = self.options(**kw)
        st = self.lib.nbp_solve(self.ctx, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info))
        self._check(st, (0, 4) if allow_not_converged else (0,))
        return x, info.as_dict()

    def solve_host(self, b_host: np.ndarray, x_host: np.ndarray = None, **kw):
        """b_host: pinned or pageable float64 numpy/tensor on the host; copies inside the call."""
        if x_host is None:
            x_host = np.zeros(4 * self.N)
        info = nbp_info()
        o = self.options(**kw)
        bp = b_host.data_ptr() if hasattr(b_host, "data_ptr") else b_host.ctypes.data
        xp = x_host.data_ptr() if hasattr(x_host, "data_ptr") else x_host.ctypes.data
        st = self.lib.nbp_solve_host(self.ctx, ctypes.c_void_p(bp), ctypes.c_void_p(xp), ctypes.byref(o),
                                     ctypes.byref(info))
        self._check(st)
        return x_host, info.as_dict()

    def adjoint(self, g, x):
        lam = self.zeros(4 * self.N)
        dldr = np.zeros(max(self.n_out, 1))
        info = nbp_info()
        st = self.lib.nbp_adjoint(self.ctx, _ptr(g), _ptr(x), _ptr(lam),
                                  dldr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(info))
        self._check(st)
        return lam, dldr[:self.n_out], info.as_dict()

    def apply_A(self, x, precision=0):
        y = self.torch.empty_like(x)
        self._check(self.lib.nbp_apply_A(self.ctx, _ptr(x), _ptr(y), precision))
        return y

    def apply_full(self, x):
        y = self.torch.empty_like(x)
        self._check(self.lib.nbp_apply_full(self.ctx, _ptr(x), _ptr(y)))
        return y

    def apply_S(self, xp):
        y = self.torch.empty_like(xp)
        self._check(self.lib.nbp_apply_S(self.ctx, _ptr(xp), _ptr(y)))
        return y

    def apply_pscr(self, s):
        y = self.torch.empty_like(s)
        self._check(self.lib.nbp_apply_pscr(self.ctx, _ptr(s), _ptr(y)))
        return y

    def solve_A(self, s, rtol):
        y = self.torch.empty_like(s)
        its = ctypes.c_int32(0)
        st = self.lib.nbp_solve_A(self.ctx, _ptr(s), _ptr(y), rtol, ctypes.byref(its))
        self._check(st, (0, 4))
        return y, its.value

    def vcycle(self, which, b):
        x = self.torch.empty_like(b)
        self._check(self.lib.nbp_vcycle(self.ctx, which, _ptr(b), _ptr(x)))
        return x

    def amg_levels(self, which=0):
        rows = (ctypes.c_int32 * 16)()
        nnz = (ctypes.c_int64 * 16)()
        nl = self.lib.nbp_amg_level_sizes(self.ctx, which, rows, nnz, 16)
        bs = 3 if which == 0 else 1
        out = []
        for l in range(nl):
            n, z = rows[l], nnz[l]
            rp = np.zeros(n + 1, np.int32)
            ci = np.zeros(max(z, 1), np.int32)
            v = np.zeros(max(z, 1) * bs * bs)
            agg = np.full(n, -1, np.int32)
            rho = ctypes.c_double(0)
            self._check(self.lib.nbp_amg_level_get(self.ctx, which, l, rp.ctypes.data, ci.ctypes.data, v.ctypes.data,
                                                   agg.ctypes.data, ctypes.byref(rho)))
            out.append(dict(rowptr=rp, col=ci[:z], val=(v[:z * bs * bs].reshape(z, bs, bs) if bs > 1 else v[:z]),
                            agg=agg if l + 1 < nl else None, rho=rho.value))
        return out

    def shat(self):
        z = self.lib.nbp_shat_nnz(self.ctx)
        rp = np.zeros(self.N + 1, np.int32)
        ci = np.zeros(max(z, 1), np.int32)
        v = np.zeros(max(z, 1))
        self._check(self.lib.nbp_shat_get(self.ctx, rp.ctypes.data, ci.ctypes.data, v.ctypes.data))
        return rp, ci[:z], v[:z]

    def outlet_flows(self, v):
        """Q^k = a^k . v for the 3N velocity dofs v (CUDA float64)."""
        Q = self.zeros(self.n_out)
        self._check(self.lib.nbp_outlet_flows(self.ctx, _ptr(v), _ptr(Q)))
        return Q

    def rcr_update(self, rcr: dict, v_np1, dt, nts, scale, eps_abs=1e-8, eps_rel=1e-5):
        """Outlet coupling of one Newton iteration (nbp_rcr_update): rcr holds
        CUDA float64 tensors Rp, C, Rd, Pd, Pi_n, Q_n; the weights r_k =
        scale m^k are installed in the context.  Returns dict Q, P, Pi, m."""
        p = rcr_params(rcr["Rp"], rcr["C"], rcr["Rd"], rcr["Pd"], rcr["Pi_n"], rcr["Q_n"], eps_abs, eps_rel)
        out = {k: self.zeros(self.n_out) for k in ("Q", "P", "Pi", "m")}
        self._check(self.lib.nbp_rcr_update(self.ctx, ctypes.byref(p), _ptr(v_np1), float(dt), int(nts), float(scale),
                                             _ptr(out["Q"]), _ptr(out["P"]), _ptr(out["Pi"]), _ptr(out["m"])))
        return out

    def set_values(self, A, B, C, D):
        """New tangent values (CUDA float64 tensors on the context's pattern,
        9, 3, 3, 1 per entry); call setup() again before solving."""
        self._check(self.lib.nbp_set_values(self.ctx, _ptr(A), _ptr(B), _ptr(C), _ptr(D)))

    def profile(self, enable=True):
        self._check(self.lib.nbp_profile(self.ctx, int(enable)))

    def profile_info(self):
        p = nbp_profile_info()
        self._check(self.lib.nbp_profile_get(self.ctx, ctypes.byref(p)))
        return p.as_dict()

    def profile_report(self):
        import json
        return json.loads(self.lib.nbp_profile_report(self.ctx).decode())


class Vms:
    """On-device VMS residual, tangent and Newton time step bound to a Solver
    (nbp_vms_*, Sec. 2.3-2.5).  mesh: dict X (N,3), tets (E,4), tris (T,3),
    dir (N,) as host numpy arrays.  Close it before the Solver."""

    def __init__(self, solver: "Solver", mesh: dict, rho, mu, dt, rho_inf, beta=0.2, CI=36.0, CT=4.0,
                 tangent_fp32=True):
        self.s = solver
        self.lib = solver.lib
        self.N = solver.N
        X = np.ascontiguousarray(mesh["X"], dtype=np.float64)
        tets = np.ascontiguousarray(mesh["tets"], dtype=np.int32)
        tris = np.ascontiguousarray(mesh["tris"], dtype=np.int32).reshape(-1, 3)
        dirn = np.ascontiguousarray(mesh["dir"], dtype=np.uint8)
        m = nbp_mesh(self.N, len(tets), len(tris), X.ctypes.data, tets.ctypes.data,
                     tris.ctypes.data if len(tris) else None, dirn.ctypes.data)
        par = nbp_vms_params(rho, mu, dt, rho_inf, beta, CI, CT, 1 if tangent_fp32 else 0)
        h = ctypes.c_void_p()
        solver._check(self.lib.nbp_vms_create(ctypes.byref(h), solver.ctx, ctypes.byref(m), ctypes.byref(par)))
        self.h = h
        if not hasattr(solver, "_children"):
            solver._children = weakref.WeakSet()
        solver._children.add(self)

    def close(self):
        if getattr(self, "h", None):
            self.lib.nbp_vms_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def residual(self, vd, v, p, P=None, vtau=None):
        """R (4N) at vdot_{n+alpha_m}, v_{n+alpha_f}, p_{n+alpha_f}; P the outlet pressures."""
        R = self.s.zeros(4 * self.N)
        self.s._check(self.lib.nbp_vms_residual(self.h, _ptr(vd), _ptr(v), _ptr(p), _ptr(vtau) if vtau is not None else None,
                                                 _ptr(P) if P is not None else None, _ptr(R)))
        return R

    def tangent(self, vd, v, p, nnz=None, vtau=None):
        """Tangent values (A 9 nnz, B 3 nnz, C 3 nnz, D nnz) at the same state
        (nnz: entries of the solver's pattern, by default the Solver's)."""
        nnz = self.s.nnz if nnz is None else nnz
        out = {k: self.s.zeros(w * nnz) for k, w in (("A", 9), ("B", 3), ("C", 3), ("D", 1))}
        self.s._check(self.lib.nbp_vms_tangent(self.h, _ptr(vd), _ptr(v), _ptr(p),
                                                _ptr(vtau) if vtau is not None else None,
                                                _ptr(out["A"]), _ptr(out["B"]), _ptr(out["C"]), _ptr(out["D"])))
        return out

    def newton_step(self, y_n, yd_n, rcr: dict = None, tol_R=1e-6, tol_A=1e-6, l_max=20, nts=10, eps_abs=1e-8,
                    eps_rel=1e-5, allow_not_converged=False, pc_rebuild=0):
        """One predictor multi-corrector time step (nbp_newton_step).  rcr:
        CUDA float64 tensors Rp, C, Rd, Pd, Pi (Pi^k_n).  pc_rebuild: 0 a
        preconditioner per tangent, 1 one per step, 2 keep the context's, 3 a
        numeric re-setup on the held aggregates per tangent, 4 one per step.
        Returns (y, ydot, Pi_np1, info)."""
        y = self.s.zeros(4 * self.N)
        yd = self.s.zeros(4 * self.N)
        Pi = self.s.zeros(max(self.s.n_out, 1))
        p = None
        if rcr is not None:
            p = rcr_params(rcr["Rp"], rcr["C"], rcr["Rd"], rcr["Pd"], rcr["Pi"], rcr["Pi"], eps_abs, eps_rel)
        o = nbp_newton_opts(tol_R, tol_A, l_max, nts, pc_rebuild)
        info = nbp_newton_info()
        st = self.lib.nbp_newton_step(self.h, ctypes.byref(p) if p is not None else None, _ptr(y_n), _ptr(yd_n),
                                      _ptr(y), _ptr(yd), _ptr(Pi), ctypes.byref(o), ctypes.byref(info))
        self.s._check(st, (0, 4) if allow_not_converged else (0,))
        return y, yd, Pi[:self.s.n_out], info.as_dict()
