"""GPU test of nbp_apply_A_noalloc, the entry point for callers that cannot
call cudaMalloc (frozen memory pools, allocation-free real-time loops, callers
without a library context).  It must give the same y = A x as nbp_apply_A on
two calls in a row (the fixed scratch array keeps the previous call's
contents), and reject more outlets than its fixed array holds.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver, load  # noqa: E402

MAX_OUTLETS = 1024


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda:0")


def _call(lib, N, rp, col, val, n_out, optr, oidx, oval, r, x, y):
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    return lib.nbp_apply_A_noalloc(N, p(rp), p(col), p(val), n_out, p(optr), p(oidx), p(oval), p(r), p(x), p(y),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_apply_A_noalloc_matches_apply_A_twice():
    spec = synth.MeshSpec(9, 11, 23, Lz=2.0, Re=300.0, seed=5, R=(1e2, 1e3, 3e3, 1e4), name="box9x11x23_q4")
    d = synth.generate(spec)
    N = d["n_nodes"]
    lib = load()
    s = Solver(d)
    rp, col = _dev(d["rowptr"], torch.int32), _dev(d["col"], torch.int32)
    val = _dev(d["A"].reshape(-1), torch.float64)
    optr, oidx = _dev(d["out_ptr"], torch.int32), _dev(d["out_idx"], torch.int32)
    oval, r = _dev(d["out_val"], torch.float64), _dev(d["r"], torch.float64)
    rng = np.random.default_rng(11)
    for call in range(2):
        x = _dev(rng.standard_normal(3 * N), torch.float64)
        y = torch.full((3 * N,), float("nan"), dtype=torch.float64, device="cuda:0")
        st = _call(lib, N, rp, col, val, len(d["out_ptr"]) - 1, optr, oidx, oval, r, x, y)
        assert st == 0
        torch.cuda.synchronize()
        ref = s.apply_A(x)
        yh, rh = y.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(yh))
        assert np.abs(yh - rh).max() <= 1e-12 * np.abs(rh).max(), f"call {call}"
    s.close()


def _host_A(d, x, optr=None, oidx=None, oval=None, r=None):
    """A_sp x (+ sum_k r_k a^k (a^k . x)) on the host, FP64."""
    N = d["n_nodes"]
    A = d["A"].reshape(-1, 3, 3)
    y = np.zeros(3 * N)
    rows = np.repeat(np.arange(N), np.diff(d["rowptr"]))
    np.add.at(y.reshape(N, 3), rows, np.einsum("eab,eb->ea", A, x.reshape(N, 3)[d["col"]]))
    if optr is not None:
        for k in range(len(optr) - 1):
            sl = slice(optr[k], optr[k + 1])
            y[oidx[sl]] += r[k] * (oval[sl] @ x[oidx[sl]]) * oval[sl]
    return y


def test_apply_A_noalloc_without_outlets():
    """n_out = 0 with null outlet pointers is the plain sparse product."""
    d = synth.generate(synth.tiny())
    N = d["n_nodes"]
    lib = load()
    rp, col = _dev(d["rowptr"], torch.int32), _dev(d["col"], torch.int32)
    val = _dev(d["A"].reshape(-1), torch.float64)
    xh = np.random.default_rng(3).standard_normal(3 * N)
    x = _dev(xh, torch.float64)
    y = torch.full((3 * N,), float("nan"), dtype=torch.float64, device="cuda:0")
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    null = ctypes.c_void_p(None)
    st = lib.nbp_apply_A_noalloc(N, p(rp), p(col), p(val), 0, null, null, null, null, p(x), p(y),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    ref = _host_A(d, xh)
    yh = y.cpu().numpy()
    assert np.abs(yh - ref).max() <= 1e-12 * np.abs(ref).max()


def test_apply_A_noalloc_at_the_outlet_limit():
    """n_out = 1024 (the fixed array's size): small outlets that share nodes
    with each other, against the host product."""
    d = synth.generate(synth.tiny())
    N = d["n_nodes"]
    lib = load()
    rng = np.random.default_rng(7)
    per = 3
    oidx_h = np.concatenate([rng.choice(3 * N, per, replace=False) for _ in range(MAX_OUTLETS)]).astype(np.int32)
    optr_h = (np.arange(MAX_OUTLETS + 1) * per).astype(np.int32)
    oval_h = rng.uniform(0.1, 1.0, MAX_OUTLETS * per)
    r_h = rng.uniform(0.5, 2.0, MAX_OUTLETS)
    rp, col = _dev(d["rowptr"], torch.int32), _dev(d["col"], torch.int32)
    val = _dev(d["A"].reshape(-1), torch.float64)
    optr, oidx = _dev(optr_h, torch.int32), _dev(oidx_h, torch.int32)
    oval, r = _dev(oval_h, torch.float64), _dev(r_h, torch.float64)
    xh = rng.standard_normal(3 * N)
    x = _dev(xh, torch.float64)
    ref = _host_A(d, xh, optr_h, oidx_h, oval_h, r_h)
    for _ in range(2):
        y = torch.full((3 * N,), float("nan"), dtype=torch.float64, device="cuda:0")
        st = _call(lib, N, rp, col, val, MAX_OUTLETS, optr, oidx, oval, r, x, y)
        assert st == 0
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
        assert np.abs(yh - ref).max() <= 1e-12 * np.abs(ref).max()


def test_apply_A_noalloc_rejects_too_many_outlets():
    d = synth.generate(synth.tiny())
    N = d["n_nodes"]
    lib = load()
    rp, col = _dev(d["rowptr"], torch.int32), _dev(d["col"], torch.int32)
    val = _dev(d["A"].reshape(-1), torch.float64)
    optr = _dev(np.zeros(MAX_OUTLETS + 2, np.int32), torch.int32)
    oidx = _dev(np.zeros(1, np.int32), torch.int32)
    oval = _dev(np.zeros(1), torch.float64)
    r = _dev(np.zeros(MAX_OUTLETS + 1), torch.float64)
    x = _dev(np.ones(3 * N), torch.float64)
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda:0")
    st = _call(lib, N, rp, col, val, MAX_OUTLETS + 1, optr, oidx, oval, r, x, y)
    assert st == 1   # NBP_ERR_INVALID, nothing launched
    torch.cuda.synchronize()
    assert float(y.abs().max()) == 0.0
