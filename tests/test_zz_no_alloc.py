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
