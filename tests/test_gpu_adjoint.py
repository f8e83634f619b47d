"""Adjoint on the 32x32x128 box (140,481 nodes, Re 300, 4 outlets with R_k
log-uniform in [1e2, 1e4]): L = sum_k (a^k . u - q_k)^2, gradient through
torch.autograd (NestedSolveFn -> nbp_adjoint, FP64 outer / FP32 inner) against
central finite differences h = 1e-6 r_k of FP64 forward solves."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver  # noqa: E402
from paper_1911_10814_gb300.autograd import nested_solve  # noqa: E402


def test_adjoint_gradient_vs_central_differences():
    spec = synth.adjoint_case()
    d = synth.generate(spec)
    N = d["n_nodes"]
    nv = 3 * N
    n_out = len(d["out_ptr"]) - 1
    A = torch.zeros((n_out, nv), dtype=torch.float64)
    for k in range(n_out):
        sl = slice(d["out_ptr"][k], d["out_ptr"][k + 1])
        A[k, torch.as_tensor(d["out_idx"][sl], dtype=torch.long)] = torch.as_tensor(d["out_val"][sl])
    A = A.to("cuda:0")
    s = Solver(d, precision=1, rtol=1e-12)
    s.setup()
    b = torch.as_tensor(d["b"], device="cuda:0")
    r0 = torch.as_tensor(d["r"], device="cuda:0")
    with torch.no_grad():
        u0 = nested_solve(b, r0, s)[:nv]
    flux0 = (A @ u0).cpu().numpy()
    q = torch.as_tensor((2 * synth.uniforms(4 ^ 0xA11, n_out) - 1) * np.abs(flux0).max(), device="cuda:0")

    r = r0.clone().requires_grad_(True)
    x = nested_solve(b, r, s)
    L = ((A @ x[:nv] - q) ** 2).sum()
    L.backward()
    g = r.grad.cpu().numpy()

    def loss(rv):
        s.set_resistances(rv)
        xx, info = s.solve(b, precision=0, rtol=1e-13, allow_not_converged=True)
        return float(((A @ xx[:nv] - q) ** 2).sum())

    for k in range(n_out):
        h = 1e-6 * d["r"][k]
        rp, rm = d["r"].copy(), d["r"].copy()
        rp[k] += h
        rm[k] -= h
        fd = (loss(rp) - loss(rm)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-5 * abs(fd), (k, g[k], fd)
    # dL/db = lambda: directional check on one random direction
    s.set_resistances(d["r"])
    db = torch.as_tensor(np.random.default_rng(3).standard_normal(4 * N), device="cuda:0")
    bb = b.clone().requires_grad_(True)
    x = nested_solve(bb, r0, s)
    L2 = ((A @ x[:nv] - q) ** 2).sum()
    L2.backward()
    eps = 1e-3

    def loss_b(bv):
        xx, _ = s.solve(bv, precision=0, rtol=1e-13, allow_not_converged=True)
        return float(((A @ xx[:nv] - q) ** 2).sum())

    fdb = (loss_b(b + eps * db) - loss_b(b - eps * db)) / (2 * eps)
    assert abs(float(bb.grad @ db) - fdb) <= 1e-5 * abs(fdb)
    s.close()
