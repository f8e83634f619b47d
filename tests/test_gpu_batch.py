"""Batched solves of independent uneven tangents (48 cubes 12^3..40^3 hexes,
Re in [100, 1000], 1-4 outlets, FP32 inner / FP64 outer): every instance
agrees bitwise with its own single solve and meets the FP64 true residual
1e-8 checked by the oracle's product."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import BatchSolver, Solver  # noqa: E402


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


@pytest.mark.parametrize("prec", [1, 3])
def test_small_batch_matches_single_solves(prec):
    specs = synth.batch(count=6, seed=7, smin=5, smax=11)
    systems = [synth.generate(sp) for sp in specs]
    B = BatchSolver(systems, precision=prec)
    B.setup()
    xs, infos = B.solve([_t(d["b"]) for d in systems])
    torch.cuda.synchronize()
    for d, x, info in zip(systems, xs, infos):
        s = Solver(d, precision=prec)
        s.setup()
        x1, info1 = s.solve(_t(d["b"]))
        assert torch.equal(x, x1)
        assert info["outer_iters"] == info1["outer_iters"]
        s.close()
    B.close()


def test_batch_of_48_uneven_tangents():
    specs = synth.batch()
    systems = [synth.generate(sp) for sp in specs]
    B = BatchSolver(systems, precision=1)
    B.setup()
    xs, infos = B.solve([_t(d["b"]) for d in systems])
    torch.cuda.synchronize()
    assert len(xs) == 48
    sizes = [4 * d["n_nodes"] for d in systems]
    assert min(sizes) == 4 * 13 ** 3 or min(sizes) >= 4 * 13 ** 3
    for d, x, info in zip(systems, xs, infos):
        o = oracle.Oracle(d)
        r = d["b"] - o.apply_full(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(d["b"]) <= 1e-8
        assert info["status"] == 0
    B.close()
