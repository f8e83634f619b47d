"""The smallest meshes: every AMG hierarchy has one level (at most 300 block
rows), so each cycle is the coarsest level's dense inverse alone, and the
Krylov vectors are shorter than one reduction chunk.  The nested solve is
checked against dense LU of the whole tangent and against the oracle's
iteration counts, in FP64 and in the mixed mode, with the device-driven
loops (the default) and the host loop.  A single hexahedron is the
degenerate case: every node lies on the boundary and the tangent is singular
(2-norm condition number about 3e22); the solve must end with an error
status, not a result."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver  # noqa: E402
from paper_1911_10814_gb300.nbp import NbpError  # noqa: E402

SMALL = [(2, 2, 2), (2, 3, 5), (3, 3, 6)]


def _spec(nx, ny, nz):
    return synth.MeshSpec(nx, ny, nz, Lz=float(nz) / nx, Re=100.0, seed=3, R=(1e3,), name=f"box{nx}x{ny}x{nz}")


@pytest.mark.parametrize("shape", SMALL, ids=[f"{a}x{b}x{c}" for a, b, c in SMALL])
@pytest.mark.parametrize("prec,device_loop", [(0, 1), (0, 0), (3, 1)])
def test_single_level_hierarchies(shape, prec, device_loop):
    d = synth.generate(_spec(*shape))
    *_, F = oracle.dense_system(d)
    x_lu = np.linalg.solve(F, d["b"])
    s = Solver(d, precision=prec)
    s.setup()
    assert len(s.amg_levels(0)) == 1 and len(s.amg_levels(1)) == 1
    x, info = s.solve(torch.as_tensor(d["b"], device="cuda:0"), device_loop=device_loop)
    xh = x.cpu().numpy()
    assert info["rel_res_true"] <= 1e-8
    assert np.linalg.norm(xh - x_lu) / np.linalg.norm(x_lu) <= (1e-6 if prec == 0 else 1e-5)
    o = oracle.Oracle(d)
    _, oinfo, rc = o.solve(d["b"])
    assert rc == 0
    assert abs(info["outer_iters"] - oinfo.outer_iters) <= (0 if prec == 0 else 1)
    if prec == 0:
        assert info["S_iters"] == oinfo.S_iters
    s.close()


@pytest.mark.parametrize("device_loop", [1, 0])
def test_singular_single_hexahedron_is_reported(device_loop):
    d = synth.generate(_spec(1, 1, 1))
    s = Solver(d, precision=3, nmax=20)
    try:
        s.setup()
        x, info = s.solve(torch.as_tensor(d["b"], device="cuda:0"), device_loop=device_loop)
    except NbpError as e:
        assert e.status in (1, 4, 5, 6)   # invalid (singular block), not converged, breakdown, NaN
    else:
        pytest.fail(f"a singular tangent gave a result: {info}")
    finally:
        s.close()
