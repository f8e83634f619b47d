"""Status codes of the C ABI on host-made failures (no GPU fault is caused):
call order, non-convergence at n_max, non-finite input, bad options."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver  # noqa: E402
from paper_1911_10814_gb300.nbp import NbpError  # noqa: E402


@pytest.fixture(scope="module")
def tiny():
    return synth.generate(synth.tiny())


def test_solve_before_setup_is_a_state_error(tiny):
    s = Solver(tiny)
    with pytest.raises(NbpError) as e:
        s.solve(torch.as_tensor(tiny["b"], device="cuda:0"))
    assert e.value.status == 8
    s.close()


def test_not_converged_still_returns_x(tiny):
    s = Solver(tiny)
    s.setup()
    x, info = s.solve(torch.as_tensor(tiny["b"], device="cuda:0"), allow_not_converged=True, nmax=1, rtol=1e-14)
    assert info["status"] == 4 and info["outer_iters"] == 1
    assert torch.isfinite(x).all() and float(x.abs().max()) > 0
    s.close()


def test_nan_rhs_reported(tiny):
    s = Solver(tiny)
    s.setup()
    b = torch.as_tensor(tiny["b"], device="cuda:0").clone()
    b[7] = float("nan")
    with pytest.raises(NbpError) as e:
        s.solve(b)
    assert e.value.status == 6
    # the context stays usable
    x, info = s.solve(torch.as_tensor(tiny["b"], device="cuda:0"))
    assert info["status"] == 0
    s.close()


def test_bad_options_rejected(tiny):
    with pytest.raises(NbpError):
        Solver(tiny, m=0)
    s = Solver(tiny)
    s.setup()
    with pytest.raises(NbpError) as e:
        s.solve(torch.as_tensor(tiny["b"], device="cuda:0"), precision=7)
    assert e.value.status == 1
    s.close()


def test_nan_matrix_rejected_at_create(tiny):
    bad = dict(tiny)
    A = tiny["A"].copy()
    A[3, 1, 1] = np.inf
    bad["A"] = A
    with pytest.raises(NbpError) as e:
        Solver(bad)
    assert e.value.status == 1
