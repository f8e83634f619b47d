"""GPU numeric re-setup (nbp_setup_numeric) against the oracle's
(or_setup_numeric): after new values on the same patterns, both AMG
hierarchies are rebuilt on the aggregates of the last full setup.  Aggregate
maps, Galerkin blocks and S_hat must equal the oracle's bit for bit, the
Chebyshev bounds to rounding, and the nested solve with the re-set-up
preconditioner must match the oracle's solution."""
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

SPEC = synth.MeshSpec(9, 11, 23, Lz=2.0, Re=300.0, seed=5, R=(1e2, 1e3, 3e3, 1e4), name="box9x11x23_q4")


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda:0")


def _perturbed(d, seed=4):
    rng = np.random.default_rng(seed)
    return {k: np.asarray(d[k], dtype=np.float64) * rng.uniform(0.9, 1.1, np.shape(d[k])) for k in ("A", "B", "C", "D")}


def _same_hierarchies(s, o):
    for which in (0, 1):
        G, O = s.amg_levels(which), o.amg_levels(which)
        assert len(G) == len(O)
        for lg, lo in zip(G, O):
            assert np.array_equal(lg["rowptr"], lo["rowptr"]) and np.array_equal(lg["col"], lo["col"])
            assert np.array_equal(lg["val"], lo["val"])
            if lo["agg"] is not None:
                assert np.array_equal(lg["agg"], lo["agg"])
                assert lg["rho"] == pytest.approx(lo["rho"], rel=1e-9)
    rp, ci, v = s.shat()
    rpo, cio, vo = o.shat()
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio) and np.array_equal(v, vo)


@pytest.mark.parametrize("prec", [0, 3])
def test_numeric_setup_matches_oracle(prec):
    d = synth.generate(SPEC)
    s = Solver(d, precision=prec)
    s.setup()
    o = oracle.Oracle(d)
    o.setup()
    aggs = [[lv["agg"] for lv in s.amg_levels(w)] for w in (0, 1)]
    new = _perturbed(d)
    s.set_values(*(_t(new[k].reshape(-1)) for k in ("A", "B", "C", "D")))
    o.set_values(new["A"], new["B"], new["C"], new["D"])
    s.setup(numeric=True)
    o.setup_numeric()
    _same_hierarchies(s, o)
    for w in (0, 1):   # the maps of the first setup
        for a, lv in zip(aggs[w], s.amg_levels(w)):
            assert (a is None and lv["agg"] is None) or np.array_equal(a, lv["agg"])
    x, info = s.solve(_t(d["b"]))
    assert info["rel_res_true"] <= 1e-8
    o.set_options(rtol=1e-12)
    xo, _, rc = o.solve(d["b"])
    assert rc == 0
    xh = x.cpu().numpy()
    assert np.linalg.norm(xh - xo) / np.linalg.norm(xo) <= (1e-6 if prec == 0 else 1e-5)
    s.close()


def test_numeric_setup_without_setup_is_a_state_error():
    d = synth.generate(synth.tiny())
    s = Solver(d)
    with pytest.raises(NbpError) as e:
        s.setup(numeric=True)
    assert e.value.status == 8   # NBP_ERR_STATE
    s.close()
