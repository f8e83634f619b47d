"""The setup's two grouping paths against the FP64 oracle.

The coarse graphs of the aggregation passes, the Galerkin products and
S_hat are grouped one coarse row per warp in shared memory when a row holds
at most 1024 entries (S_hat: 256 products), and through a global sort of
all entries otherwise.  The regular meshes stay below those capacities, so
this case couples an interior node (the hub) with every node (its row and
column of the tangent full): the aggregate holding the hub, the coarse-graph
rows above it and S_hat's hub row go past them and take the global path,
every other row the row-local one.  Both must give
the oracle's aggregate maps, Galerkin blocks and S_hat bit for bit."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1911_10814_gb300 import Solver  # noqa: E402

ROW_CAPACITY = 1024     # entries of a coarse row grouped in shared memory
SHAT_CAPACITY = 256     # products of an S_hat row sorted in shared memory


def with_dense_row(d, hub, scale=1e-3, seed=7):
    """`d` with node `hub` coupled to every node: the new blocks of A are
    `scale` x (mean |diag A|) x uniform(-1, 1) entries, those of B, C and D
    the same relative to their own mean magnitudes; every existing block
    keeps its value."""
    N, rp, ci = d["n_nodes"], d["rowptr"], d["col"]
    rng = np.random.default_rng(seed)
    cols = [ci[rp[i]:rp[i + 1]] for i in range(N)]
    new_cols = [np.union1d(c, [hub]) for c in cols]
    new_cols[hub] = np.arange(N, dtype=np.int32)
    nrp = np.zeros(N + 1, dtype=np.int32)
    nrp[1:] = np.cumsum([len(c) for c in new_cols])
    nci = np.concatenate(new_cols).astype(np.int32)
    nnz = int(nrp[-1])
    diag = np.array([d["A"][rp[i] + np.searchsorted(cols[i], i)] for i in range(N)])
    a_mag = np.abs(np.einsum("kaa->ka", diag)).mean()
    mags = {k: np.abs(d[k]).mean() for k in ("B", "C", "D")}
    out = dict(d)
    out["rowptr"], out["col"] = nrp, nci
    out["A"] = scale * a_mag * rng.uniform(-1.0, 1.0, (nnz, 3, 3))
    out["B"] = scale * mags["B"] * rng.uniform(-1.0, 1.0, (nnz, 3))
    out["C"] = scale * mags["C"] * rng.uniform(-1.0, 1.0, (nnz, 3))
    out["D"] = scale * mags["D"] * rng.uniform(-1.0, 1.0, nnz)
    for i in range(N):   # old entries keep their blocks
        pos = nrp[i] + np.searchsorted(new_cols[i], cols[i])
        for k in ("A", "B", "C", "D"):
            out[k][pos] = d[k][rp[i]:rp[i + 1]]
    return out


@pytest.fixture(scope="module")
def dense_case():
    base = synth.generate(synth.MeshSpec(11, 11, 11, Re=100.0, seed=3, R=(1e3, 1e4), name="cube11_dense_row"))
    hub = 6 * 12 * 12 + 6 * 12 + 6   # node (6, 6, 6) of the 12^3 nodes
    d = with_dense_row(base, hub)
    assert d["n_nodes"] > ROW_CAPACITY
    s = Solver(d)
    s.setup()
    o = oracle.Oracle(d)
    o.setup()
    yield d, hub, s, o
    s.close()


def test_hierarchies_bit_exact_past_the_row_capacity(dense_case):
    d, hub, s, o = dense_case
    for which in (0, 1):
        G, O = s.amg_levels(which), o.amg_levels(which)
        assert len(G) == len(O) >= 2
        for lg, lo in zip(G, O):
            assert np.array_equal(lg["rowptr"], lo["rowptr"])
            assert np.array_equal(lg["col"], lo["col"])
            assert np.array_equal(lg["val"], lo["val"])
            if lo["agg"] is not None:
                assert np.array_equal(lg["agg"], lo["agg"])
    # in both hierarchies the aggregate holding the hub sums more fine
    # entries than a row-local group holds
    for which in (0, 1):
        L0 = s.amg_levels(which)[0]
        assert L0["agg"][hub] >= 0
        members = np.flatnonzero(L0["agg"] == L0["agg"][hub])
        assert sum(L0["rowptr"][m + 1] - L0["rowptr"][m] for m in members) > ROW_CAPACITY


def test_shat_bit_exact_past_the_row_capacity(dense_case):
    d, hub, s, o = dense_case
    rp, ci, v = s.shat()
    rpo, cio, vo = o.shat()
    assert np.array_equal(rp, rpo) and np.array_equal(ci, cio) and np.array_equal(v, vo)
    # S_hat's hub row gathers D's full row and C's full row times B
    assert rp[hub + 1] - rp[hub] == d["n_nodes"] > SHAT_CAPACITY
