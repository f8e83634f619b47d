"""Host logic of the on-device assembly, on the CPU: the gather maps that fix
the summation order of every residual row and tangent slot (nbp_vms_maps,
the host step of nbp_vms_create) against a brute-force construction."""
import ctypes

import numpy as np
import pytest

import synth


def _maps(lib, rowptr, col, el, N):
    w = el.shape[1]
    E = el.shape[0]
    nnz = int(rowptr[-1])
    inc_ptr = np.zeros(N + 1, np.int32)
    inc = np.zeros(max(w * E, 1), np.int32)
    slot_ptr = np.zeros(nnz + 1, np.int32)
    slot_src = np.zeros(max(w * w * E, 1), np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = lib.nbp_vms_maps(N, p(rowptr), p(col), E, w, p(np.ascontiguousarray(el, np.int32)), p(inc_ptr), p(inc),
                          p(slot_ptr), p(slot_src))
    return st, inc_ptr, inc[:w * E], slot_ptr, slot_src[:w * w * E]


@pytest.fixture(scope="module")
def lib():
    from paper_1911_10814_gb300 import nbp
    return nbp.load()


@pytest.mark.parametrize("kind", ["tets", "tris"])
def test_maps_match_brute_force(lib, kind):
    sp = synth.MeshSpec(3, 2, 4, R=(1e3, 1e4), name="box3x2x4")
    d, m = synth.generate(sp), synth.mesh(sp)
    N, rp, col = d["n_nodes"], d["rowptr"], d["col"]
    el = m[kind]
    w = el.shape[1]
    st, inc_ptr, inc, slot_ptr, slot_src = _maps(lib, rp, col, el, N)
    assert st == 0
    for A in range(N):
        ref = [w * e + a for e in range(len(el)) for a in range(w) if el[e, a] == A]
        assert list(inc[inc_ptr[A]:inc_ptr[A + 1]]) == ref
    for A in range(N):
        for s in range(rp[A], rp[A + 1]):
            B = col[s]
            ref = [w * w * e + w * a + b for e in range(len(el)) for a in range(w) for b in range(w)
                   if el[e, a] == A and el[e, b] == B]
            assert list(slot_src[slot_ptr[s]:slot_ptr[s + 1]]) == ref
    # every element pair lands in exactly one slot
    assert slot_ptr[-1] == w * w * len(el)


def test_maps_reject_pairs_outside_the_pattern(lib):
    sp = synth.MeshSpec(2, 2, 2, R=(1e3,), name="box2")
    d = synth.generate(sp)
    N = d["n_nodes"]
    el = np.array([[0, 1, 2, N - 1]], np.int32)       # corner to corner: not neighbours
    st, *_ = _maps(lib, d["rowptr"], d["col"], el, N)
    assert st == 1                                      # NBP_ERR_INVALID
    st, *_ = _maps(lib, d["rowptr"], d["col"], np.array([[0, 1, 2, N]], np.int32), N)
    assert st == 1
