"""Oracle against the hand-worked fixtures in tests/golden/."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import synth
from golden_io import worked_example, triangle_forms, family_edges


def _eq(res, want):
    assert np.array_equal(res["rowptr"], want.rowptr)
    assert np.array_equal(res["colidx"], want.colidx)
    assert np.array_equal(res["values"].astype(np.int64), want.values)


@pytest.mark.parametrize("meth", [O.MERGE, O.ESC])
def test_worked_example(meth):
    g = worked_example()
    A, B, M = g["A"], g["B"], g["M"]
    Af = A.with_values(A.values.astype(np.float32))
    Bf = B.with_values(B.values.astype(np.float32))
    _eq(O.masked_spgemm(M, Af, Bf, "plus_times_f32", method=meth), g["C_plus_times"])
    _eq(O.masked_spgemm(M, A, B, "plus_times_i64", method=meth), g["C_plus_times"])
    _eq(O.masked_spgemm(M, A, B, "plus_pair_i64", method=meth), g["C_plus_pair"])
    if meth == O.ESC:
        _eq(O.masked_spgemm(M, A, B, "plus_times_i64", complement=True, method=meth), g["C_complement_plus_times"])
        _eq(O.masked_spgemm(M, A, B, "plus_pair_i64", complement=True, method=meth), g["C_complement_plus_pair"])


def test_triangle_fixture():
    for kind, params, want in triangle_forms():
        n, edges = family_edges(kind, params)
        src = np.array([e[0] for e in edges], np.int32)
        dst = np.array([e[1] for e in edges], np.int32)
        g = synth.coo_to_csr(n, n, src, dst, symmetrize=True, drop_loops=True)
        L = synth.degree_relabel_lower(g)
        r = O.masked_spgemm(L, L, L, "plus_pair_i64")
        assert int(r["values"].sum()) == want, (kind, params)
