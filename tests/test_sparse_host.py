"""Host-side checks of the sparse entry points, without a GPU: malformed
compressed-sparse-row descriptors and out-of-range sizes are refused with
GRBK_EINVAL before any device work, and the binding builds the CSR arrays the
C ABI expects (offsets from 0 to nnz, ascending columns per row)."""
import numpy as np
import pytest

import paper_2408_05444_gb300 as g
from paper_2408_05444_gb300 import build as gbuild


@pytest.fixture(scope="module", autouse=True)
def built():
    gbuild.build()


def _csr(rows, cols, rowptr, colind, val):
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    v = np.ascontiguousarray(val, dtype=np.float64)
    keep = (rp, ci, v)
    return g.grbk_csr(rows, cols, len(v), rp.ctypes.data, ci.ctypes.data, v.ctypes.data), keep


def _create(A, B, C):
    import ctypes
    a = (g.grbk_csr * 1)(A)
    b = (g.grbk_csr * 1)(B)
    c = g._mat_array([C])
    h = ctypes.c_void_p()
    return g.lib().grbk_sparse_create(ctypes.byref(h), 1, a, b, c, None)


def test_binding_builds_csr_arrays():
    D = np.array([[0.0, 2.0, 0.0, 1.0], [0.0, 0.0, 0.0, 0.0], [3.0, 0.0, 4.0, 0.0]])
    rows, cols, rp, ci, v = g.csr_arrays(D)
    assert (rows, cols) == (3, 4)
    assert rp.tolist() == [0, 2, 2, 4] and ci.tolist() == [1, 3, 0, 2] and v.tolist() == [2.0, 1.0, 3.0, 4.0]
    sps = pytest.importorskip("scipy.sparse")
    M = sps.csr_matrix(D)
    M.indices = M.indices[::-1].copy()      # unsorted indices are sorted by the binding
    M.data = M.data[::-1].copy()
    M.has_sorted_indices = False
    rows2, cols2, rp2, ci2, v2 = g.csr_arrays(M)
    assert rp2.tolist() == rp.tolist()
    for i in range(3):
        seg = slice(rp2[i], rp2[i + 1])
        assert list(ci2[seg]) == sorted(ci2[seg])


@pytest.mark.parametrize("case", ["unsorted", "duplicate", "range", "rowptr_start", "rowptr_end", "rowptr_decreasing"])
def test_malformed_csr_is_refused(case):
    good = dict(rows=2, cols=3, rowptr=[0, 2, 3], colind=[0, 2, 1], val=[1.0, 2.0, 3.0])
    bad = dict(good)
    if case == "unsorted":
        bad.update(colind=[2, 0, 1])
    elif case == "duplicate":
        bad.update(colind=[1, 1, 1])
    elif case == "range":
        bad.update(colind=[0, 3, 1])
    elif case == "rowptr_start":
        bad.update(rowptr=[1, 2, 3])
    elif case == "rowptr_end":
        bad.update(rowptr=[0, 2, 2])
    elif case == "rowptr_decreasing":
        bad.update(rowptr=[0, 3, 2], colind=[0, 1, 2])
    A, ka = _csr(**bad)
    B, kb = _csr(3, 2, [0, 1, 2, 2], [0, 1], [1.0, 1.0])
    C = np.zeros((2, 2))
    assert _create(A, B, C) == g.GRBK_EINVAL


def test_shape_mismatch_and_limits_are_refused():
    A, ka = _csr(2, 3, [0, 1, 2], [0, 1], [1.0, 1.0])
    B, kb = _csr(3, 2, [0, 1, 2, 2], [0, 1], [1.0, 1.0])
    assert _create(A, B, np.zeros((3, 2))) == g.GRBK_EINVAL          # C must be m x n
    Bw, kw = _csr(3, 2000, [0, 1, 2, 2], [0, 1], [1.0, 1.0])         # n above 1024
    assert _create(A, Bw, np.zeros((2, 2000))) == g.GRBK_EINVAL
