"""Oracle pins of fill-in dropout (Supplementary 5, Eq. (10)) and of the
factor deviation diagnostic (Figure 5)."""
import numpy as np

import oracle as O
from paper_2412_07127_gb300 import inputs as I


def _dense_lower(L):
    D = np.zeros((L.n, L.n))
    for i in range(L.n):
        for p in range(L.rowptr[i], L.rowptr[i + 1]):
            D[i, L.col[p]] = L.val[p]
    return D


def test_dropout_hand_case():
    D = np.array([[2.0, 0.0, 0.0], [0.005, 1.0, 0.0], [-0.5, 0.001, 3.0]])
    A = O.csr_from_dense(D + np.tril(D, -1).T)
    L = O.lower(A)
    L = O.CSR(L.rowptr, L.col, np.array([2.0, 0.005, 1.0, -0.5, 0.001, 3.0]))
    Ld = O.dropout(L, 0.01)
    assert list(Ld.rowptr) == [0, 1, 2, 4]
    assert list(Ld.col) == [0, 1, 0, 2]
    assert list(Ld.val) == [2.0, 1.0, -0.5, 3.0]


def test_dropout_limits():
    A = O.fem_hex_assemble(3, I.material_field(3, 2))
    L, _ = O.ic0(A)
    same = O.dropout(L, 0.0)
    assert np.array_equal(same.rowptr, L.rowptr) and np.array_equal(same.col, L.col)
    assert np.array_equal(same.val, L.val)
    diag = O.dropout(L, 1e300)
    assert np.array_equal(diag.rowptr, np.arange(L.n + 1))
    assert np.array_equal(diag.col, np.arange(L.n))
    assert np.array_equal(diag.val, np.diag(_dense_lower(L)))
    # a thinned factor still preconditions: PCG converges with it
    b = I.rhs(A.n, 2)
    Lt = O.dropout(L, 0.05 * np.abs(L.val).max())
    assert len(Lt.col) < len(L.col)
    r = O.pcg(A, b, Lt, tol=1e-8)
    assert r["status"] == 0


def test_factor_deviation_hand_case():
    A = O.csr_from_dense(np.array([[4.0, 1.0], [1.0, 3.0]]))
    L = O.lower(A)
    LIC = np.array([2.0, 0.5, 1.0])
    Lp = np.array([2.2, 1.0, 1.0])
    out = O.factor_deviation(L, LIC, Lp)
    assert np.allclose(out, [0.05, 0.1, 1.0, 1.0, 2.0, 1.0], rtol=0, atol=1e-15)
    assert np.array_equal(O.factor_deviation(L, LIC, LIC), [0, 0, 0, 0, 2, 1])
