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


def test_row_groups():
    A = O.fem_hex_assemble(3, I.material_field(3, 1))
    assert np.array_equal(O.row_groups(A), np.arange(0, A.n + 1, 3))      # a node's three dofs
    D = np.eye(6) * 4
    D[2, 0] = D[0, 2] = D[3, 0] = D[0, 3] = D[3, 1] = D[1, 3] = -1       # rows 2 and 3 differ
    st = O.row_groups(O.csr_from_dense(D), gmax=2)
    assert list(st) == [0, 1, 2, 3, 4, 5, 6]
    E = 4 * np.eye(5) + np.ones((5, 5))                                   # dense: one run
    assert list(O.row_groups(O.csr_from_dense(E), gmax=2)) == [0, 2, 4, 5]
    # runs of 6 and 3 rows: cut at their common length 3
    F = 4 * np.eye(9)
    F[:6, :6] += 1
    F[6:, 6:] += 1
    assert list(O.row_groups(O.csr_from_dense(F))) == [0, 3, 6, 9]
    # runs of 6 and 4 rows: common length 2
    F = 4 * np.eye(10)
    F[:6, :6] += 1
    F[6:, 6:] += 1
    assert list(O.row_groups(O.csr_from_dense(F))) == [0, 2, 4, 6, 8, 10]


def test_dropout_grouped():
    A = O.fem_hex_assemble(3, I.material_field(3, 2))
    L, _ = O.ic0(A)
    st = O.row_groups(A)
    same = O.dropout_grouped(L, 0.0, st)
    assert np.array_equal(same.col, L.col) and np.array_equal(same.val, L.val)
    # with one row per group it is the entry-wise dropout
    single = np.arange(L.n + 1, dtype=np.int32)
    thr = 0.05 * np.abs(L.val).max()
    a, b = O.dropout_grouped(L, thr, single), O.dropout(L, thr)
    assert np.array_equal(a.rowptr, b.rowptr) and np.array_equal(a.col, b.col) and np.array_equal(a.val, b.val)
    # grouped keeps a superset of the entries, and the groups' rows stay alike
    g = O.dropout_grouped(L, thr, st)
    assert len(g.col) >= len(b.col)
    for k in range(len(st) - 1):
        s, e = st[k], st[k + 1]
        ext = [set(c for c in g.col[g.rowptr[r]:g.rowptr[r + 1]] if c < s) for r in range(s, e)]
        assert all(x == ext[0] for x in ext)


def test_dropout_grouped_hand_case():
    # rows 1 and 2 form a group (identical columns {0, 1, 2}); column 0 is kept
    # for both because row 2's entry is large, although row 1's is small
    D = np.array([[4.0, 0.005, -0.5], [0.005, 2.0, 0.1], [-0.5, 0.1, 3.0]])
    L = O.lower(O.csr_from_dense(D))
    Lv = O.CSR(L.rowptr, L.col, np.array([2.0, 0.005, 1.0, -0.5, 0.1, 3.0]))
    g = O.dropout_grouped(Lv, 0.01, np.array([0, 1, 3], np.int32))
    assert list(g.col) == [0, 0, 1, 0, 1, 2]


def test_dropout_grouped_blocks():
    # groups {0, 1} and {2, 3}: the external block rows 2-3 x columns 0-1
    # stays whole when one of its four entries is large, and leaves whole
    # when none is; in-group entries (1,0) and (3,2) always stay
    L = O.lower(O.csr_from_dense(np.ones((4, 4)) + 4 * np.eye(4)))
    st = np.array([0, 2, 4], np.int32)
    small = np.array([2.0, 0.001, 2.0, 0.002, 0.003, 2.0, 0.004, 0.005, 0.006, 2.0])
    big = small.copy()
    big[7] = 0.5                                       # entry (3, 1)
    kb = O.dropout_grouped(O.CSR(L.rowptr, L.col, big), 0.01, st)
    assert list(kb.rowptr) == [0, 1, 3, 6, 10] and np.array_equal(kb.val, big)
    ks = O.dropout_grouped(O.CSR(L.rowptr, L.col, small), 0.01, st)
    assert list(ks.rowptr) == [0, 1, 3, 4, 6]
    assert list(ks.col) == [0, 0, 1, 2, 2, 3]
    assert np.array_equal(ks.val, small[[0, 1, 2, 5, 8, 9]])


def test_dropout_grouped_keeps_node_blocks():
    # hex elasticity: every external node block is kept with all 9 entries or
    # none, so S = L' + L'^T keeps A's row groups (one per node)
    N = 3
    A = O.fem_hex_assemble(N, I.material_field(N, 4))
    L, _ = O.ic0(A)
    st = O.row_groups(A)
    thr = 0.05 * np.abs(L.val).max()
    g = O.dropout_grouped(L, thr, st)
    assert len(g.col) < len(L.col)
    gof = np.repeat(np.arange(len(st) - 1), np.diff(st))
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    blocks = {}
    for r, c in zip(rows, g.col):
        blocks[(gof[r], gof[c])] = blocks.get((gof[r], gof[c]), 0) + 1
    assert all(v == 9 or (a == b and v == 6) for (a, b), v in blocks.items())
    D = np.zeros((g.n, g.n))
    D[rows, g.col] = 1
    S = O.csr_from_dense(D + D.T + np.eye(g.n))
    assert np.array_equal(O.row_groups(S), st)
