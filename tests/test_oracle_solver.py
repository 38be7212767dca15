"""Pins of the oracle's IC(0), triangular solves, SpMV and PCG (A3, A7) to
textbook facts: Cholesky on no-fill patterns, the IC(0) identity on the
pattern, a dense masked brute force, CG's finite termination, Eq.(6), and the
equivalence of PCG with CG on the split-preconditioned system."""
import numpy as np
import pytest
from scipy.linalg import solve_triangular

import oracle as O
from paper_2412_07127_gb300 import inputs as I


def _spd_sparse(n, density, seed):
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density) * rng.standard_normal((n, n))
    S = M + M.T
    return S + np.diag(np.abs(S).sum(1) + 1.0)


def _dense_ic0(D):
    """IC(0) brute force: dense right-looking Cholesky with every update
    outside the pattern of D dropped."""
    n = D.shape[0]
    P = D != 0
    W = np.tril(D).astype(float)
    for k in range(n):
        W[k, k] = np.sqrt(W[k, k])
        for i in range(k + 1, n):
            if P[i, k]:
                W[i, k] /= W[k, k]
        for j in range(k + 1, n):
            for i in range(j, n):
                if P[i, j] and P[i, k] and P[j, k]:
                    W[i, j] -= W[i, k] * W[j, k]
    return np.tril(W)


def test_ic0_diagonal_and_tridiagonal_is_cholesky():
    rng = np.random.default_rng(0)
    d = rng.uniform(1, 5, 40)
    L, bad = O.ic0(O.csr_from_dense(np.diag(d)))
    assert bad == -1
    assert np.allclose(L.to_dense(), np.diag(np.sqrt(d)), rtol=1e-15)
    n = 60
    T = np.diag(rng.uniform(3, 4, n)) + np.diag(rng.uniform(-1, 1, n - 1), -1)
    T = np.tril(T) + np.tril(T, -1).T
    L, bad = O.ic0(O.csr_from_dense(T))
    assert bad == -1
    assert np.allclose(L.to_dense(), np.linalg.cholesky(T), rtol=1e-14, atol=1e-15)


def test_ic0_block_diagonal_dense_blocks_is_cholesky():
    rng = np.random.default_rng(1)
    blocks = []
    for s in (3, 5, 4):
        M = rng.standard_normal((s, s))
        blocks.append(M @ M.T + s * np.eye(s))
    from scipy.linalg import block_diag
    D = block_diag(*blocks)
    L, bad = O.ic0(O.csr_from_dense(D))
    assert bad == -1
    assert np.allclose(L.to_dense(), np.linalg.cholesky(D), rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("which", ["fem2", "rand"])
def test_ic0_matches_dense_brute_force(which):
    if which == "fem2":
        A = O.fem_hex_assemble(2, I.material_field(2, 7))
        D = A.to_dense()
    else:
        D = _spd_sparse(150, 0.04, 3)
        A = O.csr_from_dense(D)
    L, bad = O.ic0(A)
    assert bad == -1
    W = _dense_ic0(D)
    assert np.allclose(L.to_dense(), W, rtol=1e-12, atol=1e-12 * np.abs(W).max())


def test_ic0_identity_on_pattern_fem():
    N = 4
    A = O.fem_hex_assemble(N, I.material_field(N, 2))
    L, bad = O.ic0(A)
    assert bad == -1
    Ld = L.to_dense()
    D = A.to_dense()
    P = np.tril(D) != 0
    R = (Ld @ Ld.T - D)[P]
    assert np.abs(R).max() <= 1e-12 * np.abs(D).max()
    assert np.all(L.to_dense()[~P] == 0)


def test_ic0_breakdown_row_and_shift():
    D = np.array([[1.0, 2.0, 0.0], [2.0, 1.0, 0.5], [0.0, 0.5, 3.0]])
    L, bad = O.ic0(O.csr_from_dense(D))
    assert bad == 1
    L, alpha, bad = O.ic0_auto(O.csr_from_dense(D))
    assert bad == -1
    # 1 + alpha needs (1+alpha)^2 > 4: alpha = 1e-3 * 2^k first exceeding 1
    assert alpha == 1e-3 * 2 ** 10
    Ls = L.to_dense()
    Ds = D + alpha * np.diag(np.diag(D))
    P = np.tril(D) != 0
    assert np.allclose((Ls @ Ls.T)[P], Ds[P], rtol=1e-13)


def test_spmv_and_triangular_solves_vs_dense():
    N = 3
    A = O.fem_hex_assemble(N, I.material_field(N, 5))
    D = A.to_dense()
    x = np.random.default_rng(0).standard_normal(A.n)
    assert np.allclose(O.spmv(A, x), D @ x, rtol=1e-13, atol=1e-13 * np.abs(D).max())
    L, _ = O.ic0(A)
    Ld = L.to_dense()
    y = O.lsolve(L, x)
    assert np.allclose(y, solve_triangular(Ld, x, lower=True), rtol=1e-11, atol=1e-12)
    z = O.ltsolve(L, y)
    assert np.allclose(z, solve_triangular(Ld.T, y, lower=False), rtol=1e-11, atol=1e-12)


def test_cg_finite_termination_distinct_eigenvalues():
    """CG on a matrix with k distinct eigenvalues terminates in k steps."""
    rng = np.random.default_rng(4)
    n = 120
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat([1.0, 2.0, 5.0, 9.0, 20.0], n // 5)
    D = (Q * lam) @ Q.T
    D = (D + D.T) / 2
    A = O.csr_from_dense(D)
    b = rng.uniform(-1, 1, n)
    r = O.pcg(A, b, None, tol=1e-10)
    assert r["status"] == 0 and r["iters"] <= 6
    assert np.allclose(r["x"], np.linalg.solve(D, b), rtol=1e-8)


def test_pcg_converges_within_n_and_matches_dense_solve():
    D = _spd_sparse(180, 0.03, 9)
    A = O.csr_from_dense(D)
    b = np.random.default_rng(1).uniform(-1, 1, 180)
    for L in (None, O.ic0(A)[0]):
        r = O.pcg(A, b, L, tol=1e-12, maxit=180)
        assert r["status"] == 0 and r["iters"] <= 180
        x = np.linalg.solve(D, b)
        assert np.linalg.norm(r["x"] - x) <= 1e-9 * np.linalg.norm(x)


def test_pcg_with_exact_cholesky_takes_one_iteration():
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 0))
    D = A.to_dense()
    C = np.linalg.cholesky(D)
    Lfull = O.csr_from_dense(C, lower=True)
    b = I.rhs(A.n, 0)
    r = O.pcg(A, b, Lfull, tol=1e-10)
    assert r["iters"] == 1 and r["status"] == 0


def test_cg_error_bound_eq6():
    """Eq.(6): ||x* - x_l||_A <= 2 ||x* - x0||_A ((sqrt k - 1)/(sqrt k + 1))^l."""
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 1))
    D = A.to_dense()
    b = I.rhs(A.n, 1)
    xs = np.linalg.solve(D, b)
    w = np.linalg.eigvalsh(D)
    kap = w[-1] / w[0]
    q = (np.sqrt(kap) - 1) / (np.sqrt(kap) + 1)
    r = O.pcg(A, b, None, tol=1e-12, history=True)
    anorm = lambda v: np.sqrt(v @ D @ v)
    e0 = anorm(xs)
    for l, x in enumerate(r["hist"], start=1):
        assert anorm(xs - x) <= 2 * e0 * q ** l * (1 + 1e-9) + 1e-12


def test_pcg_equals_cg_on_split_system():
    """PCG with P = L L^T produces x_k = L^-T xhat_k where xhat_k are the CG
    iterates on (L^-1 A L^-T) xhat = L^-1 b (textbook equivalence)."""
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 6))
    D = A.to_dense()
    L, _ = O.ic0(A)
    Ld = L.to_dense()
    b = I.rhs(A.n, 6)
    Li = np.linalg.inv(Ld)
    Ah = Li @ D @ Li.T
    Ah = (Ah + Ah.T) / 2
    bh = Li @ b
    r1 = O.pcg(A, b, L, tol=1e-12, history=True)
    r2 = O.pcg(O.csr_from_dense(Ah), bh, None, tol=1e-12, history=True)
    k = min(8, len(r1["hist"]), len(r2["hist"]))
    for t in range(k):
        xa = r1["hist"][t]
        xb = Li.T @ r2["hist"][t]
        assert np.linalg.norm(xa - xb) <= 1e-8 * np.linalg.norm(xa)


def test_pcg_zero_rhs_and_converged_start():
    A = O.fem_hex_assemble(2, I.material_field(2, 0))
    r = O.pcg(A, np.zeros(A.n), None)
    assert r["iters"] == 0 and np.all(r["x"] == 0)
    b = I.rhs(A.n, 2)
    x = np.linalg.solve(A.to_dense(), b)
    r = O.pcg(A, b, None, x0=x, tol=1e-8)
    assert r["iters"] == 0


def test_fem8_ic0_pcg_reaches_tolerance():
    N = 8
    A = O.fem_hex_assemble(N, I.material_field(N, 0))
    L, alpha, bad = O.ic0_auto(A)
    assert bad == -1
    b = I.rhs(A.n, 0)
    r = O.pcg(A, b, L, tol=1e-8)
    r0 = O.pcg(A, b, None, tol=1e-8)
    assert r["status"] == 0 and r["relres"] <= 1e-8
    assert r["iters"] < r0["iters"] / 4
    res = b - O.spmv(A, r["x"])
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(b)
