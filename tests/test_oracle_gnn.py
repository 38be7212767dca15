"""Pins of the oracle's graph inputs, GNN correction, probe loss, gradients and
Adam (A4-A6, A8-A10): hand-worked features, g = 0 => L = L_IC, an independent
vectorised dense restatement of the network, the Hutchinson estimator's
unbiasedness (Eq.(4)), and central finite differences for every gradient."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2412_07127_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_features_hand_worked_4x4():
    g = json.load(open(os.path.join(GOLD, "features_4x4.json")))
    A = O.csr_from_dense(np.array(g["A"], float))
    x9, e, s = O.features(A)
    assert np.allclose(x9[:, :7], np.array(g["x9_without_position"]), rtol=1e-15)
    idx = np.arange(4)
    assert np.allclose(x9[:, 7], np.sin(idx)) and np.allclose(x9[:, 8], np.cos(idx))
    assert np.isclose(s * s, g["scale_squared"], rtol=1e-14)
    assert np.allclose(e, np.array(g["tril_values_row_order"]) / s, rtol=1e-15)


def _theta(seed, out_scale=1.0):
    return I.gnn_init(seed, out_scale=out_scale)


def _dense_gnn(T, x9, e0, theta, bf16=False):
    """Independent restatement: edge lists, numpy matmuls, an incidence
    matrix for the sum aggregation."""
    sl = I.param_slices()
    P = lambda k: theta[sl[k][0]:sl[k][0] + int(np.prod(sl[k][1]))].reshape(sl[k][1])
    rb = (lambda a: O.round_bf16(a)) if bf16 else (lambda a: a)
    n = T.n
    rows = np.repeat(np.arange(n), np.diff(T.rowptr))
    cols = T.col.astype(np.int64)
    E = len(cols)
    B = np.zeros((n, E))
    B[rows, np.arange(E)] = 1.0
    B[cols, np.arange(E)] = 1.0
    deg = B.sum(1)
    mu = x9.mean(0)
    c = x9 - P("gn_alpha") * mu
    sig = np.sqrt((c ** 2).mean(0) + 1e-5)
    x = P("gn_gamma") * c / sig + P("gn_beta")
    e = e0.copy()
    for l in range(3):
        h = np.concatenate([e[:, None], e0[:, None], x[rows], x[cols]], axis=1)
        a = np.tanh(rb(h) @ rb(P(f"W1_{l}")).T + P(f"b1_{l}"))
        e_new = a @ P(f"W2_{l}") + P(f"b2_{l}")[0]
        if l < 2:
            S = B @ e_new
            M = S / deg
            u = np.concatenate([x, S[:, None], M[:, None]], axis=1)
            rn = (lambda a: O.round_bf16(a)) if bf16 == 3 else (lambda a: a)
            x = rn(np.tanh(rn(u) @ rn(P(f"W3_{l}")).T + P(f"b3_{l}"))) @ rn(P(f"W4_{l}")).T + P(f"b4_{l}")
        e = e_new
    return e


@pytest.mark.parametrize("bf16", [False, True, 3])
def test_gnn_forward_matches_dense_restatement(bf16):
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 3))
    T = O.lower(A)
    x9, e0, s = O.features(A)
    theta = _theta(1)
    g = O.gnn_forward(T, x9, e0, theta, bf16=bf16)
    gd = _dense_gnn(T, x9, e0, theta, bf16=bf16)
    assert np.allclose(g, gd, rtol=1e-12, atol=1e-12)


def test_bf16_rounding_rule():
    # ties to even at 8 significant bits
    assert O.round_bf16(1.0 + 2 ** -8) == 1.0
    assert O.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6
    assert O.round_bf16(1.0 + 2 ** -8 + 2 ** -20) == 1.0 + 2 ** -7
    assert O.round_bf16(-3.0) == -3.0


def test_zero_output_layer_gives_ic0():
    N = 3
    A = O.fem_hex_assemble(N, I.material_field(N, 2))
    T = O.lower(A)
    x9, e0, s = O.features(A)
    theta = _theta(2)
    off, shape = I.param_slices()["W2_2"]
    theta[off:off + 32] = 0.0
    off, _ = I.param_slices()["b2_2"]
    theta[off] = 0.0
    g = O.gnn_forward(T, x9, e0, theta)
    assert np.all(g == 0.0)
    L, _ = O.ic0(A)
    assert np.array_equal(O.correct(T, L.val, g), L.val)


def test_correction_keeps_positive_diagonal():
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 2))
    T = O.lower(A)
    L, _ = O.ic0(A)
    g = np.random.default_rng(0).normal(0, 5, T.nnz)
    Lc = O.correct(T, L.val, g)
    diag = T.rowptr[1:] - 1
    assert np.all(Lc[diag] > 0)
    off = np.setdiff1d(np.arange(T.nnz), diag)
    assert np.allclose(Lc[off], L.val[off] + g[off], rtol=1e-15)
    assert np.allclose(Lc[diag], L.val[diag] * np.exp(g[diag] / 2), rtol=1e-15)


def test_correct_backward_finite_differences():
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 2))
    T = O.lower(A)
    L, _ = O.ic0(A)
    rng = np.random.default_rng(4)
    g = rng.normal(0, 0.3, T.nnz)
    c = rng.standard_normal(T.nnz)
    dg = O.correct_backward(T, L.val, g, c)
    h = 1e-6
    for p in range(0, T.nnz, 7):
        gp, gm = g.copy(), g.copy()
        gp[p] += h
        gm[p] -= h
        fd = (c @ O.correct(T, L.val, gp) - c @ O.correct(T, L.val, gm)) / (2 * h)
        assert np.isclose(dg[p], fd, rtol=1e-7, atol=1e-9)


def test_probe_loss_single_probe_equals_dense():
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 8))
    L, _ = O.ic0(A)
    rng = np.random.default_rng(1)
    L.val = L.val * (1 + 0.1 * rng.standard_normal(L.nnz))
    D, Ld = A.to_dense(), L.to_dense()
    z = rng.standard_normal(A.n)
    assert np.isclose(O.probe_loss(A, L, z[None]), np.sum(((Ld @ Ld.T - D) @ z) ** 2), rtol=1e-12)


def test_probe_loss_unbiased_frobenius():
    """Eq.(4): E_z ||(LL^T - A) z||^2 = ||LL^T - A||_F^2 for Gaussian and
    Rademacher z; the mean of 20000 probes lies within 4 standard errors."""
    N = 1
    A = O.fem_hex_assemble(N, I.material_field(N, 8))
    L, _ = O.ic0(A)
    rng = np.random.default_rng(3)
    L.val = L.val * (1 + 0.2 * rng.standard_normal(L.nnz))
    D, Ld = A.to_dense(), L.to_dense()
    fro2 = np.sum((Ld @ Ld.T - D) ** 2)
    for kind in ("gaussian", "rademacher"):
        Z = I.probes(20000, A.n, 5, kind).astype(np.float64)
        per = np.array([O.probe_loss(A, L, Z[k:k + 1]) for k in range(0, 20000, 1)])
        se = per.std() / np.sqrt(len(per))
        assert abs(per.mean() - fro2) < 4 * se


def test_probe_loss_gradient_finite_differences():
    N = 1
    A = O.fem_hex_assemble(N, I.material_field(N, 9))
    L, _ = O.ic0(A)
    Z = I.probes(3, A.n, 2).astype(np.float64)
    loss, dL = O.probe_loss(A, L, Z, grad=True)
    h = 1e-6
    for p in range(L.nnz):
        Lp = O.CSR(L.rowptr, L.col, L.val.copy())
        Lm = O.CSR(L.rowptr, L.col, L.val.copy())
        Lp.val[p] += h
        Lm.val[p] -= h
        fd = (O.probe_loss(A, Lp, Z) - O.probe_loss(A, Lm, Z)) / (2 * h)
        assert np.isclose(dL[p], fd, rtol=1e-6, atol=1e-6 * (1 + abs(loss)))


def test_gnn_backward_finite_differences():
    """d/dtheta of sum_p c_p g_p(theta) against central differences, for every
    one of the 3504 parameters, on a 16-row random sparse SPD matrix whose
    rows differ in degree (so no GraphNorm feature has zero variance)."""
    rng = np.random.default_rng(4)
    n = 16
    M = (rng.random((n, n)) < 0.25) * rng.standard_normal((n, n))
    D = M + M.T + np.diag(rng.uniform(4, 8, n))
    A = O.csr_from_dense(D)
    T = O.lower(A)
    x9, e0, s = O.features(A)
    theta = _theta(3)
    c = np.random.default_rng(6).standard_normal(T.nnz)
    grad = O.gnn_backward(T, x9, e0, theta, c)
    h = 1e-5
    fd = np.zeros_like(theta)

    def f(k, d):
        t = theta.copy()
        t[k] += d
        return c @ O.gnn_forward(T, x9, e0, t)

    for k in range(theta.size):  # fourth-order central difference
        fd[k] = (-f(k, 2 * h) + 8 * f(k, h) - 8 * f(k, -h) + f(k, -2 * h)) / (12 * h)
    assert np.all(np.abs(grad - fd) <= 1e-6 * np.maximum(np.abs(fd), 1.0))
    # every parameter group receives gradient
    for name, (off, shape) in I.param_slices().items():
        size = int(np.prod(shape))
        assert np.abs(grad[off:off + size]).max() > 0, name


def test_adam_constant_gradient_steps():
    """With a constant gradient the bias-corrected Adam step is
    lr * g / (|g| + eps) at every step."""
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 2.0])
    m1 = np.zeros(3); m2 = np.zeros(3)
    t0 = theta.copy()
    for t in range(1, 6):
        O.adam_step(theta, g, m1, m2, t, 0.005)
        assert np.allclose(theta, t0 - t * 0.005 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert O.lr_at(0, 10) == 0.0 and O.lr_at(5, 10) == 0.0025 and O.lr_at(50, 10) == 0.005


# ---------------------------------------------------------------- closed forms of the forward
def _set(theta, name, index, value):
    """theta[name][index] = value (index a tuple into the parameter's shape)."""
    off, shape = I.param_slices()[name]
    theta[off + int(np.ravel_multi_index(index, shape))] = value


def _graph(n, seed):
    """A random symmetric pattern with a stored diagonal (diagonally dominant)."""
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < 0.15) * rng.standard_normal((n, n))
    S = M + M.T
    A = O.csr_from_dense(S + np.diag(np.abs(S).sum(1) + 1.0))
    return A, O.lower(A)


def test_graphnorm_output_moments_closed_form():
    """GraphNorm: out = gamma (x - alpha mu) / sqrt(m2 + 1e-5) + beta with m2
    the mean square of x - alpha mu, so per feature mean(out) = gamma (1 -
    alpha) mu / sqrt(m2 + 1e-5) + beta and mean((out - beta)^2) = gamma^2 m2
    / (m2 + 1e-5), m2 = var(x) + ((1 - alpha) mu)^2."""
    A, T = _graph(40, 3)
    rng = np.random.default_rng(4)
    x9 = rng.standard_normal((A.n, 9)) * 2.0 + 0.7
    e0 = rng.standard_normal(T.nnz)
    th = np.zeros(I.N_PARAMS)
    gam, bet, alp = rng.uniform(0.5, 2, 9), rng.standard_normal(9), rng.uniform(0, 1, 9)
    for f in range(9):
        _set(th, "gn_gamma", (f,), gam[f])
        _set(th, "gn_beta", (f,), bet[f])
        _set(th, "gn_alpha", (f,), alp[f])
    _, x0, _, _, _ = O.gnn_forward_parts(T, x9, e0, th)
    mu, var = x9.mean(0), x9.var(0)
    m2 = var + ((1 - alp) * mu) ** 2
    assert np.allclose(x0.mean(0), gam * (1 - alp) * mu / np.sqrt(m2 + 1e-5) + bet, rtol=1e-12, atol=1e-12)
    assert np.allclose(((x0 - bet) ** 2).mean(0), gam ** 2 * m2 / (m2 + 1e-5), rtol=1e-12)


def test_aggregation_counts_each_edge_at_both_ends_and_a_self_loop_once():
    """Block 0's edge outputs all 1 (W2 = 0, b2 = 1): a node's sum is its
    incident-edge count, which on a symmetric pattern with a stored diagonal
    is the full row count of A; its mean is 1."""
    A, T = _graph(50, 5)
    rng = np.random.default_rng(6)
    th = np.zeros(I.N_PARAMS)
    _set(th, "b2_0", (0,), 1.0)
    _, _, S0, M0, _ = O.gnn_forward_parts(T, rng.standard_normal((A.n, 9)), rng.standard_normal(T.nnz), th)
    assert np.array_equal(S0, np.diff(A.rowptr).astype(float))
    assert np.array_equal(M0, np.ones(A.n))


def test_aggregation_sums_edge_values_over_the_full_row():
    """Block 0's edge output ~ e0 (one hidden unit in its linear range: tanh(eps
    e0) / eps = e0 + O(eps^2)): with e0 = tril(A) / s, a node's sum is its full
    row sum of A over s (the lower entries of its row plus, through the
    transposed edges, those of its column) and its mean that over the row
    count."""
    A, T = _graph(50, 7)
    x9, e0, s = O.features(A)
    eps = 1e-5
    th = np.zeros(I.N_PARAMS)
    _set(th, "W1_0", (0, 1), eps)
    _set(th, "W2_0", (0,), 1.0 / eps)
    _, _, S0, M0, _ = O.gnn_forward_parts(T, x9, e0, th)
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    rowsum = np.bincount(rows, weights=A.val, minlength=A.n) / s
    cnt = np.diff(A.rowptr).astype(float)
    tol = 1e-9 * np.abs(A.val).max() / s * cnt.max()
    assert np.max(np.abs(S0 - rowsum)) <= tol
    assert np.max(np.abs(M0 - rowsum / cnt)) <= tol


def test_gnn_forward_hand_worked_two_nodes():
    gold = json.load(open(os.path.join(GOLD, "gnn_2node.json")))
    A = O.csr_from_dense(np.array([[4.0, -1.0], [-1.0, 3.0]]))
    T = O.lower(A)
    th = np.zeros(I.N_PARAMS)
    for key, val in gold["weights"].items():
        if isinstance(val, list):
            for f, v in enumerate(val):
                _set(th, key, (f,), v)
            continue
        name, idx = (key.split("[", 1) + [""])[:2]
        index = tuple(int(k) for k in idx.replace("]", " ").replace("[", " ").split()) or (0,)
        _set(th, name, index, val)
    g, x0, S0, M0, x1 = O.gnn_forward_parts(T, np.array(gold["x9"]), np.array(gold["e0"]), th)
    assert np.allclose(S0, gold["S0"], rtol=1e-14, atol=1e-15)
    assert np.allclose(M0, gold["M0"], rtol=1e-14, atol=1e-15)
    assert np.allclose(x1[:, :2], gold["x1_f0_f1"], rtol=1e-14, atol=1e-15)
    assert np.allclose(g, gold["g"], rtol=1e-14, atol=1e-15)


def _two_copies(A):
    """A (+) A: the block-diagonal matrix of two disjoint copies of A."""
    n, nnz = A.n, A.nnz
    rowptr = np.concatenate([A.rowptr, A.rowptr[1:] + nnz])
    return O.CSR(rowptr, np.concatenate([A.col, A.col + n]), np.concatenate([A.val, A.val]))


def test_two_disjoint_copies_give_each_copy_its_own_output():
    """One graph made of two disjoint copies of a graph: the features are the
    copy's own except the row position (sin i, cos i), the scale s (a
    population deviation) is unchanged, and with the copy's inputs stacked
    twice the network's output is the copy's output twice: messages stay
    within a component (one added to the next row instead of its own leaks
    across the border between the copies) and GraphNorm's statistics are
    means over all nodes, unchanged by duplication (a divisor other than
    the node count would change them). Both mistakes, planted in the
    oracle, fail this test."""
    A, T = _graph(36, 11)
    A2 = _two_copies(A)
    T2 = O.lower(A2)
    assert np.array_equal(T2.rowptr, np.concatenate([T.rowptr, T.rowptr[1:] + T.nnz]))
    x9, e0, s = O.features(A)
    x92, e02, s2 = O.features(A2)
    assert abs(s2 - s) <= 1e-14 * s
    assert np.allclose(x92[:A.n, :7], x9[:, :7], rtol=1e-13, atol=1e-13)
    assert np.allclose(x92[A.n:, :7], x9[:, :7], rtol=1e-13, atol=1e-13)
    assert np.allclose(x92[:, 7], np.sin(np.arange(2 * A.n)), atol=1e-13)
    assert np.allclose(e02, np.concatenate([e0, e0]), rtol=1e-13, atol=1e-15)
    th = I.gnn_init(3, out_scale=1.0)
    rng = np.random.default_rng(12)
    for name in ("gn_gamma", "gn_beta", "gn_alpha"):
        off, shape = I.param_slices()[name]
        th[off:off + int(np.prod(shape))] = rng.uniform(0.3, 1.5, int(np.prod(shape)))
    g = O.gnn_forward(T, x9, e0, th)
    g2 = O.gnn_forward(T2, np.vstack([x9, x9]), np.concatenate([e0, e0]), th)
    assert np.abs(g).max() > 0
    assert np.allclose(g2, np.concatenate([g, g]), rtol=1e-11, atol=1e-13 * np.abs(g).max())
