"""GPU parity of the solver path (A1-A3, A7) against the CPU oracle, through
the C-ABI. Integer work (patterns, levels, groups, breakdown rows) must match
bit for bit; float64 results to round-off; PCG to the stated tolerances:
same 1e-8 relative residual, ||x_gpu - x_oracle|| / ||x_oracle|| <= 1e-6,
iteration counts within 2% (at least 1)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_07127_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, gicpcg
    build.build()
    return gicpcg


@pytest.fixture(scope="module")
def h(G):
    return G.Handle(0)


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(DEV)


def _np(t):
    return t.detach().cpu().numpy()


def _upload(A):
    return _dev(A.rowptr), _dev(A.col), _dev(A.val)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _iters_ok(gi, oi):
    return abs(gi - oi) <= max(1, int(0.02 * oi))


def _spd_pattern(n, density, seed, band=None):
    rng = np.random.default_rng(seed)
    M = (rng.random((n, n)) < density) * rng.standard_normal((n, n))
    if band is not None:
        i, j = np.indices((n, n))
        M[np.abs(i - j) > band] = 0
    S = M + M.T
    return S + np.diag(np.abs(S).sum(1) + 1.0)


# ---------------------------------------------------------------- A1
@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_assemble_matches_oracle(G, h, N):
    E = I.material_field(N, N)
    rp, c, v = G.fem_hex_assemble(h, N, _dev(E))
    A = O.fem_hex_assemble(N, E)
    assert np.array_equal(_np(rp), A.rowptr) and np.array_equal(_np(c), A.col)
    assert _rel(_np(v), A.val) <= 1e-13


def test_assemble_batched_block_diagonal(G, h):
    N, nb = 3, 3
    Es = [I.material_field(N, 100 + k) for k in range(nb)]
    rp, c, v = G.fem_hex_assemble(h, N, _dev(np.concatenate(Es)), nb=nb)
    n, nnz = G.fem_hex_sizes(N)
    rp, c, v = _np(rp), _np(c), _np(v)
    for k in range(nb):
        A = O.fem_hex_assemble(N, Es[k])
        assert np.array_equal(rp[k * n:(k + 1) * n + 1] - k * nnz, A.rowptr)
        assert np.array_equal(c[k * nnz:(k + 1) * nnz] - k * n, A.col)
        assert _rel(v[k * nnz:(k + 1) * nnz], A.val) <= 1e-13


# ---------------------------------------------------------------- A2
@pytest.mark.parametrize("N", [1, 2, 5, 8])
def test_analysis_fem(G, h, N):
    A = O.fem_hex_assemble(N, I.material_field(N, 1))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lr, Lc, lev, grp = (_np(t) for t in P.export(h))
    T = O.lower(A, with_values=False)
    olev, onl = O.levels(T)
    assert np.array_equal(Lr, T.rowptr) and np.array_equal(Lc, T.col)
    assert np.array_equal(lev, olev) and P.nlevels == onl == 21 * N - 9
    assert np.array_equal(grp, _expected_groups(A))
    if N >= 2:  # then every group is the 3 dofs of one node
        assert P.ngroups == A.n // 3 and np.array_equal(grp, np.arange(0, A.n + 1, 3))
        # the hex systems admit the fastest solve kernels (so the tests run them)
        assert P.warp_specialised == 1 and P.level_sliced == 1 and P.slices > 0
        assert P.node_blocks == 1  # 3x3 node blocks: the PCG runs the block SpMV


def _expected_groups(A):
    """Runs of rows with identical column sets, cut at the runs' common
    length (8 when that is 1 or above 8): the oracle's row groups."""
    return O.row_groups(A)


@pytest.mark.parametrize("case", ["random", "banded", "tridiag", "diag"])
def test_analysis_generic(G, h, case):
    if case == "random":
        D = _spd_pattern(300, 0.02, 1)
    elif case == "banded":
        D = _spd_pattern(400, 0.3, 2, band=6)
    elif case == "tridiag":
        D = 4 * np.eye(3000) - np.eye(3000, k=1) - np.eye(3000, k=-1)
    else:
        D = np.diag(np.arange(1.0, 501.0))
    A = O.csr_from_dense(D)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lr, Lc, lev, grp = (_np(t) for t in P.export(h))
    T = O.lower(A, with_values=False)
    olev, onl = O.levels(T)
    assert np.array_equal(Lr, T.rowptr) and np.array_equal(Lc, T.col)
    assert np.array_equal(lev, olev) and P.nlevels == onl
    assert np.array_equal(grp, _expected_groups(A))
    assert P.node_blocks == 0  # none of these is made of 3x3 node blocks


def _node_block_spd(nodes, density, seed):
    """A random SPD matrix made of dense 3x3 node blocks (not a mesh)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((nodes, nodes)) < density
    mask = mask | mask.T | np.eye(nodes, dtype=bool)
    M = np.kron(mask, np.ones((3, 3))) * rng.standard_normal((3 * nodes, 3 * nodes))
    S = M + M.T
    return S + np.diag(np.abs(S).sum(1) + 1.0)


@pytest.mark.parametrize("pipeline", [4, 5])
@pytest.mark.parametrize("nodes,density", [(7, 0.3), (100, 0.05), (333, 0.012)])
def test_pcg_node_block_pattern_matches_oracle(G, h, nodes, density, pipeline):
    """The block SpMV path of the PCG on a non-mesh node-block matrix
    (slices of 32 nodes with ragged widths and a partial last slice; rows
    within the IC(0) kernel's 48 lower entries), with the automatic and the
    pair-sliced solves (where the analysis built them)."""
    A = O.csr_from_dense(_node_block_spd(nodes, density, nodes))
    rp, c, v = _upload(A)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, pipeline) # before the analysis: it builds the pair schedule
    P = G.Pattern(h, rp, c)
    assert P.node_blocks == 1
    b = np.random.default_rng(nodes).uniform(-1, 1, A.n)
    Lg, bad = G.ic0(h, P, v)
    assert bad == -1
    res = G.pcg(h, P, v, Lg, _dev(b), rtol=1e-10)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)
    Lo, _ = O.ic0(A)
    ro = O.pcg(A, b, Lo, tol=1e-10)
    assert res["status"] == 0 and _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    x = _np(res["x"])
    assert np.linalg.norm(x - ro["x"]) <= 1e-8 * np.linalg.norm(ro["x"])
    assert np.linalg.norm(b - O.spmv(A, x)) <= 1e-9 * np.linalg.norm(b)


def test_analysis_rejects_bad_patterns(G, h):
    D = _spd_pattern(50, 0.1, 3)
    A = O.csr_from_dense(D)
    # asymmetric: drop one off-diagonal entry of row 0
    row0 = [p for p in range(A.rowptr[0], A.rowptr[1]) if A.col[p] != 0]
    drop = row0[0]
    col = np.delete(A.col, drop)
    rowptr = A.rowptr.copy()
    rowptr[1:] -= 1
    with pytest.raises(G.GicError) as e:
        G.Pattern(h, _dev(rowptr), _dev(col))
    assert e.value.status == G.GIC_ERR_INVALID_ARG
    # unsorted columns in a row
    col = A.col.copy()
    a, b = A.rowptr[5], A.rowptr[6]
    col[a:b] = col[a:b][::-1]
    with pytest.raises(G.GicError) as e:
        G.Pattern(h, _dev(A.rowptr), _dev(col))
    assert e.value.status == G.GIC_ERR_INVALID_ARG
    # missing diagonal
    D2 = D.copy()
    D2[7, 7] = 0.0
    rp, cl = [0], []
    for i in range(50):
        cl += [j for j in range(50) if D2[i, j] != 0]
        rp.append(len(cl))
    with pytest.raises(G.GicError) as e:
        G.Pattern(h, _dev(np.array(rp, np.int32)), _dev(np.array(cl, np.int32)))
    assert e.value.status == G.GIC_ERR_INVALID_ARG
    # empty input: no rows
    with pytest.raises(G.GicError) as e:
        G.Pattern(h, _dev(np.zeros(1, np.int32)), _dev(np.zeros(0, np.int32)))
    assert e.value.status == G.GIC_ERR_INVALID_ARG


# ---------------------------------------------------------------- A3
@pytest.mark.parametrize("N", [1, 2, 8, 12])
def test_ic0_matches_oracle(G, h, N):
    A = O.fem_hex_assemble(N, I.material_field(N, 3))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, bad = G.ic0(h, P, v)
    Lo, obad = O.ic0(A)
    assert bad == obad == -1
    assert _rel(_np(Lg), Lo.val) <= 1e-11


@pytest.mark.parametrize("case", ["random", "banded", "tridiag", "diag"])
def test_ic0_generic(G, h, case):
    if case == "random":
        D = _spd_pattern(300, 0.02, 1)
    elif case == "banded":
        D = _spd_pattern(400, 0.3, 2, band=6)
    elif case == "tridiag":
        D = 4 * np.eye(3000) - np.eye(3000, k=1) - np.eye(3000, k=-1)
    else:
        D = np.diag(np.arange(1.0, 501.0))
    A = O.csr_from_dense(D)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, bad = G.ic0(h, P, v)
    Lo, obad = O.ic0(A)
    assert bad == obad == -1
    assert _rel(_np(Lg), Lo.val) <= 1e-11


def test_ic0_breakdown_row_and_shift(G, h):
    """Seeds whose IC(0) breaks down in the oracle (lognormal sigma = 2.5):
    same first failing row, same shift, same shifted factor."""
    found = 0
    for seed in range(40):
        N = 4
        E = I.material_field(N, seed, sigma=2.5)
        A = O.fem_hex_assemble(N, E)
        Lo, obad = O.ic0(A)
        if obad < 0:
            continue
        found += 1
        rp, c, v = _upload(A)
        P = G.Pattern(h, rp, c)
        _, bad = G.ic0(h, P, v)
        assert bad == obad
        Lg, alpha, bad2 = G.ic0_auto(h, P, v)
        Lo2, oalpha, obad2 = O.ic0_auto(A)
        assert alpha == oalpha and bad2 == obad2 == -1
        assert _rel(_np(Lg), Lo2.val) <= 1e-11
        if found == 3:
            break
    assert found >= 1


# ---------------------------------------------------------------- A7 kernels
def test_spmv_matches_oracle(G, h):
    N = 8
    A = O.fem_hex_assemble(N, I.material_field(N, 4))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    x = np.random.default_rng(0).standard_normal(A.n)
    y, d = G.spmv(h, P, v, _dev(x), with_dot=True)
    yo = O.spmv(A, x)
    assert _rel(_np(y), yo) <= 1e-13
    assert abs(_np(d)[0] - x @ yo) <= 1e-12 * abs(x @ yo)


@pytest.mark.parametrize("pipeline", [5, 4, 3, 2, 1, 0])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("case", ["fem8", "fem5", "random", "tridiag"])
def test_triangular_solves_match_oracle(G, h, dtype, case, pipeline):
    """Every solve path (pair-sliced, level-sliced, warp-specialised and
    pipelined where the pattern allows, generic) against the oracle on the
    same factor."""
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, pipeline)
    if case == "fem8":
        A = O.fem_hex_assemble(8, I.material_field(8, 5))
    elif case == "fem5":
        A = O.fem_hex_assemble(5, I.material_field(5, 6))
    elif case == "random":
        A = O.csr_from_dense(_spd_pattern(300, 0.02, 1))
    else:
        A = O.csr_from_dense(4 * np.eye(3000) - np.eye(3000, k=1) - np.eye(3000, k=-1))
    Lo, _ = O.ic0(A)
    # the factor the GPU sees, exactly, in float64 for the oracle
    Lval = Lo.val.astype(np.float32).astype(np.float64) if dtype == torch.float32 else Lo.val
    Lref = O.CSR(Lo.rowptr, Lo.col, Lval)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Ld = _dev(Lval).to(dtype)
    if pipeline == 5 and case.startswith("fem"):
        assert P.pair_mode == 1 and G.solve_kernels_chosen(h, P) == "pair-sliced"
    r = np.random.default_rng(2).uniform(-1, 1, A.n)
    y = G.lsolve(h, P, Ld, _dev(r))
    z = G.ltsolve(h, P, Ld, y)
    yo = O.lsolve(Lref, r)
    zo = O.ltsolve(Lref, yo)
    if dtype == torch.float64:
        assert _rel(_np(y), yo) <= 1e-11
        assert _rel(_np(z), zo) <= 1e-11
    else:  # the FP32 preconditioner apply sums in FP32
        nrel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
        assert nrel(_np(y), yo) <= 1e-5 and nrel(_np(z), zo) <= 1e-5
    assert G.error_flags(h) == 0
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)


@pytest.mark.parametrize("pipeline", [3, 2])
@pytest.mark.parametrize("qdelta", [0, 3, 30])
def test_solve_late_window_variants(G, h, qdelta, pipeline):
    """The split of a group's dependencies into early and late ones only
    changes when the solve waits, not its result."""
    G.set_tuning(h, G.GIC_TUNE_QDELTA, qdelta)
    A = O.fem_hex_assemble(6, I.material_field(6, 4))
    Lo, _ = O.ic0(A)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    G.set_tuning(h, G.GIC_TUNE_QDELTA, 6)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, pipeline)
    r = np.random.default_rng(3).uniform(-1, 1, A.n)
    y = G.lsolve(h, P, _dev(Lo.val), _dev(r))
    z = G.ltsolve(h, P, _dev(Lo.val), y)
    yo = O.lsolve(Lo, r)
    assert _rel(_np(y), yo) <= 1e-11
    assert _rel(_np(z), O.ltsolve(Lo, yo)) <= 1e-11
    assert G.error_flags(h) == 0
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)


@pytest.mark.parametrize("pair_levels", [0, 1])
def test_pair_sliced_schedule_variants(G, h, pair_levels):
    """Pair-sliced solves with the levels paired (second level substituted)
    and one level per step: hex 6^3 against the oracle, and the schedule's
    group levels are the node levels x + 2y + 4z (7N - 3 of them)."""
    N = 6
    A = O.fem_hex_assemble(N, I.material_field(N, 12))
    Lo, _ = O.ic0(A)
    rp, c, v = _upload(A)
    G.set_tuning(h, G.GIC_TUNE_PAIR_LEVELS, pair_levels)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 5)
    P = G.Pattern(h, rp, c)
    G.set_tuning(h, G.GIC_TUNE_PAIR_LEVELS, 0)
    assert P.group_levels == 7 * N - 3 and P.nlevels == 3 * P.group_levels
    assert P.pair_mode == (1 if pair_levels == 0 else 2), P.pair_mode
    r = np.random.default_rng(4).uniform(-1, 1, A.n)
    y = G.lsolve(h, P, _dev(Lo.val), _dev(r))
    z = G.ltsolve(h, P, _dev(Lo.val), y)
    b = I.rhs(A.n, 12)
    Lg, _ = G.ic0(h, P, v)
    res = G.pcg(h, P, v, Lg, _dev(b), rtol=1e-8)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)
    yo = O.lsolve(Lo, r)
    assert _rel(_np(y), yo) <= 1e-11
    assert _rel(_np(z), O.ltsolve(Lo, yo)) <= 1e-11
    ro = O.pcg(A, b, Lo, tol=1e-8)
    assert res["status"] == 0 and _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    assert np.linalg.norm(_np(res["x"]) - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])
    assert G.error_flags(h) == 0


def test_pair_schedule_built_only_when_used(G, h):
    """With the automatic choice a small system (below the pair-sliced band)
    gets no pair schedule (reason 256: not asked for); asked for, it gets one."""
    A = O.fem_hex_assemble(4, I.material_field(4, 3))
    rp, c, v = _upload(A)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)
    P = G.Pattern(h, rp, c)
    assert P.pair_mode == -256 and G.solve_kernels_chosen(h, P) == "warp-specialised"
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 5)
    P5 = G.Pattern(h, rp, c)
    assert P5.pair_mode == 1 and G.solve_kernels_chosen(h, P5) == "pair-sliced"
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)


# ---------------------------------------------------------------- A7 PCG
@pytest.mark.parametrize("pipeline", [5, 4, 3])
@pytest.mark.parametrize("N", [2, 4, 8, 12])
def test_pcg_matches_oracle(G, h, N, pipeline):
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, pipeline)
    E = I.material_field(N, 7)
    A = O.fem_hex_assemble(N, E)
    b = I.rhs(A.n, 7)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, bad = G.ic0(h, P, v)
    res = G.pcg(h, P, v, Lg, _dev(b), rtol=1e-8)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)
    Lo, _ = O.ic0(A)
    ro = O.pcg(A, b, Lo, tol=1e-8)
    assert res["status"] == 0 and ro["status"] == 0
    assert _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    assert res["relres"] <= 1e-8
    x = _np(res["x"])
    assert np.linalg.norm(x - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])
    true_rel = np.linalg.norm(b - O.spmv(A, x)) / np.linalg.norm(b)
    assert true_rel <= 1e-7


def test_plain_cg_matches_oracle(G, h):
    N = 4
    A = O.fem_hex_assemble(N, I.material_field(N, 8))
    b = I.rhs(A.n, 8)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    res = G.pcg(h, P, v, None, _dev(b), rtol=1e-8)
    ro = O.pcg(A, b, None, tol=1e-8)
    assert _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    x = _np(res["x"])
    assert np.linalg.norm(x - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])


@pytest.mark.parametrize("pipeline", [5, 3, 2, 1, 0])
def test_pcg_f32_factor(G, h, pipeline):
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, pipeline)
    N = 8
    A = O.fem_hex_assemble(N, I.material_field(N, 9))
    b = I.rhs(A.n, 9)
    Lo, _ = O.ic0(A)
    L32 = O.CSR(Lo.rowptr, Lo.col, Lo.val.astype(np.float32).astype(np.float64))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, _ = G.ic0(h, P, v)
    res = G.pcg(h, P, v, G.to_f32(h, Lg), _dev(b), rtol=1e-8)
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, 4)
    ro = O.pcg(A, b, L32, tol=1e-8)
    assert _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    x = _np(res["x"])
    assert np.linalg.norm(x - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])


def test_pcg_edge_cases(G, h):
    N = 3
    A = O.fem_hex_assemble(N, I.material_field(N, 1))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, _ = G.ic0(h, P, v)
    # b = 0: no iteration, x = 0
    res = G.pcg(h, P, v, Lg, torch.zeros(A.n, dtype=torch.float64, device=DEV))
    assert res["iters"] == 0 and res["status"] == 0 and torch.all(res["x"] == 0)
    # x0 already the solution
    b = I.rhs(A.n, 1)
    xs = np.linalg.solve(A.to_dense(), b)
    res = G.pcg(h, P, v, Lg, _dev(b), x=_dev(xs), rtol=1e-8)
    assert res["iters"] == 0
    # iteration cap
    res = G.pcg(h, P, v, Lg, _dev(b), rtol=1e-14, maxit=3)
    assert res["status"] == G.GIC_ERR_NO_CONVERGENCE and res["iters"] == 3
    Lo, _ = O.ic0(A)
    ro = O.pcg(A, b, Lo, tol=1e-14, maxit=3)
    assert np.linalg.norm(_np(res["x"]) - ro["x"]) <= 1e-9 * np.linalg.norm(ro["x"])


def test_pcg_deterministic(G, h):
    N = 8
    A = O.fem_hex_assemble(N, I.material_field(N, 2))
    b = _dev(I.rhs(A.n, 2))
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, _ = G.ic0(h, P, v)
    r1 = G.pcg(h, P, v, Lg, b)
    r2 = G.pcg(h, P, v, Lg, b)
    assert r1["iters"] == r2["iters"] and torch.equal(r1["x"], r2["x"])


def test_full_size_40_cube(G, h):
    """The 40^3-element system (201,720 dofs, 15.5M nonzeros) the benchmark
    times: assembly, analysis, IC(0) and PCG against the oracle."""
    N = 40
    E = I.material_field(N, 0)
    b = I.rhs(3 * N * (N + 1) ** 2, 0)
    rp, c, v = G.fem_hex_assemble(h, N, _dev(E))
    A = O.fem_hex_assemble(N, E)
    assert np.array_equal(_np(rp), A.rowptr) and np.array_equal(_np(c), A.col)
    assert _rel(_np(v), A.val) <= 1e-13
    P = G.Pattern(h, rp, c)
    assert P.nlevels == 21 * N - 9 and P.ngroups == A.n // 3
    Lg, alpha, bad = G.ic0_auto(h, P, v)
    Lo, oalpha, obad = O.ic0_auto(A)
    assert alpha == oalpha and bad == obad == -1
    assert _rel(_np(Lg), Lo.val) <= 1e-10
    res = G.pcg(h, P, v, Lg, _dev(b), rtol=1e-8)
    ro = O.pcg(A, b, Lo, tol=1e-8)
    assert _iters_ok(res["iters"], ro["iters"]), (res["iters"], ro["iters"])
    x = _np(res["x"])
    assert np.linalg.norm(x - ro["x"]) <= 1e-6 * np.linalg.norm(ro["x"])


def test_bounded_wait_times_out_and_handle_survives(G, h):
    """A device wait on a flag that nothing sets runs out, is reported as
    GIC_ERR_TIMEOUT, and the handle still solves correctly afterwards."""
    assert G.selftest_wait_timeout(h, 4096) == G.GIC_ERR_TIMEOUT
    assert G.error_flags(h) == 0
    N = 3
    A = O.fem_hex_assemble(N, I.material_field(N, 1))
    b = I.rhs(A.n, 1)
    rp, c, v = _upload(A)
    P = G.Pattern(h, rp, c)
    Lg, _ = G.ic0(h, P, v)
    res = G.pcg(h, P, v, Lg, _dev(b))
    Lo, _ = O.ic0(A)
    ro = O.pcg(A, b, Lo)
    assert _iters_ok(res["iters"], ro["iters"])
