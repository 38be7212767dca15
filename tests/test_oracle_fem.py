"""Pins of the oracle's FE assembly and pattern analysis (A1, A2) to closed
forms of linear elasticity and of the structured hex mesh, not to itself."""
import numpy as np
import pytest

import oracle as O
from paper_2412_07127_gb300 import inputs as I


def _sigma(eps, nu):
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1 / (2 * (1 + nu))
    return lam * np.trace(eps) * np.eye(3) + 2 * mu * eps


def _node_xyz(a, h):
    return np.array([(a & 1), (a >> 1) & 1, (a >> 2) & 1], float) * h


def test_element_symmetric_and_rigid_modes():
    Ke = O.element_stiffness(0.3, 0.5)
    assert np.allclose(Ke, Ke.T, rtol=0, atol=1e-14 * np.abs(Ke).max())
    w = np.linalg.eigvalsh(Ke)
    assert np.sum(np.abs(w) < 1e-12 * w.max()) == 6
    assert w[6] > 1e-3 * w.max()
    # translations and infinitesimal rotations are null vectors
    X = np.array([_node_xyz(a, 0.5) for a in range(8)])
    for t in np.eye(3):
        u = np.tile(t, 8)
        assert np.abs(Ke @ u).max() < 1e-13 * np.abs(Ke).max()
    for om in np.eye(3):
        u = np.cross(om, X).ravel()
        assert np.abs(Ke @ u).max() < 1e-13 * np.abs(Ke).max()


@pytest.mark.parametrize("nu,h", [(0.3, 1.0), (0.3, 0.125), (0.2, 0.5)])
def test_element_uniform_strain_patch(nu, h):
    """u = eps X gives nodal forces f_a = sigma n_a h^2/4 with
    sigma = lam tr(eps) I + 2 mu eps and n_a = (2ax-1, 2ay-1, 2az-1):
    the exact integral of sigma grad N_a over the cube."""
    rng = np.random.default_rng(5)
    e = rng.standard_normal((3, 3))
    eps = (e + e.T) / 2
    Ke = O.element_stiffness(nu, h)
    X = np.array([_node_xyz(a, h) for a in range(8)])
    u = (X @ eps.T).ravel()
    f = (Ke @ u).reshape(8, 3)
    sig = _sigma(eps, nu)
    for a in range(8):
        na = np.array([2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1], float)
        assert np.allclose(f[a], sig @ na * h * h / 4, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8])
def test_sizes_closed_form(N):
    n, nnz = O.fem_hex_sizes(N)
    n_cf, nnz_cf, _, _ = I.fem_sizes(N)
    assert (n, nnz) == (n_cf, nnz_cf)


def test_assembly_structure():
    N = 4
    A = O.fem_hex_assemble(N, I.material_field(N, 3))
    D = A.to_dense()
    assert np.abs(D - D.T).max() <= 1e-15 * np.abs(D).max()
    assert np.diff(A.rowptr).max() == 81
    for i in range(A.n):
        c = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)
    assert np.linalg.eigvalsh(D).min() > 0


def test_assembly_linear_in_E():
    N = 3
    E = I.material_field(N, 1)
    A1 = O.fem_hex_assemble(N, E)
    A2 = O.fem_hex_assemble(N, 2.5 * E)
    assert np.allclose(A2.val, 2.5 * A1.val, rtol=1e-14)


def test_single_element_lands_on_its_dofs():
    """Only element (1,0,1) of a 2^3 mesh switched on: its free-node block is
    K_e at the dofs 3*(x + 3*(y + 3*(z-1))) + c."""
    N = 2
    E = np.zeros(8)
    ex, ey, ez = 1, 0, 1
    E[ex + N * (ey + N * ez)] = 1.0
    A = O.fem_hex_assemble(N, E)
    D = A.to_dense()
    Ke = O.element_stiffness(0.3, 0.5)
    dofs = []
    for a in range(8):
        x, y, z = ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)
        node = x + (N + 1) * (y + (N + 1) * (z - 1))
        dofs += [3 * node + c for c in range(3)]
    assert np.allclose(D[np.ix_(dofs, dofs)], Ke, rtol=0, atol=1e-15)
    mask = np.ones_like(D, bool)
    mask[np.ix_(dofs, dofs)] = False
    assert np.all(D[mask] == 0)


def test_unclamped_rigid_modes_and_patch():
    """Free-floating body: exactly 6 zero eigenvalues; with uniform E a linear
    displacement field leaves zero force on interior nodes."""
    N = 2
    A = O.fem_hex_assemble(N, np.ones(N ** 3), clamp=False)
    D = A.to_dense()
    w = np.linalg.eigvalsh(D)
    assert np.sum(np.abs(w) < 1e-10 * w.max()) == 6
    assert w[6] > 1e-3 * w.max()
    N = 3
    A = O.fem_hex_assemble(N, np.ones(N ** 3), clamp=False)
    h = 1.0 / N
    rng = np.random.default_rng(2)
    e = rng.standard_normal((3, 3))
    eps = (e + e.T) / 2
    u = np.zeros(A.n)
    for z in range(N + 1):
        for y in range(N + 1):
            for x in range(N + 1):
                node = x + (N + 1) * (y + (N + 1) * z)
                u[3 * node:3 * node + 3] = eps @ (np.array([x, y, z]) * h)
    f = O.spmv(A, u)
    for z in range(1, N):
        for y in range(1, N):
            for x in range(1, N):
                node = x + (N + 1) * (y + (N + 1) * z)
                assert np.abs(f[3 * node:3 * node + 3]).max() < 1e-12


@pytest.mark.parametrize("N", [2, 3, 5])
def test_levels_closed_form(N):
    """Node (x,y,z) sits on level x + 2y + 4(z-1); dof c of it on
    3*(that) + c; there are 21N - 9 levels."""
    A = O.fem_hex_assemble(N, I.material_field(N, 0))
    T = O.lower(A)
    lev, nl = O.levels(T)
    assert nl == 21 * N - 9
    exp = np.zeros(A.n, np.int32)
    for z in range(1, N + 1):
        for y in range(N + 1):
            for x in range(N + 1):
                node = x + (N + 1) * (y + (N + 1) * (z - 1))
                for c in range(3):
                    exp[3 * node + c] = 3 * (x + 2 * y + 4 * (z - 1)) + c
    assert np.array_equal(lev, exp)


def test_lower_pattern_matches_dense_tril():
    N = 2
    A = O.fem_hex_assemble(N, I.material_field(N, 4))
    T = O.lower(A)
    D = A.to_dense()
    assert T.nnz == (A.nnz + A.n) // 2
    assert np.array_equal(T.to_dense(), np.tril(D))


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 3, 4), (5, 2, 1), (4, 4, 2)])
def test_box_sizes_closed_form(dims):
    """Per direction, summing a node's 1-D neighbour count over the nodes of
    a line of k elements gives 3k + 1 (free) or 3k - 2 (z, clamped at 0), so
    nnz = 9 (3Nx+1)(3Ny+1)(3Nz-2) and n = 3 (Nx+1)(Ny+1)Nz."""
    Nx, Ny, Nz = dims
    A = O.fem_box_assemble(Nx, Ny, Nz, 0.5, np.ones(Nx * Ny * Nz))
    assert A.n == 3 * (Nx + 1) * (Ny + 1) * Nz
    assert A.nnz == 9 * (3 * Nx + 1) * (3 * Ny + 1) * (3 * Nz - 2)
    D = A.to_dense()
    assert np.allclose(D, D.T, rtol=0, atol=1e-14 * np.abs(D).max())


def test_box_of_the_cube_is_the_cube():
    N = 6
    E = I.material_field(N, 3)
    A = O.fem_hex_assemble(N, E)
    B = O.fem_box_assemble(N, N, N, 1.0 / N, E)
    assert np.array_equal(A.rowptr, B.rowptr) and np.array_equal(A.col, B.col)
    assert np.array_equal(A.val, B.val)


@pytest.mark.parametrize("m", [1, 2, 4])
def test_slab_rows_equal_the_cube_rows(m):
    """The elements of the cube's first m + 1 layers hold every element that
    touches a node of the first m free planes, so the slab's rows of those
    nodes are the cube's rows, columns and values alike (node numbering is
    the same up to plane m + 1)."""
    N = 7
    E = I.material_field(N, 4)
    A = O.fem_hex_assemble(N, E)
    S = O.fem_box_assemble(N, N, m + 1, 1.0 / N, E[: N * N * (m + 1)])
    k = 3 * (N + 1) ** 2 * m
    assert np.array_equal(A.rowptr[: k + 1], S.rowptr[: k + 1])
    e = A.rowptr[k]
    assert np.array_equal(A.col[:e], S.col[:e]) and np.array_equal(A.val[:e], S.val[:e])
