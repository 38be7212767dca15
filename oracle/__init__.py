"""CPU oracle for the GNN-corrected IC(0)-PCG path (arxiv 2412.07127).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py, never by the product package. It is
a thin numpy <-> ctypes marshalling layer over gic_oracle.c (plain sequential
FP64 C); every computation happens there. It shares no code with the CUDA
path: inputs come from the seeded generators, never from the GPU.

Parity status of each routine is listed in the header of gic_oracle.c; the
GNN architecture is parity unpinned against the paper (its Figure 1 is not in
the text) and pinned only by g = 0 => L = L_IC, finite differences and an
independent dense restatement.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = C.c_int64
_dbl = C.c_double


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_hex_element_stiffness.argtypes = [_dbl, _dbl, _f64p]
        L.or_fem_hex_sizes.argtypes = [C.c_int, C.c_int, C.POINTER(_i64), C.POINTER(_i64)]
        L.or_fem_hex_assemble.argtypes = [C.c_int, C.c_int, _dbl, _f64p, _i32p, _i32p, _f64p]
        L.or_fem_box_sizes.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(_i64), C.POINTER(_i64)]
        L.or_fem_box_assemble.argtypes = [C.c_int, C.c_int, C.c_int, _dbl, C.c_int, _dbl, _f64p, _i32p, _i32p,
                                          _f64p]
        L.or_spmv_threads.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_spmv_threads.restype = None
        L.or_threads.restype = C.c_int
        L.or_lower_nnz.argtypes = [_i64, _i32p, _i32p]
        L.or_lower_nnz.restype = _i64
        L.or_lower_pattern.argtypes = [_i64, _i32p, _i32p, C.c_void_p, _i32p, _i32p, C.c_void_p]
        L.or_levels.argtypes = [_i64, _i32p, _i32p, _i32p]
        L.or_levels.restype = C.c_int32
        L.or_ic0.argtypes = [_i64, _i32p, _i32p, _f64p, _dbl]
        L.or_ic0.restype = _i64
        L.or_ic0_auto.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, C.c_int, C.POINTER(_dbl)]
        L.or_ic0_auto.restype = _i64
        L.or_spmv.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_lsolve.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_ltsolve.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_pcg.argtypes = [_i64, _i32p, _i32p, _f64p, C.c_void_p, C.c_void_p, C.c_void_p,
                             _f64p, _f64p, _dbl, C.c_int, C.POINTER(C.c_int), C.POINTER(_dbl),
                             C.c_void_p, C.c_void_p]
        L.or_pcg.restype = C.c_int
        L.or_features.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _i32p, _f64p, C.POINTER(_dbl)]
        L.or_gnn_param_count.restype = C.c_int
        L.or_round_bf16.argtypes = [_dbl]
        L.or_round_bf16.restype = _dbl
        L.or_gnn_forward.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_int, _f64p]
        L.or_gnn_forward_parts.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_int, _f64p, _f64p,
                                           _f64p, _f64p, _f64p]
        L.or_gnn_forward_parts.restype = None
        L.or_correct.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_correct_backward.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        L.or_gnn_backward.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p, C.c_int, _f64p, _f64p]
        L.or_probe_loss.argtypes = [_i64, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, _f64p,
                                    C.c_int, C.c_void_p]
        L.or_probe_loss.restype = _dbl
        L.or_adam_step.argtypes = [_i64, _f64p, _f64p, _f64p, _f64p, C.c_int, _dbl]
        L.or_dropout.argtypes = [_i64, _i32p, _i32p, _f64p, _dbl, _i32p, _i32p, _f64p]
        L.or_dropout.restype = _i64
        L.or_factor_deviation.argtypes = [_i64, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.or_row_groups.argtypes = [_i64, _i32p, _i32p, C.c_int, _i32p]
        L.or_row_groups.restype = _i64
        L.or_dropout_grouped.argtypes = [_i64, _i32p, _i32p, _f64p, _dbl, _i64, _i32p, _i32p, _i32p, _f64p]
        L.or_dropout_grouped.restype = _i64
        L.or_lr_at.argtypes = [C.c_int, C.c_int, _dbl]
        L.or_lr_at.restype = _dbl
        _lib = L
    return _lib


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class CSR:
    """Plain CSR triple (int32 rowptr/col, float64 val)."""

    def __init__(self, rowptr, col, val):
        self.rowptr = _c32(rowptr)
        self.col = _c32(col)
        self.val = _c64(val) if val is not None else None

    @property
    def n(self):
        return len(self.rowptr) - 1

    @property
    def nnz(self):
        return int(self.rowptr[-1])

    def to_dense(self):
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            for p in range(self.rowptr[i], self.rowptr[i + 1]):
                D[i, self.col[p]] += self.val[p]
        return D


def csr_from_dense(D, lower=False):
    D = np.asarray(D, dtype=np.float64)
    n = D.shape[0]
    rowptr = [0]
    col, val = [], []
    for i in range(n):
        for j in range(n):
            if (not lower or j <= i) and (D[i, j] != 0.0 or i == j):
                col.append(j)
                val.append(D[i, j])
        rowptr.append(len(col))
    return CSR(np.array(rowptr), np.array(col), np.array(val))


# ---------------------------------------------------------------- A1
def element_stiffness(nu=0.3, h=1.0):
    Ke = np.zeros(576)
    lib().or_hex_element_stiffness(nu, h, Ke)
    return Ke.reshape(24, 24)


def fem_hex_sizes(N, clamp=True):
    n, nnz = _i64(), _i64()
    if lib().or_fem_hex_sizes(N, 1 if clamp else 0, C.byref(n), C.byref(nnz)) != 0:
        raise ValueError("bad N")
    return n.value, nnz.value


def fem_hex_assemble(N, E, nu=0.3, clamp=True):
    """A = sum_e E_e K_e on the N^3 hex mesh; E has N^3 entries."""
    E = _c64(E)
    assert E.size == N ** 3
    n, nnz = fem_hex_sizes(N, clamp)
    rowptr = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    rc = lib().or_fem_hex_assemble(N, 1 if clamp else 0, nu, E, rowptr, col, val)
    if rc != 0:
        raise RuntimeError(f"or_fem_hex_assemble failed: {rc}")
    return CSR(rowptr, col, val)


def fem_box_assemble(Nx, Ny, Nz, h, E, nu=0.3, clamp=True):
    """A = sum_e E_e K_e on a box of Nx x Ny x Nz hex elements of side h
    (element id ex + Nx (ey + Ny ez)); E has Nx Ny Nz entries. The first z
    layers of the N^3 cube (h = 1/N) give the cube's rows of the nodes they
    hold, except on the box's top node plane."""
    E = _c64(E)
    assert E.size == Nx * Ny * Nz
    n, nnz = _i64(), _i64()
    if lib().or_fem_box_sizes(Nx, Ny, Nz, 1 if clamp else 0, C.byref(n), C.byref(nnz)) != 0:
        raise ValueError("bad box")
    rowptr = np.zeros(n.value + 1, np.int32)
    col = np.zeros(nnz.value, np.int32)
    val = np.zeros(nnz.value)
    rc = lib().or_fem_box_assemble(Nx, Ny, Nz, h, 1 if clamp else 0, nu, E, rowptr, col, val)
    if rc != 0:
        raise RuntimeError(f"or_fem_box_assemble failed: {rc}")
    return CSR(rowptr, col, val)


def spmv_threads(A: CSR, x):
    """or_spmv with its rows split over the host's cores (same result)."""
    y = np.zeros(A.n)
    lib().or_spmv_threads(A.n, A.rowptr, A.col, A.val, _c64(x), y)
    return y


def threads():
    """Threads or_spmv_threads uses (OpenMP's default: the host's cores)."""
    return int(lib().or_threads())


# ---------------------------------------------------------------- A2
def lower(A: CSR, with_values=True):
    n = A.n
    nnzL = lib().or_lower_nnz(n, A.rowptr, A.col)
    Lr = np.zeros(n + 1, np.int32)
    Lc = np.zeros(nnzL, np.int32)
    Lv = np.zeros(nnzL) if with_values else None
    lib().or_lower_pattern(n, A.rowptr, A.col,
                           A.val.ctypes.data if with_values else None,
                           Lr, Lc, Lv.ctypes.data if with_values else None)
    return CSR(Lr, Lc, Lv if with_values else np.zeros(nnzL))


def levels(L: CSR):
    lev = np.zeros(L.n, np.int32)
    nlev = lib().or_levels(L.n, L.rowptr, L.col, lev)
    return lev, int(nlev)


# ---------------------------------------------------------------- A3
def ic0(A: CSR, alpha=0.0):
    """Returns (L, bad_row) with bad_row = -1 on success."""
    T = lower(A)
    Lv = T.val.copy()
    bad = lib().or_ic0(T.n, T.rowptr, T.col, Lv, alpha)
    return CSR(T.rowptr, T.col, Lv), int(bad)


def ic0_auto(A: CSR, max_tries=20):
    """IC(0) with the shift restart. Returns (L, alpha, bad_row)."""
    T = lower(A)
    Lv = np.zeros_like(T.val)
    a = _dbl()
    bad = lib().or_ic0_auto(T.n, T.rowptr, T.col, T.val, Lv, max_tries, C.byref(a))
    return CSR(T.rowptr, T.col, Lv), a.value, int(bad)


# ---------------------------------------------------------------- A7
def spmv(A: CSR, x):
    y = np.zeros(A.n)
    lib().or_spmv(A.n, A.rowptr, A.col, A.val, _c64(x), y)
    return y


def lsolve(L: CSR, r):
    y = np.zeros(L.n)
    lib().or_lsolve(L.n, L.rowptr, L.col, L.val, _c64(r), y)
    return y


def ltsolve(L: CSR, y):
    z = np.zeros(L.n)
    lib().or_ltsolve(L.n, L.rowptr, L.col, L.val, _c64(y), z)
    return z


def pcg(A: CSR, b, L: CSR = None, x0=None, tol=1e-8, maxit=10000, history=False):
    """Algorithm 1 of the supplementary material. L=None: plain CG.
    Returns dict(x, iters, relres, status[, hist, rhist])."""
    n = A.n
    b = _c64(b)
    x = np.zeros(n) if x0 is None else _c64(x0).copy()
    it = C.c_int()
    rr = _dbl()
    hist = np.zeros((maxit, n)) if history else None
    rhist = np.zeros(maxit + 1) if history else None
    st = lib().or_pcg(n, A.rowptr, A.col, A.val,
                      L.rowptr.ctypes.data if L is not None else None,
                      L.col.ctypes.data if L is not None else None,
                      L.val.ctypes.data if L is not None else None,
                      b, x, tol, maxit, C.byref(it), C.byref(rr),
                      hist.ctypes.data if history else None,
                      rhist.ctypes.data if history else None)
    out = dict(x=x, iters=it.value, relres=rr.value, status=st)
    if history:
        out["hist"] = hist[: it.value]
        out["rhist"] = rhist[: it.value + 1]
    return out


# ---------------------------------------------------------------- A4-A6
N_PARAMS = None


def gnn_param_count():
    return lib().or_gnn_param_count()


def features(A: CSR):
    """Returns (x9 (n,9), e (nnzL,), scale s)."""
    T = lower(A, with_values=False)
    x9 = np.zeros(A.n * 9)
    e = np.zeros(T.nnz)
    s = _dbl()
    lib().or_features(A.n, A.rowptr, A.col, A.val, x9, T.rowptr, e, C.byref(s))
    return x9.reshape(A.n, 9), e, s.value


def round_bf16(v):
    f = lib().or_round_bf16
    return np.array([f(float(t)) for t in np.ravel(v)]).reshape(np.shape(v))


def _bf16_bits(bf16):
    """bf16: False / True (the edge MLP's first layer) or the oracle's bit set
    (1 edge MLP, 2 node MLP, 3 both: the tensor-core inference path)."""
    return int(bf16)


def gnn_forward(T: CSR, x9, e0, theta, bf16=False):
    g = np.zeros(T.nnz)
    lib().or_gnn_forward(T.n, T.rowptr, T.col, _c64(x9).ravel(), _c64(e0), _c64(theta),
                         _bf16_bits(bf16), g)
    return g


def gnn_forward_parts(T: CSR, x9, e0, theta, bf16=False):
    """(g, x0, S0, M0, x1): the output and the intermediates tests pin:
    GraphNorm output, block 0's node sums and means, block 0's node update."""
    n = T.n
    g = np.zeros(T.nnz)
    x0, x1 = np.zeros(9 * n), np.zeros(9 * n)
    S0, M0 = np.zeros(n), np.zeros(n)
    lib().or_gnn_forward_parts(T.n, T.rowptr, T.col, _c64(x9).ravel(), _c64(e0), _c64(theta),
                               _bf16_bits(bf16), g, x0, S0, M0, x1)
    return g, x0.reshape(n, 9), S0, M0, x1.reshape(n, 9)


def correct(T: CSR, LIC_val, g):
    out = np.zeros(T.nnz)
    lib().or_correct(T.n, T.rowptr, T.col, _c64(LIC_val), _c64(g), out)
    return out


def correct_backward(T: CSR, LIC_val, g, dLout):
    dg = np.zeros(T.nnz)
    lib().or_correct_backward(T.n, T.rowptr, T.col, _c64(LIC_val), _c64(g), _c64(dLout), dg)
    return dg


def gnn_backward(T: CSR, x9, e0, theta, dg, bf16=False):
    d = np.zeros(gnn_param_count())
    lib().or_gnn_backward(T.n, T.rowptr, T.col, _c64(x9).ravel(), _c64(e0), _c64(theta),
                          _bf16_bits(bf16), _c64(dg), d)
    return d


def probe_loss(A: CSR, L: CSR, Z, grad=False):
    """Eq.(5) averaged over the m rows of Z (m, n). Returns loss or (loss, dL)."""
    Z = _c64(np.atleast_2d(Z))
    m = Z.shape[0]
    dL = np.zeros(L.nnz) if grad else None
    loss = lib().or_probe_loss(A.n, A.rowptr, A.col, A.val, L.rowptr, L.col, L.val,
                               Z.ravel(), m, dL.ctypes.data if grad else None)
    return (loss, dL) if grad else loss


def adam_step(theta, grad, m1, m2, t, lr):
    """In-place Adam on float64 arrays."""
    lib().or_adam_step(theta.size, theta, _c64(grad), m1, m2, t, lr)


def lr_at(t, warm, lr_max=0.005):
    return lib().or_lr_at(t, warm, lr_max)


# ---------------------------------------------------------------- Eq. (10), Figure 5
def dropout(L: CSR, thr):
    """Fill-in dropout of the factor: off-diagonal |L_ij| <= thr removed."""
    rp = np.zeros(L.n + 1, np.int32)
    col = np.zeros(len(L.col), np.int32)
    val = np.zeros(len(L.col))
    k = lib().or_dropout(L.n, L.rowptr, L.col, np.ascontiguousarray(L.val, np.float64), thr, rp, col, val)
    return CSR(rp, col[:k].copy(), val[:k].copy())


def factor_deviation(L: CSR, LIC_val, Lpred_val):
    out = np.zeros(6)
    lib().or_factor_deviation(L.n, L.rowptr, L.col, np.ascontiguousarray(LIC_val, np.float64),
                              np.ascontiguousarray(Lpred_val, np.float64), out)
    return out


def row_groups(A: CSR, gmax=8):
    """Start rows of the runs of identical-pattern rows (cut every gmax), n last."""
    st = np.zeros(A.n + 1, np.int32)
    ng = lib().or_row_groups(A.n, A.rowptr, A.col, gmax, st)
    return st[:ng + 1].copy()


def dropout_grouped(L: CSR, thr, starts):
    """Node-granular dropout: the external block of row group g against an
    earlier group h leaves the factor only if all its entries are <= thr."""
    rp = np.zeros(L.n + 1, np.int32)
    col = np.zeros(len(L.col), np.int32)
    val = np.zeros(len(L.col))
    st = np.ascontiguousarray(starts, np.int32)
    k = lib().or_dropout_grouped(L.n, L.rowptr, L.col, np.ascontiguousarray(L.val, np.float64), thr,
                                 len(st) - 1, st, rp, col, val)
    return CSR(rp, col[:k].copy(), val[:k].copy())
