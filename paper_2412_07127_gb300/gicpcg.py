"""ctypes binding of libgicpcg.so (the C-ABI in include/gicpcg.h).

Argument marshalling only: every function takes torch tensors (device memory
owned by torch) or host scalars, passes raw pointers and sizes through the
C-ABI, and turns a non-zero status into GicError. There is no fallback: if
the CUDA library is missing or fails to load, every call raises.
"""
import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgicpcg.so")

GIC_OK = 0
GIC_ERR_INVALID_ARG = -1
GIC_ERR_NOT_SPD = -2
GIC_ERR_NO_CONVERGENCE = -3
GIC_ERR_TIMEOUT = -4
GIC_ERR_CUDA = -5
GIC_ERR_TOO_LARGE = -6
GIC_ERR_UNSUPPORTED = -7
GIC_ERR_BREAKDOWN = -8
GIC_ERR_WORKSPACE = -9

GIC_F64, GIC_F32, GIC_IDENTITY = 0, 1, 2
GIC_WS_SOLVE, GIC_WS_PCG = 0, 1
PROF_CLASSES = ("lsolve", "ltsolve", "spmv", "vector")

_vp = C.c_void_p
_i64 = C.c_int64
_i32 = C.c_int32
_int = C.c_int
_dbl = C.c_double
_sz = C.c_size_t

# name -> (restype, argtypes)
_SIGS = {
    "gic_create": (_int, [C.POINTER(_vp), _int, _vp]),
    "gic_set_stream": (_int, [_vp, _vp]),
    "gic_destroy": (_int, [_vp]),
    "gic_status_string": (C.c_char_p, [_int]),
    "gic_last_cuda_error": (C.c_char_p, []),
    "gic_fem_hex_sizes": (_int, [_int, C.POINTER(_i64), C.POINTER(_i64)]),
    "gic_fem_hex_assemble": (_int, [_vp, _int, _dbl, _int, _vp, _vp, _vp, _vp]),
    "gic_analyze": (_int, [_vp, _i64, _i64, _vp, _vp, C.POINTER(_vp)]),
    "gic_pattern_destroy": (_int, [_vp]),
    "gic_pattern_info": (_int, [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64),
                                C.POINTER(_i32), C.POINTER(_i32)]),
    "gic_pattern_export": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "gic_pattern_schedule": (_int, [_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i64)]),
    "gic_pattern_solve_kernels": (_int, [_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32)]),
    "gic_pattern_spmv_layout": (_int, [_vp, C.POINTER(_i32), C.POINTER(_i64)]),
    "gic_pattern_pair_schedule": (_int, [_vp, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32)]),
    "gic_solve_kernels_chosen": (_int, [_vp, _vp, _int, C.POINTER(_i32)]),
    "gic_ic0": (_int, [_vp, _vp, _vp, _vp, _dbl, C.POINTER(_i64)]),
    "gic_ic0_auto": (_int, [_vp, _vp, _vp, _vp, _int, C.POINTER(_dbl), C.POINTER(_i64)]),
    "gic_convert_f64_f32": (_int, [_vp, _i64, _vp, _vp]),
    "gic_spmv": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "gic_lsolve": (_int, [_vp, _vp, _vp, _int, _vp, _vp, _vp, _sz]),
    "gic_ltsolve": (_int, [_vp, _vp, _vp, _int, _vp, _vp, _vp, _sz]),
    "gic_pcg": (_int, [_vp, _vp, _vp, _vp, _int, _vp, _vp, _dbl, _int, C.POINTER(_i32),
                       C.POINTER(_dbl), _vp, _sz]),
    "gic_workspace_size_split": (_int, [_vp, _vp, _vp, _int, C.POINTER(_sz)]),
    "gic_pcg_split": (_int, [_vp, _vp, _vp, _vp, _vp, _int, _vp, _vp, _dbl, _int, C.POINTER(_i32),
                             C.POINTER(_dbl), _vp, _sz]),
    "gic_dropout": (_int, [_vp, _vp, _vp, _dbl, _vp, _vp, _vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "gic_dropout_grouped": (_int, [_vp, _vp, _vp, _dbl, _vp, _vp, _vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "gic_factor_deviation": (_int, [_vp, _vp, _vp, _vp, C.POINTER(_dbl)]),
    "gic_identity_factor": (_int, [_vp, _vp, _int, _vp, _vp, _vp]),
    "gic_workspace_size": (_int, [_vp, _vp, _int, _int, C.POINTER(_sz)]),
    "gic_profile_enable": (_int, [_vp, _int]),
    "gic_profile_read": (_int, [_vp, C.POINTER(_dbl), C.POINTER(_i64)]),
    "gic_solve_error_flags": (_int, [_vp, C.POINTER(C.c_uint)]),
    "gic_launch_count": (_int, [_vp, C.POINTER(_i64)]),
    "gic_set_tuning": (_int, [_vp, _int, _int]),
    "gic_selftest_wait_timeout": (_int, [_vp, _i64]),
    "gic_spmv_dot_noalloc": (_int, [_i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gic_solve_host": (_int, [_vp, _i64, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _int, _dbl, _int,
                              C.POINTER(_i32), C.POINTER(_dbl), C.POINTER(_dbl), C.POINTER(_int),
                              _vp, _sz]),
    "gic_solve_host_workspace_size": (_int, [_vp, _i64, _i64, _int, _int, C.POINTER(_sz)]),
    "gic_gnn_param_count": (_int, []),
    "gic_features": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _vp, _vp, _vp]),
    "gic_gnn_workspace_size": (_int, [_vp, _vp, _int, _int, C.POINTER(_sz)]),
    "gic_gnn_forward": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _vp, _vp, _sz]),
    "gic_gnn_forward_train": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _vp, _vp, _sz]),
    "gic_gnn_backward": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _vp, _vp, _vp, _sz]),
    "gic_gnn_correct": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _vp, C.POINTER(_int)]),
    "gic_scale_factor": (_int, [_vp, _vp, _int, _vp, _vp, _vp]),
    "gic_gnn_correct_scaled": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "gic_gnn_correct_backward": (_int, [_vp, _vp, _vp, _vp, _vp]),
    "gic_probe_workspace_size": (_int, [_vp, _vp, _int, _int, C.POINTER(_sz)]),
    "gic_probe_loss": (_int, [_vp, _vp, _int, _vp, _vp, _vp, _int, _vp, _vp, _vp, _sz]),
    "gic_adam_step": (_int, [_vp, _i64, _vp, _vp, _vp, _vp, _int, _dbl]),
}

_lib = None


class GicError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        text = lib().gic_status_string(status).decode()
        extra = ""
        if status == GIC_ERR_CUDA:
            extra = ": " + lib().gic_last_cuda_error().decode()
        super().__init__(f"{fn} failed with status {status} ({text}){extra}")


def lib():
    """Load libgicpcg.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != GIC_OK:
        raise GicError(name, st)
    return st


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return _vp(t.data_ptr())


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


class Handle:
    """A library handle bound to a device and a torch stream."""

    def __init__(self, device=0, stream=None):
        self.device = device
        h = _vp()
        with torch.cuda.device(device):
            _call("gic_create", C.byref(h), device, _stream_ptr(stream))
        self.h = h

    def set_stream(self, stream):
        _call("gic_set_stream", self.h, _stream_ptr(stream))

    def close(self):
        if getattr(self, "h", None):
            lib().gic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Pattern:
    """Analysis of a symmetric CSR pattern (library-owned device arrays).
    Keeps references to rowptr/col, which the library borrows."""

    def __init__(self, h: Handle, rowptr, col):
        assert rowptr.dtype == torch.int32 and col.dtype == torch.int32
        self.rowptr, self.col = rowptr, col
        n = rowptr.numel() - 1
        p = _vp()
        _call("gic_analyze", h.h, n, col.numel(), _ptr(rowptr), _ptr(col), C.byref(p))
        self.p = p
        n_, nA, nL, nl, ng = _i64(), _i64(), _i64(), _i32(), _i32()
        _call("gic_pattern_info", p, C.byref(n_), C.byref(nA), C.byref(nL), C.byref(nl), C.byref(ng))
        self.n, self.nnzA, self.nnzL = n_.value, nA.value, nL.value
        self.nlevels, self.ngroups = nl.value, ng.value
        nc, ch, sn = _i32(), _i32(), _i64()
        _call("gic_pattern_schedule", p, C.byref(nc), C.byref(ch), C.byref(sn))
        self.nchunks, self.chunked, self.sell_nnz = nc.value, ch.value, sn.value
        q, b, mr = _i32(), _i32(), _i32()
        _call("gic_pattern_solve_kernels", p, C.byref(q), C.byref(b), C.byref(mr))
        self.warp_specialised, self.level_sliced, self.slices = q.value, b.value, mr.value
        nbk, ent = _i32(), _i64()
        _call("gic_pattern_spmv_layout", p, C.byref(nbk), C.byref(ent))
        self.node_blocks, self.spmv_entries = nbk.value, ent.value
        pm, ps, gl = _i32(), _i32(), _i32()
        _call("gic_pattern_pair_schedule", p, C.byref(pm), C.byref(ps), C.byref(gl))
        self.pair_mode, self.pair_slices, self.group_levels = pm.value, ps.value, gl.value

    def export(self, h: Handle):
        dev = self.rowptr.device
        Lr = torch.empty(self.n + 1, dtype=torch.int32, device=dev)
        Lc = torch.empty(self.nnzL, dtype=torch.int32, device=dev)
        lev = torch.empty(self.n, dtype=torch.int32, device=dev)
        grp = torch.empty(self.ngroups + 1, dtype=torch.int32, device=dev)
        _call("gic_pattern_export", h.h, self.p, _ptr(Lr), _ptr(Lc), _ptr(lev), _ptr(grp))
        return Lr, Lc, lev, grp

    def close(self):
        if getattr(self, "p", None):
            lib().gic_pattern_destroy(self.p)
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fem_hex_sizes(N):
    n, nnz = _i64(), _i64()
    _call("gic_fem_hex_sizes", N, C.byref(n), C.byref(nnz))
    return n.value, nnz.value


def fem_hex_assemble(h: Handle, N, E, nu=0.3, nb=1):
    """E: float64 device tensor of nb*N^3 element moduli. Returns rowptr, col, val."""
    n, nnz = fem_hex_sizes(N)
    dev = E.device
    rowptr = torch.empty(nb * n + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nb * nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nb * nnz, dtype=torch.float64, device=dev)
    _call("gic_fem_hex_assemble", h.h, N, nu, nb, _ptr(E), _ptr(rowptr), _ptr(col), _ptr(val))
    return rowptr, col, val


def ic0(h: Handle, P: Pattern, valA, alpha=0.0, out=None):
    """Returns (valL, bad_row); bad_row = -1 on success. Raises on other errors."""
    valL = out if out is not None else torch.empty(P.nnzL, dtype=torch.float64, device=valA.device)
    bad = _i64()
    st = lib().gic_ic0(h.h, P.p, _ptr(valA), _ptr(valL), alpha, C.byref(bad))
    if st not in (GIC_OK, GIC_ERR_NOT_SPD):
        raise GicError("gic_ic0", st)
    return valL, bad.value


def ic0_auto(h: Handle, P: Pattern, valA, max_tries=20, out=None):
    """Returns (valL, alpha, bad_row)."""
    valL = out if out is not None else torch.empty(P.nnzL, dtype=torch.float64, device=valA.device)
    a, bad = _dbl(), _i64()
    st = lib().gic_ic0_auto(h.h, P.p, _ptr(valA), _ptr(valL), max_tries, C.byref(a), C.byref(bad))
    if st not in (GIC_OK, GIC_ERR_NOT_SPD):
        raise GicError("gic_ic0_auto", st)
    return valL, a.value, (bad.value if st != GIC_OK else -1)


def to_f32(h: Handle, src):
    dst = torch.empty(src.numel(), dtype=torch.float32, device=src.device)
    _call("gic_convert_f64_f32", h.h, src.numel(), _ptr(src), _ptr(dst))
    return dst


def spmv(h: Handle, P: Pattern, valA, x, y=None, with_dot=False):
    y = y if y is not None else torch.empty_like(x)
    d = torch.empty(1, dtype=torch.float64, device=x.device) if with_dot else None
    _call("gic_spmv", h.h, P.p, _ptr(valA), _ptr(x), _ptr(y), _ptr(d))
    return (y, d) if with_dot else y


def workspace(h: Handle, P: Pattern, op, l_dtype):
    b = _sz()
    _call("gic_workspace_size", h.h, P.p, op, l_dtype, C.byref(b))
    return torch.empty(max(b.value, 1), dtype=torch.uint8, device=P.rowptr.device)


def _ldtype(valL):
    if valL is None:
        return GIC_IDENTITY
    return {torch.float64: GIC_F64, torch.float32: GIC_F32}[valL.dtype]


def lsolve(h: Handle, P: Pattern, valL, r, y=None, ws=None):
    dt = _ldtype(valL)
    ws = ws if ws is not None else workspace(h, P, GIC_WS_SOLVE, dt)
    y = y if y is not None else torch.empty_like(r)
    _call("gic_lsolve", h.h, P.p, _ptr(valL), dt, _ptr(r), _ptr(y), _ptr(ws), ws.numel())
    return y


def ltsolve(h: Handle, P: Pattern, valL, y, z=None, ws=None):
    dt = _ldtype(valL)
    ws = ws if ws is not None else workspace(h, P, GIC_WS_SOLVE, dt)
    z = z if z is not None else torch.empty_like(y)
    _call("gic_ltsolve", h.h, P.p, _ptr(valL), dt, _ptr(y), _ptr(z), _ptr(ws), ws.numel())
    return z


def pcg(h: Handle, P: Pattern, valA, valL, b, x=None, rtol=1e-8, maxit=10000, ws=None, check=True):
    """Supplementary Algorithm 1. valL None = plain CG. Returns dict."""
    dt = _ldtype(valL)
    ws = ws if ws is not None else workspace(h, P, GIC_WS_PCG, dt)
    x = x if x is not None else torch.zeros_like(b)
    it, rr = _i32(), _dbl()
    st = lib().gic_pcg(h.h, P.p, _ptr(valA), _ptr(valL), dt, _ptr(b), _ptr(x), rtol, maxit,
                       C.byref(it), C.byref(rr), _ptr(ws), ws.numel())
    if check and st not in (GIC_OK, GIC_ERR_NO_CONVERGENCE):
        raise GicError("gic_pcg", st)
    return dict(x=x, iters=it.value, relres=rr.value, status=st)


def pcg_split(h: Handle, PA: Pattern, valA, PL: Pattern, valL, b, x=None, rtol=1e-8, maxit=10000, check=True):
    """PCG with the SpMV on PA and the solves on PL's lower triangle."""
    dt = _ldtype(valL)
    nb = _sz()
    _call("gic_workspace_size_split", h.h, PA.p, PL.p, dt, C.byref(nb))
    ws = torch.empty(max(nb.value, 1), dtype=torch.uint8, device=b.device)
    x = x if x is not None else torch.zeros_like(b)
    it, rr = _i32(), _dbl()
    st = lib().gic_pcg_split(h.h, PA.p, _ptr(valA), PL.p, _ptr(valL), dt, _ptr(b), _ptr(x), rtol, maxit,
                             C.byref(it), C.byref(rr), _ptr(ws), ws.numel())
    if check and st not in (GIC_OK, GIC_ERR_NO_CONVERGENCE):
        raise GicError("gic_pcg_split", st)
    return dict(x=x, iters=it.value, relres=rr.value, status=st)


def dropout(h: Handle, P: Pattern, valL, threshold, grouped=False):
    """Fill-in dropout (Eq. (10)): returns (Srowptr, Scol, Lval) -- the
    symmetric pattern of the kept factor and its values in tril(S) order.
    grouped: the node-granular variant (gic_dropout_grouped)."""
    dev = valL.device
    Srp = torch.empty(P.n + 1, dtype=torch.int32, device=dev)
    Sc = torch.empty(P.nnzA, dtype=torch.int32, device=dev)
    Lv = torch.empty(P.nnzL, dtype=torch.float64, device=dev)
    ns, nl = _i64(), _i64()
    _call("gic_dropout_grouped" if grouped else "gic_dropout", h.h, P.p, _ptr(valL), float(threshold), _ptr(Srp),
          _ptr(Sc), _ptr(Lv), C.byref(ns), C.byref(nl))
    return Srp, Sc[:ns.value].clone(), Lv[:nl.value].clone()


def factor_deviation(h: Handle, P: Pattern, LIC, Lpred):
    """(mean diag, max diag, mean off-diag, max off-diag, n diag, n off-diag)
    of |Lpred - LIC| / |LIC|."""
    out = (_dbl * 6)()
    _call("gic_factor_deviation", h.h, P.p, _ptr(LIC), _ptr(Lpred), out)
    return tuple(out)


def identity_factor(h: Handle, P: Pattern, scale=None, ngraphs=1, want_L=True, want_hat=False):
    dev = P.rowptr.device
    L = torch.empty(P.nnzL, dtype=torch.float64, device=dev) if want_L else None
    Lh = torch.empty(P.nnzL, dtype=torch.float32, device=dev) if want_hat else None
    _call("gic_identity_factor", h.h, P.p, ngraphs, _ptr(scale), _ptr(L), _ptr(Lh))
    return L, Lh


def profile_enable(h: Handle, on=True):
    _call("gic_profile_enable", h.h, 1 if on else 0)


def profile_read(h: Handle):
    ms = (_dbl * len(PROF_CLASSES))()
    la = (_i64 * len(PROF_CLASSES))()
    _call("gic_profile_read", h.h, ms, la)
    return {k: dict(ms=ms[i], launches=la[i]) for i, k in enumerate(PROF_CLASSES)}


def error_flags(h: Handle):
    f = C.c_uint()
    _call("gic_solve_error_flags", h.h, C.byref(f))
    return f.value


GIC_TUNE_SOLVE_WARPS_PER_SM, GIC_TUNE_POLL, GIC_TUNE_PIPELINE, GIC_TUNE_QDELTA, GIC_TUNE_GNN_BF16 = 1, 2, 3, 4, 5
GIC_TUNE_TRAIN_BF16 = 6
GIC_TUNE_PAIR_LEVELS = 7
POLL_ONE_LANE = 1 << 16


def set_tuning(h: Handle, key, value):
    _call("gic_set_tuning", h.h, key, value)


def spmv_dot_noalloc(rowptr, col, val, x, y, xdoty, stream=None):
    """y = A x and xdoty[0] = x^T y with no handle, workspace or allocation
    (y and xdoty are caller-provided device tensors)."""
    _call("gic_spmv_dot_noalloc", rowptr.numel() - 1, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(x), _ptr(y),
          _ptr(xdoty), _stream_ptr(stream))


def selftest_wait_timeout(h: Handle, polls=4096):
    """Status of a deliberately unsatisfiable bounded wait (GIC_ERR_TIMEOUT expected)."""
    return lib().gic_selftest_wait_timeout(h.h, polls)


SOLVE_KERNELS = {5: "pair-sliced", 3: "level-sliced", 2: "warp-specialised", 1: "staged one-warp", 0: "generic"}


def solve_kernels_chosen(h: Handle, P: Pattern, l_dtype=GIC_F64):
    """Name of the triangular-solve kernels the PCG will run on P."""
    k = _i32()
    _call("gic_solve_kernels_chosen", h.h, P.p, l_dtype, C.byref(k))
    return SOLVE_KERNELS[k.value]


def launch_count(h: Handle):
    c = _i64()
    _call("gic_launch_count", h.h, C.byref(c))
    return c.value


def solve_host(h: Handle, rowptr, col, val, b, theta=None, l_dtype=GIC_F64, rtol=1e-8,
               maxit=10000, ws=None, x=None):
    """End-to-end solve from host (numpy or CPU torch) buffers; x returned on the host.
    theta: None (plain IC(0)) or float32 host array of GNN parameters."""
    import numpy as np
    n, nnz = len(rowptr) - 1, len(col)
    if ws is None:
        ws = solve_host_workspace(h, n, nnz, theta is not None, l_dtype)
    x = x if x is not None else np.zeros(n)
    it, rr, a, used = _i32(), _dbl(), _dbl(), _int()

    def hp(arr):
        return None if arr is None else _vp(arr.ctypes.data if hasattr(arr, "ctypes") else arr.data_ptr())
    st = lib().gic_solve_host(h.h, n, nnz, hp(rowptr), hp(col), hp(val), hp(b), hp(x), hp(theta),
                              l_dtype, rtol, maxit, C.byref(it), C.byref(rr), C.byref(a),
                              C.byref(used), _ptr(ws), ws.numel())
    if st not in (GIC_OK, GIC_ERR_NO_CONVERGENCE):
        raise GicError("gic_solve_host", st)
    return dict(x=x, iters=it.value, relres=rr.value, alpha=a.value, used_gnn=used.value, status=st)


def solve_host_workspace(h: Handle, n, nnz, with_gnn, l_dtype=GIC_F64, device=0):
    b = _sz()
    _call("gic_solve_host_workspace_size", h.h, n, nnz, 1 if with_gnn else 0, l_dtype, C.byref(b))
    return torch.empty(b.value, dtype=torch.uint8, device=torch.device("cuda", device))


# ------------------------------------------------------------------ GNN
def gnn_param_count():
    return lib().gic_gnn_param_count()


def features(h: Handle, P: Pattern, valA, ngraphs=1, with_ahat=False):
    """Returns (x9 (n,9) f32, e0 (nnzL) f32, scale (ngraphs) f64 device, Ahat or None)."""
    dev = valA.device
    x9 = torch.empty(P.n, 9, dtype=torch.float32, device=dev)
    e0 = torch.empty(P.nnzL, dtype=torch.float32, device=dev)
    Ahat = torch.empty(P.nnzA, dtype=torch.float32, device=dev) if with_ahat else None
    scale = torch.empty(ngraphs, dtype=torch.float64, device=dev)
    _call("gic_features", h.h, P.p, ngraphs, _ptr(valA), _ptr(x9), _ptr(e0), _ptr(Ahat),
          _ptr(scale), None)
    return x9, e0, scale, Ahat


def gnn_workspace(h: Handle, P: Pattern, ngraphs=1, training=False):
    b = _sz()
    _call("gic_gnn_workspace_size", h.h, P.p, ngraphs, 1 if training else 0, C.byref(b))
    return torch.empty(b.value, dtype=torch.uint8, device=P.rowptr.device)


def gnn_forward(h: Handle, P: Pattern, theta, x9, e0, ngraphs=1, ws=None, g=None):
    ws = ws if ws is not None else gnn_workspace(h, P, ngraphs, False)
    g = g if g is not None else torch.empty(P.nnzL, dtype=torch.float32, device=x9.device)
    _call("gic_gnn_forward", h.h, P.p, ngraphs, _ptr(theta), _ptr(x9), _ptr(e0), _ptr(g),
          _ptr(ws), ws.numel())
    return g


def gnn_forward_train(h: Handle, P: Pattern, theta, x9, e0, ws, ngraphs=1, g=None):
    g = g if g is not None else torch.empty(P.nnzL, dtype=torch.float32, device=x9.device)
    _call("gic_gnn_forward_train", h.h, P.p, ngraphs, _ptr(theta), _ptr(x9), _ptr(e0), _ptr(g),
          _ptr(ws), ws.numel())
    return g


def gnn_backward(h: Handle, P: Pattern, theta, x9, e0, dg, ws, ngraphs=1, dtheta=None):
    dtheta = dtheta if dtheta is not None else torch.empty_like(theta)
    _call("gic_gnn_backward", h.h, P.p, ngraphs, _ptr(theta), _ptr(x9), _ptr(e0), _ptr(dg),
          _ptr(dtheta), _ptr(ws), ws.numel())
    return dtheta


def gnn_correct(h: Handle, P: Pattern, LIC, g, scale, ngraphs=1, out=None):
    out = out if out is not None else torch.empty_like(LIC)
    ok = _int()
    _call("gic_gnn_correct", h.h, P.p, ngraphs, _ptr(LIC), _ptr(g), _ptr(scale), _ptr(out),
          C.byref(ok))
    return out, bool(ok.value)


def scale_factor(h: Handle, P: Pattern, LIC, scale, ngraphs=1):
    out = torch.empty(P.nnzL, dtype=torch.float32, device=LIC.device)
    _call("gic_scale_factor", h.h, P.p, ngraphs, _ptr(LIC), _ptr(scale), _ptr(out))
    return out


def gnn_correct_scaled(h: Handle, P: Pattern, LIChat, g, out=None):
    out = out if out is not None else torch.empty_like(LIChat)
    _call("gic_gnn_correct_scaled", h.h, P.p, _ptr(LIChat), _ptr(g), _ptr(out))
    return out


def gnn_correct_backward(h: Handle, P: Pattern, Lhat, dLhat, out=None):
    out = out if out is not None else torch.empty_like(Lhat)
    _call("gic_gnn_correct_backward", h.h, P.p, _ptr(Lhat), _ptr(dLhat), _ptr(out))
    return out


def probe_workspace(h: Handle, P: Pattern, ngraphs, m):
    b = _sz()
    _call("gic_probe_workspace_size", h.h, P.p, ngraphs, m, C.byref(b))
    return torch.empty(b.value, dtype=torch.uint8, device=P.rowptr.device)


def probe_loss(h: Handle, P: Pattern, Ahat, Lhat, Z, ngraphs=1, grad=False, ws=None):
    """Returns (loss (ngraphs+1) f32 device, dLhat or None)."""
    m = Z.shape[0]
    ws = ws if ws is not None else probe_workspace(h, P, ngraphs, m)
    loss = torch.empty(ngraphs + 1, dtype=torch.float32, device=Z.device)
    dL = torch.empty(P.nnzL, dtype=torch.float32, device=Z.device) if grad else None
    _call("gic_probe_loss", h.h, P.p, ngraphs, _ptr(Ahat), _ptr(Lhat), _ptr(Z), m, _ptr(loss),
          _ptr(dL), _ptr(ws), ws.numel())
    return loss, dL


def adam_step(h: Handle, theta, grad, m1, m2, t, lr):
    _call("gic_adam_step", h.h, theta.numel(), _ptr(theta), _ptr(grad), _ptr(m1), _ptr(m2), t, lr)
