"""The no-allocation SpMV entry point, for callers that cannot allocate device
memory, gives the same y and x^T y as gic_spmv on two calls in a row (its
scratch is shared across calls and must not leak state from one to the next),
works at exactly its stated row limit and rejects one row more. Collected last
on purpose: it runs alone or after every other test."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_07127_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MAX_ROWS = 8 * (1 << 20)  # the row limit the C-ABI header states


def test_spmv_dot_noalloc_matches_gic_spmv_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, gicpcg as G
    build.build()
    dev = torch.device("cuda:0")
    h = G.Handle(0)
    for N, seed in ((8, 1), (12, 2)):
        A = O.fem_hex_assemble(N, I.material_field(N, seed))
        rp = torch.from_numpy(A.rowptr).to(dev)
        c = torch.from_numpy(A.col).to(dev)
        v = torch.from_numpy(A.val).to(dev)
        P = G.Pattern(h, rp, c)
        for call in range(2):
            x = torch.from_numpy(np.random.default_rng(10 * N + call).standard_normal(A.n)).to(dev)
            y_ref, d_ref = G.spmv(h, P, v, x, with_dot=True)
            y = torch.full_like(x, float("nan"))
            d = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
            G.spmv_dot_noalloc(rp, c, v, x, y, d)
            torch.cuda.synchronize()
            assert torch.equal(y, y_ref)  # same per-row arithmetic
            # only the grouping of the dot's partial sums differs
            assert abs(float(d[0]) - float(d_ref[0])) <= 1e-12 * abs(float(d_ref[0]))


def test_spmv_dot_noalloc_at_the_row_limit():
    """A tridiagonal matrix of exactly the stated maximum row count, on two
    calls in a row, against the product and dot formed on the host in FP64;
    one row more is rejected before any launch."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, gicpcg as G
    build.build()
    dev = torch.device("cuda:0")
    n = MAX_ROWS
    rng = np.random.default_rng(7)
    d_main = 4.0 + rng.random(n)
    d_off = -rng.random(n - 1)
    cnt = np.full(n, 3, dtype=np.int64)
    cnt[0] = cnt[-1] = 2
    rowptr = np.zeros(n + 1, dtype=np.int32)
    rowptr[1:] = np.cumsum(cnt)
    nnz = int(rowptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    i = np.arange(n)
    # row i holds (i-1, i, i+1) where they exist, in column order
    p = rowptr[:-1].astype(np.int64)
    has_lo = i > 0
    col[p[has_lo]] = i[has_lo] - 1
    val[p[has_lo]] = d_off[i[has_lo] - 1]
    pd = p + has_lo
    col[pd] = i
    val[pd] = d_main
    has_hi = i < n - 1
    col[pd[has_hi] + 1] = i[has_hi] + 1
    val[pd[has_hi] + 1] = d_off[i[has_hi]]
    rp, c, v = (torch.from_numpy(a).to(dev) for a in (rowptr, col, val))
    for call in range(2):
        xh = rng.standard_normal(n)
        yh = d_main * xh
        yh[1:] += d_off * xh[:-1]
        yh[:-1] += d_off * xh[1:]
        x = torch.from_numpy(xh).to(dev)
        y = torch.full_like(x, float("nan"))
        d = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
        G.spmv_dot_noalloc(rp, c, v, x, y, d)
        torch.cuda.synchronize()
        yg = y.cpu().numpy()
        assert np.max(np.abs(yg - yh)) <= 1e-13 * np.max(np.abs(yh))
        dh = float(np.dot(xh, yh))
        assert abs(float(d[0]) - dh) <= 1e-11 * abs(dh)
    st = G.lib().gic_spmv_dot_noalloc(n + 1, G._ptr(rp), G._ptr(c), G._ptr(v), G._ptr(x), G._ptr(y), G._ptr(d),
                                      None)
    assert st == G.GIC_ERR_TOO_LARGE
