"""The no-allocation SpMV entry point, for callers that cannot allocate device
memory, gives the same y and x^T y as gic_spmv on two calls in a row (its
scratch is shared across calls and must not leak state from one to the next).
Collected last on purpose: it runs alone or after every other test."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2412_07127_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    with pytest.raises(G.GicError) as e:
        G.lib()  # too many rows is rejected before any launch
        st = G.lib().gic_spmv_dot_noalloc(8 * (1 << 20) + 1, G._ptr(rp), G._ptr(c), G._ptr(v), G._ptr(x),
                                          G._ptr(y), G._ptr(d), None)
        raise G.GicError("gic_spmv_dot_noalloc", st)
    assert e.value.status == G.GIC_ERR_TOO_LARGE
