"""Writes the stored oracle results that the full-size GPU parity test
(tests/test_gpu_golden.py) compares with: IC(0)-PCG to a relative residual of
1e-8 (Supplementary Algorithm 1) on the seeded hex elasticity systems of
69^3 and 148^3 elements, once with the FP64 factor and once with the factor
rounded to FP32 (the values the FP32-apply path stores; the oracle still
computes in FP64). Calls only oracle/ and the seeded input generators.

A full x does not fit in a test fixture (10M values at 148^3), so each file
keeps the iteration count, the final relative residual, ||x||_2 and x at
1,000 seeded indices.

    python tests/golden/make_pcg_golden.py 69 148     # hours of one core at 148^3
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2412_07127_gb300 import inputs as I  # noqa: E402

SEED = 0
SAMPLES = 1000


def sample_indices(n):
    return np.sort(np.random.default_rng(12345).choice(n, size=SAMPLES, replace=False))


def run(N):
    t0 = time.time()
    A = O.fem_hex_assemble(N, I.material_field(N, SEED))
    b = I.rhs(A.n, SEED)
    L, alpha, bad = O.ic0_auto(A)
    assert bad < 0
    idx = sample_indices(A.n)
    out = {"workload": f"hex elasticity {N}^3 elements, seed {SEED}, nu 0.3, E = exp(N(0,1)), b ~ U[-1,1], "
                       f"x0 = 0, IC(0)-PCG to ||r||/||b|| <= 1e-8 (Supplementary Algorithm 1)",
           "N": N, "n": int(A.n), "nnz": int(A.nnz), "ic0_shift": alpha, "indices": idx.tolist()}
    for name, Lv in (("f64", L.val), ("f32", L.val.astype(np.float32).astype(np.float64))):
        r = O.pcg(A, b, O.CSR(L.rowptr, L.col, Lv), tol=1e-8, maxit=20000)
        assert r["status"] == 0
        x = r["x"]
        out[name] = {"iters": int(r["iters"]), "relres": float(r["relres"]),
                     "x_norm": float(np.linalg.norm(x)), "x_at": x[idx].tolist()}
        print(N, name, r["iters"], f"{time.time() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, f"pcg_hex{N}_seed{SEED}.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    for a in sys.argv[1:]:
        run(int(a))
