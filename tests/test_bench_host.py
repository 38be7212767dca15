"""Host-side pieces of bench.py that need no GPU: the principal block the CPU
baseline samples (rows and columns of chosen indices, exactly), the scaling
of a sample to the full system, and the ncu traffic record's validity rule."""
import json
import os
import sys

import numpy as np

import oracle as O

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_principal_block_is_the_dense_submatrix():
    rng = np.random.default_rng(0)
    D = (rng.random((40, 40)) < 0.2) * rng.standard_normal((40, 40))
    D = D + D.T + np.diag(np.abs(D).sum(1) + 1.0)
    A = O.csr_from_dense(D)
    idx = np.array([0, 3, 4, 9, 17, 18, 30, 39])
    B = bench.principal_block(A, idx)
    assert np.array_equal(B.to_dense(), D[np.ix_(idx, idx)])


def test_oracle_estimate_scales_by_nonzeros_and_iterations():
    n, nnz, nnzL, _ = bench.workload_sizes(148)
    smp = dict(ic0_s=1.0, gnn_s=2.0, correct_s=0.5, features_s=0.25, pcg_iter_s=0.01, spmv_1_s=0.004,
               spmv_all_s=0.001, nnzA=nnz // 100, nnzL=nnzL // 100)
    one, allc, det = bench.oracle_estimate(148, smp, 600)
    fA, fL = nnz / smp["nnzA"], nnzL / smp["nnzL"]
    assert np.isclose(det["setup_s"], 3.5 * fL + 0.25 * fA)
    assert np.isclose(one, det["setup_s"] + 0.01 * fA * 600)
    assert np.isclose(allc, det["setup_s"] + (0.01 - 0.004 + 0.001) * fA * 600)


def test_ncu_traffic_needs_matching_size_precision_and_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "paper_2412_07127_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "k.cu").write_text("kernel source")
    import hashlib
    sha = hashlib.sha256(b"kernel source").hexdigest()[:16]
    (prof / "ncu_traffic.json").write_text(json.dumps(
        {"ltsolve/f64": {"source": "k.cu", "source_sha": sha, "N": 148, "bytes_per_launch": 123}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("ltsolve", 148, "f64") == 123
    assert bench.ncu_traffic("ltsolve", 69, "f64") is None
    assert bench.ncu_traffic("ltsolve", 148, "f32") is None
    (src / "k.cu").write_text("changed")
    assert bench.ncu_traffic("ltsolve", 148, "f64") is None
