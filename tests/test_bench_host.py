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


def test_clock_sampler_summary_from_nvidia_smi_rows():
    """The clock record the timing rules read: median SM clock under load,
    the maximum, and every throttle reason seen Active in any sample."""
    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = _Done()
    na, act = "Not Active", "Active"
    cs.rows = [["2070", "2070", "650.1", "0x0", na, na, na, na],
               ["2055", "2070", "731.9", "0x4", na, na, na, act],
               ["2070", "2070", "700.0", "0x0", na, na, na, na],
               ["[N/A]", "2070", "699.0", "0x0", na, na, na, na],
               ["short row"]]
    rec = cs.stop()
    assert rec["sm_mhz"] == 2070.0 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples"] == 4 and rec["power_w_max"] == 731.9
    cs.rows = [["1200", "2070", "400", "0x0", act, na, na, na]]
    assert cs.stop()["reasons"] == ["hw_slowdown"]


def test_kernel_bytes_hand_count_at_one_element():
    """Algorithmic bytes for the 1-element system (n = 12 free dofs: the
    clamped face removed), counted by hand from its sizes: CSR of A or L once
    plus the vectors once."""
    n, nnz, nnzL, _ = bench.workload_sizes(1)
    assert (n, nnz) == (12, 144) and nnzL == (nnz + n) // 2
    kb = bench.kernel_bytes(1, "f64")
    assert kb["spmv"] == 12 * 144 + 4 * 13 + 16 * 12
    assert kb["lsolve"] == 12 * 78 + 4 * 13 + 16 * 12
    assert kb["ltsolve"] == kb["lsolve"] + 8 * 12
    k32 = bench.kernel_bytes(1, "f32")
    assert k32["lsolve"] == 8 * 78 + 4 * 13 + 8 * 12
