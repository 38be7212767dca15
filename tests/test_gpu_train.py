"""The training driver end to end on tiny systems: a run interrupted after
its checkpoint and resumed ends with the same parameters, bit for bit, as
the same run made in one go (inputs are regenerated from their seeds; the
checkpoint holds the parameters, Adam's moments and the step), and the kept
weights are those of the validation with the fewest PCG iterations."""
import json
import os

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, train
    build.build()
    return train


def _args(out, extra):
    return ["--N", "3", "--batch", "2", "--train-systems", "4", "--probes", "4", "--val-N", "3",
            "--lr", "0.002", "--out", out] + extra


def test_resume_matches_an_uninterrupted_run(T, tmp_path):
    one = str(tmp_path / "one.npy")
    T.main(_args(one, ["--epochs", "3", "--log", str(tmp_path / "one_log.json")]))
    two = str(tmp_path / "two.npy")
    ck = str(tmp_path / "two.ckpt")
    T.main(_args(two, ["--epochs", "3", "--steps", "4", "--checkpoint", ck]))
    T.main(_args(two, ["--epochs", "3", "--checkpoint", ck, "--resume", "--log", str(tmp_path / "two_log.json")]))
    l1 = json.load(open(tmp_path / "one_log.json"))
    l2 = json.load(open(tmp_path / "two_log.json"))
    assert [r["mean"] for r in l1["val"]] == [r["mean"] for r in l2["val"]]
    assert np.array_equal(np.load(one), np.load(two))
    meta = json.load(open(os.path.splitext(one)[0] + ".json"))
    best = min(l1["val"], key=lambda r: (r["mean"], r["step"]))
    assert meta["training"]["kept_step"] == best["step"]
    assert meta["use_gnn"] == (meta["validation"]["iters_gnn_mean"] < meta["validation"]["iters_ic0_mean"])
