"""What the trained GNN correction gains over plain IC(0) (the learned part's
benefit, judged by plain IC(0)-PCG), on held-out 20^3-element systems:
PCG iterations to 1e-8 and probe loss (Eq. 4-5) for IC(0), the untrained
network and the shipped trained network, and the fallback rule that keeps
IC(0) unless the corrected factor lowers the iteration count."""
import os

import numpy as np
import pytest
import torch

from paper_2412_07127_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2412_07127_gb300", "weights", "gnn_theta.npy")


@pytest.fixture(scope="module")
def G():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_07127_gb300 import build, gicpcg
    build.build()
    return gicpcg


def _evaluate(G, h, theta, N, seed):
    E = torch.from_numpy(I.material_field(N, seed)).to(DEV)
    rp, c, v = G.fem_hex_assemble(h, N, E)
    P = G.Pattern(h, rp, c)
    b = torch.from_numpy(I.rhs(P.n, seed)).to(DEV)
    LIC, alpha, _ = G.ic0_auto(h, P, v)
    x9, e0, scale, Ahat = G.features(h, P, v, with_ahat=True)
    Z = torch.from_numpy(I.probes(8, P.n, seed + 77)).to(DEV)
    out = {"ic0": G.pcg(h, P, v, LIC, b)}
    out["ic0_loss"] = float(G.probe_loss(h, P, Ahat, G.scale_factor(h, P, LIC, scale), Z)[0][1])
    for name, th in theta.items():
        g = G.gnn_forward(h, P, th, x9, e0)
        L, ok = G.gnn_correct(h, P, LIC, g, scale)
        out[name] = G.pcg(h, P, v, L, b, check=False) if ok else None
        Lh = G.gnn_correct_scaled(h, P, G.scale_factor(h, P, LIC, scale), g)
        out[name + "_loss"] = float(G.probe_loss(h, P, Ahat, Lh, Z)[0][1])
    P.close()
    return out


def test_trained_network_gain_over_ic0(G):
    from paper_2412_07127_gb300.train import load_weights
    h = G.Handle(0)
    th, meta = load_weights(WEIGHTS)
    assert meta is not None and meta["validation"]["runs"]
    theta = {"trained": torch.from_numpy(th).to(DEV),
             "untrained": torch.from_numpy(I.gnn_init(0, out_scale=0.02).astype(np.float32)).to(DEV)}
    rows = []
    for seed in (9100, 9101, 9102, 9103):
        r = _evaluate(G, h, theta, 20, seed)
        assert r["ic0"]["status"] == 0 and r["ic0"]["relres"] <= 1e-8
        for name in theta:
            assert r[name] is not None and r[name]["status"] == 0 and r[name]["relres"] <= 1e-8
        chosen = r["trained"]["iters"] if meta["use_gnn"] else r["ic0"]["iters"]
        rows.append((r["ic0"]["iters"], r["untrained"]["iters"], r["trained"]["iters"], chosen,
                     r["ic0_loss"], r["untrained_loss"], r["trained_loss"]))
    rows = np.array(rows, dtype=float)
    gain_iters = rows[:, 0].mean() - rows[:, 2].mean()       # IC(0) minus trained GNN
    gain_loss = 1.0 - rows[:, 6].mean() / rows[:, 4].mean()   # relative probe-loss reduction
    print(f"\nIC(0) / untrained / trained / chosen iterations: {rows[:, :4].mean(0)}; "
          f"probe loss IC(0) / untrained / trained: {rows[:, 4:].mean(0)}; "
          f"iteration gain {gain_iters:+.2f}, loss gain {gain_loss:+.4f}")
    # training lowered its own objective relative to the untrained network
    assert rows[:, 6].mean() < rows[:, 5].mean()
    # the shipped decision agrees with what held-out systems show ...
    assert meta["use_gnn"] == bool(gain_iters > 0) or abs(gain_iters) <= 1.0
    # ... and the fallback never costs iterations against plain IC(0)
    if not meta["use_gnn"]:
        assert np.array_equal(rows[:, 3], rows[:, 0])
    else:
        assert rows[:, 3].mean() <= rows[:, 0].mean() + 1.0
