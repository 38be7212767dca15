"""Training driver of the GNN correction (Section 3: probe-vector loss of
Eq. 4-5, Adam with warm-up; Section 4's setting of many small generated
systems). Every arithmetic step runs in the library's CUDA kernels; this
module only draws the seeded inputs and sequences the calls.

One step on a batch of B independent N^3 systems (one block-diagonal pattern):
  assemble A (per-system log-normal E, sigma ~ U[0.5, 2]) -> IC(0) with the
  diagonal-shift rule -> features, scale s, A/s -> GNN forward (kept tape) ->
  L_hat = corrected L_IC/sqrt(s) -> probe loss and dL_hat -> correction
  backward -> GNN backward -> Adam.
The batch's pattern is the same at every step, so it is analysed once.

Usage: python -m paper_2412_07127_gb300.train --steps 2000 --out theta.npy
"""
import argparse
import json
import os
import time

import numpy as np
import torch

from . import gicpcg as G
from . import inputs as I


def lr_at(t, warm, lr_max):
    """Linear warm-up over the first `warm` steps (t counted from 0), then constant."""
    if warm <= 0 or t >= warm:
        return lr_max
    return lr_max * t / warm


class Trainer:
    """mode "ic": the network corrects IC(0) (Eq. (2), the method); mode
    "nic": it predicts L directly (Eq. (1), the paper's ablation), i.e. it
    corrects the identity factor instead of L_IC."""

    def __init__(self, h, N=20, batch=16, probes=8, seed0=1000, sigma_lo=0.5, sigma_hi=2.0,
                 device="cuda:0", mode="ic"):
        self.h, self.N, self.B, self.m, self.mode = h, N, batch, probes, mode
        self.seed0, self.lo, self.hi = seed0, sigma_lo, sigma_hi
        self.dev = torch.device(device)
        self.n = I.fem_sizes(N)[0]
        rp, col, _ = self._assemble(0)
        self.rp, self.col = rp, col          # kept alive: the pattern borrows them
        self.P = G.Pattern(h, rp, col)
        # one system's pattern: IC(0) and its shift rule run per system
        _, self.nnz1 = G.fem_hex_sizes(N)
        self.rp1, self.col1 = rp[:self.n + 1].clone(), col[:self.nnz1].clone()
        self.P1 = G.Pattern(h, self.rp1, self.col1)
        self.ws = G.gnn_workspace(h, self.P, batch, training=True)
        self.pws = G.probe_workspace(h, self.P, batch, probes)
        self.shifts = []

    def _seeds(self, k):
        return [self.seed0 + k * self.B + j for j in range(self.B)]

    def _assemble(self, k):
        Es = [I.material_field(self.N, s, I.training_sigma(s, self.lo, self.hi)) for s in self._seeds(k)]
        E = torch.from_numpy(np.concatenate(Es)).to(self.dev)
        return G.fem_hex_assemble(self.h, self.N, E, nb=self.B)

    def batch(self, k):
        """Device inputs of batch k: (x9, e0, A_hat, L_IC_hat, Z)."""
        _, _, v = self._assemble(k)
        LIC = torch.empty(self.P.nnzL, dtype=torch.float64, device=self.dev)
        nL = self.P1.nnzL
        for j in range(self.B):   # the batch's L is the concatenation of the systems' L
            _, alpha, bad = G.ic0_auto(self.h, self.P1, v[j * self.nnz1:(j + 1) * self.nnz1],
                                       out=LIC[j * nL:(j + 1) * nL])
            if bad != -1:
                raise RuntimeError(f"IC(0) failed on batch {k} even with shifts")
            self.shifts.append(alpha)
        x9, e0, scale, Ahat = G.features(self.h, self.P, v, ngraphs=self.B, with_ahat=True)
        if self.mode == "nic":
            LIChat = G.identity_factor(self.h, self.P, want_L=False, want_hat=True)[1]
        else:
            LIChat = G.scale_factor(self.h, self.P, LIC, scale, ngraphs=self.B)
        Z = np.concatenate([I.probes(self.m, self.n, s) for s in self._seeds(k)], axis=1)
        return x9, e0, Ahat, LIChat, torch.from_numpy(Z).to(self.dev)

    def loss_grad(self, theta, data, grad=True):
        x9, e0, Ahat, LIChat, Z = data
        h, P, B = self.h, self.P, self.B
        g = G.gnn_forward_train(h, P, theta, x9, e0, self.ws, ngraphs=B)
        Lhat = G.gnn_correct_scaled(h, P, LIChat, g)
        loss, dL = G.probe_loss(h, P, Ahat, Lhat, Z, ngraphs=B, grad=grad, ws=self.pws)
        if not grad:
            return loss, None
        dg = G.gnn_correct_backward(h, P, Lhat, dL)
        return loss, G.gnn_backward(h, P, theta, x9, e0, dg, self.ws, ngraphs=B)

    def ic0_loss(self, data):
        """Probe loss of the uncorrected factor (g = 0) on the same batch."""
        x9, e0, Ahat, LIChat, Z = data
        loss, _ = G.probe_loss(self.h, self.P, Ahat, LIChat, Z, ngraphs=self.B, ws=self.pws)
        return loss


def validate(h, theta, N=20, seeds=range(9000, 9016), sigma=1.0, l_dtype=torch.float64, mode="ic"):
    """PCG iterations to 1e-8 with plain IC(0) and with the network's factor
    (IC(0) corrected, or for mode "nic" the direct prediction)."""
    out = []
    dev = theta.device
    for s in seeds:
        E = torch.from_numpy(I.material_field(N, s, sigma)).to(dev)
        rp, col, v = G.fem_hex_assemble(h, N, E)
        P = G.Pattern(h, rp, col)
        b = torch.from_numpy(I.rhs(P.n, s)).to(dev)
        LIC, alpha, _ = G.ic0_auto(h, P, v)
        x9, e0, scale, _ = G.features(h, P, v)
        g = G.gnn_forward(h, P, theta, x9, e0)
        base = G.identity_factor(h, P, scale)[0] if mode == "nic" else LIC
        L, ok = G.gnn_correct(h, P, base, g, scale)
        r0 = G.pcg(h, P, v, LIC.to(l_dtype), b)
        r1 = G.pcg(h, P, v, L.to(l_dtype), b, check=False) if ok else dict(iters=-1, status=-1)
        if r1["status"] != 0:
            r1 = dict(iters=-1)
        out.append(dict(seed=s, ic0=r0["iters"], gnn=r1["iters"], positive=ok, shift=alpha))
        P.close()
    return out


def weights_meta(log):
    """Metadata stored beside trained weights: training record, validation
    PCG iterations against plain IC(0), and the fallback decision (the
    corrected factor is used only if it lowers the validation iterations)."""
    a = log["args"]
    v = log["final_val"]
    ic0 = float(np.mean([r["ic0"] for r in v]))
    gnn = float(np.mean([r["gnn"] if r["gnn"] >= 0 else np.inf for r in v]))
    st = log["steps"]
    return {
        "about": "GNN correction weights (3504 float32) trained by paper_2412_07127_gb300.train on the GPU "
                 "with the library's own forward/backward kernels",
        "training": {"systems": f"{a['batch']} x {a['N']}^3-element hex elasticity per batch, sigma ~ U[0.5, 2] "
                                f"per system, seeds {a['seed0']}+",
                     "probes": f"{a['probes']} Gaussian per system", "steps_done": log["steps_done"],
                     "seconds": round(log["train_seconds"], 1), "lr": a["lr"], "warmup_frac": a["warmup_frac"],
                     "ic0_shifts_seen": log["ic0_shifts"],
                     "loss_ratio_to_ic0_first": round(st[0]["ratio"], 4),
                     "loss_ratio_to_ic0_last": round(st[-1]["ratio"], 4)},
        "validation": {"systems": f"{a['val_N']}^3-element hex elasticity, sigma = 1, seeds 9000-9015, "
                                  f"PCG to 1e-8, FP64", "iters_ic0_mean": ic0, "iters_gnn_mean": gnn, "runs": v},
        "use_gnn": bool(gnn < ic0),
        "policy": "the corrected factor is used only when its validation iteration count is below plain "
                  "IC(0)'s; otherwise plain IC(0) is the fallback",
    }


def load_weights(path):
    """(theta float32, metadata dict or None) of a weights file."""
    th = np.load(path).astype(np.float32)
    meta_path = os.path.splitext(path)[0] + ".json"
    meta = json.load(open(meta_path)) if os.path.exists(meta_path) else None
    return th, meta


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--N", type=int, default=20)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--probes", type=int, default=8)
    ap.add_argument("--lr", type=float, default=0.005)
    ap.add_argument("--warmup-frac", type=float, default=0.05)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--init-out-scale", type=float, default=0.02)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--time-limit", type=float, default=1e9, help="seconds; stop early")
    ap.add_argument("--val-every", type=int, default=0)
    ap.add_argument("--val-N", type=int, default=20)
    ap.add_argument("--mode", default="ic", choices=["ic", "nic"])
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None)
    a = ap.parse_args(argv)

    h = G.Handle(0)
    tr = Trainer(h, a.N, a.batch, a.probes, a.seed0, mode=a.mode)
    dev = tr.dev
    theta = torch.from_numpy(I.gnn_init(a.init_seed, a.init_out_scale).astype(np.float32)).to(dev)
    m1, m2 = torch.zeros_like(theta), torch.zeros_like(theta)
    warm = int(a.warmup_frac * a.steps)
    log = dict(args=vars(a), steps=[], val=[])
    t0 = time.time()
    for t in range(a.steps):
        data = tr.batch(t)
        loss, grad = tr.loss_grad(theta, data)
        G.adam_step(h, theta, grad, m1, m2, t + 1, lr_at(t, warm, a.lr))
        if t % 20 == 0 or t == a.steps - 1:
            l_ic = float(tr.ic0_loss(data)[a.batch])
            rec = dict(step=t, loss=float(loss[a.batch]), loss_ic0=l_ic, ratio=float(loss[a.batch]) / l_ic,
                       gnorm=float(grad.norm()), wall=time.time() - t0)
            log["steps"].append(rec)
            print(json.dumps(rec), flush=True)
        if a.val_every and (t + 1) % a.val_every == 0:
            v = validate(h, theta, N=a.val_N, seeds=range(9000, 9004), mode=a.mode)
            log["val"].append(dict(step=t + 1, runs=v))
            print(json.dumps(dict(step=t + 1, val=v)), flush=True)
        if time.time() - t0 > a.time_limit:
            break
    torch.cuda.synchronize()
    log["train_seconds"] = time.time() - t0
    log["steps_done"] = t + 1
    log["ic0_shifts"] = sorted(set(tr.shifts))
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    np.save(a.out, theta.cpu().numpy())
    v = validate(h, theta, N=a.val_N, mode=a.mode)
    log["final_val"] = v
    print(json.dumps(dict(final_val=v)), flush=True)
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(weights_meta(log), f, indent=1)
    if a.log:
        with open(a.log, "w") as f:
            json.dump(log, f, indent=1)


if __name__ == "__main__":
    main()
