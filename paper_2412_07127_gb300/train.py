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

Training runs a fixed set of generated systems for a number of epochs,
validates every epoch (PCG iterations on held-out systems) and keeps the
weights of the validation with the fewest iterations (Section "Training and
Inference"); --checkpoint / --resume save and restore the whole state. The
gradient comes from loss.backward() through the torch.autograd Functions of
paper_2412_07127_gb300.autograd.

Usage: python -m paper_2412_07127_gb300.train --epochs 50 --out theta.npy
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

    def batch(self, k, probe_epoch=0):
        """Device inputs of batch k: (x9, e0, A_hat, L_IC_hat, Z); the probes
        of a later epoch are drawn afresh."""
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
        Z = np.concatenate([I.probes(self.m, self.n, s + 1_000_003 * probe_epoch) for s in self._seeds(k)], axis=1)
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
                     "epochs": a.get("epochs"), "train_systems": a.get("train_systems"), "mode": a.get("mode"),
                     "compute": a.get("compute", "fp32") + " edge MLP, FP32 master weights",
                     "kept_step": log.get("best_step"),
                     "validation_means": [[r["step"], r["mean"]] for r in log["val"]],
                     "ic0_shifts_seen": log["ic0_shifts"],
                     "loss_ratio_to_ic0_first": round(st[0]["ratio"], 4),
                     "loss_ratio_to_ic0_last": round(st[-1]["ratio"], 4)},
        "validation": {"systems": f"{a['val_N']}^3-element hex elasticity, sigma = 1, seeds 9000-9015, "
                                  f"PCG to 1e-8, FP64", "iters_ic0_mean": ic0, "iters_gnn_mean": gnn, "runs": v},
        "use_gnn": bool(gnn < ic0),
        "policy": "the weights kept are those of the validation with the fewest iterations (the starting "
                  "point included); the corrected factor is used only when that count is below plain IC(0)'s, "
                  "otherwise plain IC(0) is the fallback",
    }


def load_weights(path):
    """(theta float32, metadata dict or None) of a weights file."""
    th = np.load(path).astype(np.float32)
    meta_path = os.path.splitext(path)[0] + ".json"
    meta = json.load(open(meta_path)) if os.path.exists(meta_path) else None
    return th, meta


def save_checkpoint(path, theta, m1, m2, step, log):
    """Everything a run needs to resume: parameters, Adam moments, the next
    step and the log so far (the inputs are regenerated from their seeds)."""
    tmp = path + ".tmp"
    torch.save({"theta": theta.detach().cpu(), "m1": m1.cpu(), "m2": m2.cpu(), "step": step, "log": log}, tmp)
    os.replace(tmp, path)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--epochs", type=int, default=50, help="passes over the training set")
    ap.add_argument("--train-systems", type=int, default=400, help="systems in the training set")
    ap.add_argument("--steps", type=int, default=0, help="if > 0: stop after this many steps")
    ap.add_argument("--N", type=int, default=20)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--probes", type=int, default=8)
    ap.add_argument("--lr", type=float, default=0.005)
    ap.add_argument("--warmup-frac", type=float, default=0.05)
    ap.add_argument("--init-seed", type=int, default=0)
    ap.add_argument("--init-out-scale", type=float, default=0.02)
    ap.add_argument("--seed0", type=int, default=1000)
    ap.add_argument("--time-limit", type=float, default=1e9, help="seconds; stop early")
    ap.add_argument("--val-every", type=int, default=0, help="steps between validations (0: once per epoch)")
    ap.add_argument("--val-N", type=int, default=20)
    ap.add_argument("--mode", default="ic", choices=["ic", "nic"])
    ap.add_argument("--compute", default="bf16", choices=["bf16", "fp32"],
                    help="edge-MLP arithmetic of the training forward/backward (FP32 master weights either way)")
    ap.add_argument("--checkpoint", default=None, help="resumable state, written at every validation")
    ap.add_argument("--resume", action="store_true", help="continue from --checkpoint")
    ap.add_argument("--out", required=True)
    ap.add_argument("--log", default=None)
    a = ap.parse_args(argv)
    from .autograd import training_loss

    h = G.Handle(0)
    G.set_tuning(h, G.GIC_TUNE_TRAIN_BF16, 1 if a.compute == "bf16" else 0)
    tr = Trainer(h, a.N, a.batch, a.probes, a.seed0, mode=a.mode)
    dev = tr.dev
    nb = max(1, a.train_systems // a.batch)        # batches per epoch (a fixed training set)
    total = nb * a.epochs if a.steps <= 0 else a.steps
    val_every = a.val_every if a.val_every > 0 else nb
    warm = int(a.warmup_frac * total)
    theta = torch.from_numpy(I.gnn_init(a.init_seed, a.init_out_scale).astype(np.float32)).to(dev)
    m1, m2 = torch.zeros_like(theta), torch.zeros_like(theta)
    log = dict(args=vars(a), steps=[], val=[], train_seconds_before=0.0)
    t_start = 0
    if a.resume and a.checkpoint and os.path.exists(a.checkpoint):
        ck = torch.load(a.checkpoint)
        theta, m1, m2 = ck["theta"].to(dev), ck["m1"].to(dev), ck["m2"].to(dev)
        t_start, log = ck["step"], ck["log"]
    # validation baseline: plain IC(0) iterations on the held-out systems, and
    # the starting point itself, which the best-by-iterations rule may keep
    if not log["val"]:
        v0 = validate(h, theta, N=a.val_N, mode=a.mode)
        log["val"].append(dict(step=0, runs=v0, mean=float(np.mean([r["gnn"] if r["gnn"] >= 0 else np.inf
                                                                      for r in v0]))))
        print(json.dumps(dict(step=0, val_mean=log["val"][-1]["mean"])), flush=True)
    t0 = time.time()
    t = t_start
    for t in range(t_start, total):
        # batch t mod nb of the training set; fresh Gaussian probes each epoch
        data = tr.batch(t % nb, probe_epoch=t // nb)
        x9, e0, Ahat, LIChat, Z = data
        th = theta.clone().requires_grad_(True)
        loss = training_loss(th, h, tr.P, x9, e0, LIChat, Ahat, Z, ngraphs=a.batch, gnn_ws=tr.ws, probe_ws=tr.pws)
        loss.backward()
        grad = th.grad
        G.adam_step(h, theta, grad, m1, m2, t + 1, lr_at(t, warm, a.lr))
        if t % 20 == 0 or t == total - 1:
            l_ic = float(tr.ic0_loss(data)[a.batch])
            rec = dict(step=t, loss=float(loss), loss_ic0=l_ic, ratio=float(loss) / l_ic,
                       gnorm=float(grad.norm()), wall=log["train_seconds_before"] + time.time() - t0)
            log["steps"].append(rec)
            print(json.dumps(rec), flush=True)
        if (t + 1) % val_every == 0 or t == total - 1:
            v = validate(h, theta, N=a.val_N, mode=a.mode)
            mean = float(np.mean([r["gnn"] if r["gnn"] >= 0 else np.inf for r in v]))
            log["val"].append(dict(step=t + 1, runs=v, mean=mean))
            print(json.dumps(dict(step=t + 1, val_mean=mean)), flush=True)
            best = min(log["val"], key=lambda r: (r["mean"], r["step"]))
            if best["step"] == t + 1:   # the paper keeps the step with the fewest validation iterations
                np.save(a.out, theta.cpu().numpy())
            if a.checkpoint:
                save_checkpoint(a.checkpoint, theta, m1, m2, t + 1,
                                dict(log, train_seconds_before=log["train_seconds_before"] + time.time() - t0))
        if time.time() - t0 > a.time_limit:
            break
    torch.cuda.synchronize()
    log["train_seconds"] = log["train_seconds_before"] + time.time() - t0
    log["steps_done"] = t + 1
    log["ic0_shifts"] = sorted(set(tr.shifts))
    best = min(log["val"], key=lambda r: (r["mean"], r["step"]))
    if best["step"] == 0:   # nothing beat the starting point
        np.save(a.out, I.gnn_init(a.init_seed, a.init_out_scale).astype(np.float32))
    log["best_step"] = best["step"]
    log["final_val"] = best["runs"]
    with open(os.path.splitext(a.out)[0] + ".json", "w") as f:
        json.dump(weights_meta(log), f, indent=1)
    if a.log:
        with open(a.log, "w") as f:
            json.dump(log, f, indent=1)


if __name__ == "__main__":
    main()
