"""Experiments beyond the headline bench, each through the library's C-ABI
(every arithmetic step in its CUDA kernels; this module only draws inputs,
sequences calls and times them with CUDA events):

  dropout    fill-in dropout (Supplementary 5, Eq. (10), Table 3): for each
             epsilon, nnz of the thinned factor, PCG iterations, setup and CG
             time, mean triangular-solve time. --grouped thins per row
             group (a node's rows) instead of per entry.
  deviation  the factor deviation of the paper's Figure 5: mean and maximum
             |L - L_IC| / |L_IC| on and off the diagonal for the shipped
             network (correcting IC(0)) and for a direct prediction.
  sweep      PCG iterations of IC(0), of the corrected factor and (with
             --nic-weights) of the direct prediction over seeds and sizes
             (Figures 2-4).
  table      IC(0) / NIC (direct prediction, Eq. (1)) / GNN-IC (Eq. (2)) per
             size, as Table 1 lays them out: iterations, P-time (factor
             construction), CG-time, and the Figure 5 deviation of each
             learned factor from L_IC; times by CUDA events.

Usage: python -m paper_2412_07127_gb300.experiments dropout --N 69
Each line printed is one JSON record.
"""
import argparse
import json
import os

import numpy as np
import torch

from . import gicpcg as G
from . import inputs as I

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "gnn_theta.npy")
NIC_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "nic_theta.npy")


def _system(h, N, seed, sigma=1.0):
    dev = torch.device("cuda:0")
    E = torch.from_numpy(I.material_field(N, seed, sigma)).to(dev)
    rp, c, v = G.fem_hex_assemble(h, N, E)
    P = G.Pattern(h, rp, c)
    b = torch.from_numpy(I.rhs(P.n, seed)).to(dev)
    return rp, c, v, P, b


def _timed(fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def dropout(h, N, seed, eps_list, f32, grouped=False):
    rp, c, v, P, b = _system(h, N, seed)
    L, _ = G.ic0(h, P, v)
    _, _, scale, _ = G.features(h, P, v)
    sq = float(np.sqrt(scale.item()))
    for eps in eps_list:
        (Srp, Sc, Lv), t_drop = _timed(lambda: G.dropout(h, P, L, eps * sq, grouped=grouped))
        PS, t_an = _timed(lambda: G.Pattern(h, Srp, Sc))
        Lr = G.to_f32(h, Lv) if f32 else Lv
        G.pcg_split(h, P, v, PS, Lr, b, maxit=3)  # warm
        G.profile_enable(h, True)
        r, t_cg = _timed(lambda: G.pcg_split(h, P, v, PS, Lr, b))
        prof = G.profile_read(h)
        G.profile_enable(h, False)
        tri = (prof["lsolve"]["ms"] + prof["ltsolve"]["ms"]) / max(1, prof["lsolve"]["launches"]) / 1e3
        print(json.dumps({"experiment": "dropout", "N": N, "n": P.n, "eps": eps, "nnzL": int(Lv.numel()),
                          "nnzL_fraction": Lv.numel() / P.nnzL, "iters": r["iters"], "relres": r["relres"],
                          "setup_s": t_drop + t_an, "cg_s": t_cg, "trisolve_pair_s": tri,
                          "l_dtype": "f32" if f32 else "f64", "granularity": "node" if grouped else "entry",
                          "solve_kernels": "warp-specialised" if PS.warp_specialised else "staged"}),
              flush=True)
        PS.close()


def deviation(h, N, seed, weights):
    from .train import load_weights
    rp, c, v, P, b = _system(h, N, seed)
    L, _ = G.ic0(h, P, v)
    x9, e0, scale, _ = G.features(h, P, v)
    th, meta = load_weights(weights)
    g = G.gnn_forward(h, P, torch.from_numpy(th).cuda(), x9, e0)
    Lc, ok = G.gnn_correct(h, P, L, g, scale)
    d = G.factor_deviation(h, P, L, Lc)
    print(json.dumps({"experiment": "deviation", "N": N, "factor": "IC(0) corrected by the shipped network",
                      "diag_mean": d[0], "diag_max": d[1], "off_mean": d[2], "off_max": d[3],
                      "positive": ok}), flush=True)


def _learned_factor(h, P, v, L, theta, nic):
    """The network's factor: IC(0) corrected (Eq. 2) or, for NIC, the
    identity base corrected, i.e. the direct prediction (Eq. 1)."""
    x9, e0, scale, _ = G.features(h, P, v)
    g = G.gnn_forward(h, P, theta, x9, e0)
    base = G.identity_factor(h, P, scale)[0] if nic else L
    return G.gnn_correct(h, P, base, g, scale)


def sweep(h, Ns, seeds, weights, nic_weights=None):
    from .train import load_weights
    theta = torch.from_numpy(load_weights(weights)[0]).cuda()
    tnic = torch.from_numpy(load_weights(nic_weights)[0]).cuda() if nic_weights else None
    for N in Ns:
        for seed in seeds:
            rp, c, v, P, b = _system(h, N, seed)
            L, alpha, _ = G.ic0_auto(h, P, v)
            Lc, ok = _learned_factor(h, P, v, L, theta, False)
            r0 = G.pcg(h, P, v, L, b)
            r1 = G.pcg(h, P, v, Lc, b, check=False) if ok else {"iters": -1, "status": -1}
            rec = {"experiment": "sweep", "N": N, "n": P.n, "seed": seed, "ic0": r0["iters"],
                   "gnn": r1["iters"] if r1["status"] == 0 else -1, "shift": alpha}
            if tnic is not None:
                Ln, okn = _learned_factor(h, P, v, L, tnic, True)
                r2 = G.pcg(h, P, v, Ln, b, check=False) if okn else {"iters": -1, "status": -1}
                rec["nic"] = r2["iters"] if r2["status"] == 0 else -1
            print(json.dumps(rec), flush=True)
            P.close()


def table(h, Ns, seeds, weights, nic_weights, reps=2):
    from .train import load_weights
    theta = torch.from_numpy(load_weights(weights)[0]).cuda()
    tnic = torch.from_numpy(load_weights(nic_weights)[0]).cuda()
    for N in Ns:
        for seed in seeds:
            rp, c, v, P, b = _system(h, N, seed)
            rows = {}
            for name in ("ic0", "nic", "gnn_ic"):
                best = None
                for _ in range(reps):   # the first run includes one-time costs (workspaces, module load)
                    def build():
                        L, _, _ = G.ic0_auto(h, P, v)
                        if name == "ic0":
                            return L, L, True
                        Lf, ok = _learned_factor(h, P, v, L, tnic if name == "nic" else theta, name == "nic")
                        return L, Lf, ok
                    (L, Lf, ok), tp = _timed(build)
                    if name == "nic":   # the direct prediction needs no IC(0): time it without
                        (_, ok), tp = _timed(lambda: _learned_factor(h, P, v, None, tnic, True))
                    r, tc = _timed(lambda: G.pcg(h, P, v, Lf, b, check=False) if ok else {"iters": -1, "status": -1})
                    if best is None or tp + tc < best["p_time_s"] + best["cg_time_s"]:
                        best = {"iters": r["iters"] if r["status"] == 0 else -1, "p_time_s": tp, "cg_time_s": tc,
                                "positive": ok}
                        if name != "ic0":
                            d = G.factor_deviation(h, P, L, Lf)
                            best.update(dev_diag_mean=d[0], dev_off_mean=d[2])
                rows[name] = best
            print(json.dumps({"experiment": "table", "N": N, "n": P.n, "nnz": P.nnzA, "seed": seed, **rows}),
                  flush=True)
            P.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("experiment", choices=["dropout", "deviation", "sweep", "table"])
    ap.add_argument("--N", type=int, default=69)
    ap.add_argument("--Ns", default="8,12,20,40")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seeds", default="9000,9001,9002,9003")
    ap.add_argument("--eps", default="0,0.001,0.01,0.02")
    ap.add_argument("--f32", action="store_true", help="apply the thinned factor in FP32")
    ap.add_argument("--grouped", action="store_true",
                    help="node-granular dropout: a column leaves all rows of a row group or none")
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--nic-weights", default=None, help=f"NIC weights (table: default {NIC_WEIGHTS})")
    a = ap.parse_args(argv)
    h = G.Handle(0)
    if a.experiment == "dropout":
        dropout(h, a.N, a.seed, [float(x) for x in a.eps.split(",")], a.f32, a.grouped)
    elif a.experiment == "deviation":
        deviation(h, a.N, a.seed, a.weights)
    elif a.experiment == "table":
        table(h, [int(x) for x in a.Ns.split(",")], [int(x) for x in a.seeds.split(",")], a.weights,
              a.nic_weights or NIC_WEIGHTS)
    else:
        sweep(h, [int(x) for x in a.Ns.split(",")], [int(x) for x in a.seeds.split(",")], a.weights,
              a.nic_weights)


if __name__ == "__main__":
    main()
