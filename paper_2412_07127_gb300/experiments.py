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
  sweep      PCG iterations of IC(0) and of the corrected factor over seeds
             and sizes (Figures 2-4).

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


def sweep(h, Ns, seeds, weights):
    from .train import load_weights
    th, _ = load_weights(weights)
    theta = torch.from_numpy(th).cuda()
    for N in Ns:
        for seed in seeds:
            rp, c, v, P, b = _system(h, N, seed)
            L, alpha, _ = G.ic0_auto(h, P, v)
            x9, e0, scale, _ = G.features(h, P, v)
            g = G.gnn_forward(h, P, theta, x9, e0)
            Lc, ok = G.gnn_correct(h, P, L, g, scale)
            r0 = G.pcg(h, P, v, L, b)
            r1 = G.pcg(h, P, v, Lc, b, check=False) if ok else {"iters": -1}
            print(json.dumps({"experiment": "sweep", "N": N, "n": P.n, "seed": seed, "ic0": r0["iters"],
                              "gnn": r1["iters"], "shift": alpha}), flush=True)
            P.close()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("experiment", choices=["dropout", "deviation", "sweep"])
    ap.add_argument("--N", type=int, default=69)
    ap.add_argument("--Ns", default="8,12,20,40")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--seeds", default="9000,9001,9002,9003")
    ap.add_argument("--eps", default="0,0.001,0.01,0.02")
    ap.add_argument("--f32", action="store_true", help="apply the thinned factor in FP32")
    ap.add_argument("--grouped", action="store_true",
                    help="node-granular dropout: a column leaves all rows of a row group or none")
    ap.add_argument("--weights", default=WEIGHTS)
    a = ap.parse_args(argv)
    h = G.Handle(0)
    if a.experiment == "dropout":
        dropout(h, a.N, a.seed, [float(x) for x in a.eps.split(",")], a.f32, a.grouped)
    elif a.experiment == "deviation":
        deviation(h, a.N, a.seed, a.weights)
    else:
        sweep(h, [int(x) for x in a.Ns.split(",")], [int(x) for x in a.seeds.split(",")], a.weights)


if __name__ == "__main__":
    main()
