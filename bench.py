"""Benchmark: GNN-corrected IC(0)-PCG vs plain IC(0)-PCG to a 1e-8 relative
residual on the synthetic 40^3-element hex elasticity system (201,720 dofs,
15.5M nonzeros), FP64 CG, on one GB300.

A step is one pass of the hot path over one system already resident in HBM:
IC(0) factorisation, graph features, GNN forward, correction of L, PCG with
the corrected factor (the headline path) and, for comparison, PCG with the
plain IC(0) factor. `value` is the mean seconds of the GNN-IC solve
(IC(0) + features + GNN + correction + PCG). `e2e` is the same solve through
gic_solve_host: A and b copied from pinned host memory, x copied back.

Prints one JSON line (rank 0). --impl reference times the CPU oracle instead.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG s-to-1e-8 and iters, GNN-IC vs IC(0) on one GB300; SpMV/SpTRSV GB/s"
WEIGHTS = os.path.join(ROOT, "paper_2412_07127_gb300", "weights", "gnn_theta.npy")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=40)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ldtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f32", action="store_true", help="skip the FP32-apply comparison")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(seed, rank):
    """Weak scaling by replicas: every rank solves its own seeded system."""
    return seed + rank


def sync_all(world, dev=None):
    """Device synchronise, then a barrier over the ranks (taken on both sides
    of the timed region)."""
    import torch
    if dev is not None and dev.type == "cuda":
        torch.cuda.synchronize(dev)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(vals, world, dev):
    """Element-wise maximum of a list of floats over the ranks."""
    if world == 1:
        return [float(v) for v in vals]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def workload_config(N, theta_src, ldtype):
    n, nnz, nnzL, lev = workload_sizes(N)
    return {"workload": f"hex elasticity {N}^3 elements ({n} dofs, {nnz} nnz), E=exp(N(0,1)), "
                        f"nu=0.3, GNN-IC vs IC(0) PCG to 1e-8",
            "N": N, "n": n, "nnz": nnz, "nnzL": nnzL, "levels": lev,
            "gnn_weights": theta_src, "l_dtype": ldtype,
            "l2": (f"inputs larger than L2 (A {12 * nnz / 1e6:.0f} MB, L {12 * nnzL / 1e6:.0f} MB "
                   f"in FP64); no flush" if 12 * nnz > 129e6 else "inputs smaller than L2; no flush")}


def load_theta(N_PARAMS):
    import numpy as np
    from paper_2412_07127_gb300 import inputs as I
    from paper_2412_07127_gb300.train import load_weights
    if os.path.exists(WEIGHTS):
        th, _ = load_weights(WEIGHTS)
        assert th.size == N_PARAMS
        return th, "trained (" + os.path.relpath(WEIGHTS, ROOT) + ")"
    return I.gnn_init(0, out_scale=0.02).astype(np.float32), "random init (seed 0, last layer x0.02)"


def gnn_policy():
    """The shipped weights' validation record and fallback decision."""
    from paper_2412_07127_gb300.train import load_weights
    if not os.path.exists(WEIGHTS):
        return None
    _, meta = load_weights(WEIGHTS)
    if not meta:
        return None
    v = meta["validation"]
    return {"use_gnn": meta["use_gnn"], "validation_iters_ic0": v["iters_ic0_mean"],
            "validation_iters_gnn": v["iters_gnn_mean"], "validation": v["systems"]}


def workload_sizes(N):
    from paper_2412_07127_gb300 import inputs as I
    n, nnz, nnzL, lev = I.fem_sizes(N)
    return n, nnz, nnzL, lev


def kernel_bytes(N, ldtype):
    """Algorithmic bytes per launch of each kernel class:
    factor values + int32 columns once, row pointers, the vectors read and
    written once. FP32 apply: 4-byte factor values and vectors."""
    n, nnz, nnzL, _ = workload_sizes(N)
    lv = 8 if ldtype == "f64" else 4
    vb = 8 if ldtype == "f64" else 4
    return {
        "spmv": 12 * nnz + 4 * (n + 1) + 16 * n,
        "lsolve": (lv + 4) * nnzL + 4 * (n + 1) + 2 * vb * n,
        "ltsolve": (lv + 4) * nnzL + 4 * (n + 1) + 2 * vb * n + 8 * n,
        "vector": 40 * n,  # mean of the two vector kernels (32n and 48n)
    }


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        import statistics
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if its kernel
    source hash still matches (else null)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kernel)
    if not ent:
        return None
    src = os.path.join(ROOT, "paper_2412_07127_gb300", "csrc", ent["source"])
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if h != ent.get("source_sha"):
        return None
    return ent.get("bytes_per_launch_full")


# ---------------------------------------------------------------- oracle timing
def oracle_solve_seconds(N, seed, theta64):
    """One GNN-IC solve on the CPU oracle (single thread): IC(0), features,
    correction and the full PCG on the N^3 system; the GNN forward timed on
    the 20^3 system of the same recipe and scaled by edge count. The PCG runs
    with the IC(0) factor. Returns (seconds, detail)."""
    import numpy as np
    import oracle as O
    from paper_2412_07127_gb300 import inputs as I
    E = I.material_field(N, seed)
    b = I.rhs(3 * N * (N + 1) ** 2, seed)
    A = O.fem_hex_assemble(N, E)
    T = O.lower(A)
    t0 = time.perf_counter()
    L, alpha, bad = O.ic0_auto(A)
    t1 = time.perf_counter()
    x9, e0, s = O.features(A)
    t2 = time.perf_counter()
    Ns = min(N, 20)
    As = O.fem_hex_assemble(Ns, I.material_field(Ns, seed))
    Ts = O.lower(As)
    sx9, se0, _ = O.features(As)
    t3 = time.perf_counter()
    O.gnn_forward(Ts, sx9, se0, theta64)
    t4 = time.perf_counter()
    gnn_scaled = (t4 - t3) * (T.nnz / Ts.nnz)
    t5 = time.perf_counter()
    O.correct(T, L.val, np.zeros(T.nnz))
    t6 = time.perf_counter()
    r = O.pcg(A, b, L, tol=1e-8)
    t7 = time.perf_counter()
    total = (t1 - t0) + (t2 - t1) + gnn_scaled + (t6 - t5) + (t7 - t6)
    cpu_work = (t1 - t0) + (t2 - t1) + (t4 - t3) + (t6 - t5) + (t7 - t6)
    return total, dict(ic0_s=t1 - t0, features_s=t2 - t1, gnn_s_scaled=gnn_scaled, gnn_s_20=t4 - t3,
                       pcg_s=t7 - t6, iters=r["iters"], cpu_work_s=cpu_work)


def run_reference(args, rank, world):
    import numpy as np
    from paper_2412_07127_gb300 import inputs as I
    if rank != 0:
        return
    theta, theta_src = load_theta(I.N_PARAMS)
    th64 = theta.astype(np.float64)
    for _ in range(args.warmup):
        oracle_solve_seconds(args.N, args.seed, th64)
    vals, det = [], None
    for _ in range(args.steps):
        v, det = oracle_solve_seconds(args.N, args.seed, th64)
        vals.append(v)
    val = float(np.mean(vals))
    sample = (f"CPU oracle, 1 thread: IC(0), features, correction, full PCG on the {args.N}^3 system; "
              f"GNN forward timed on 20^3 and scaled by edge count ({det['cpu_work_s']:.1f} s CPU work per step)")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(args.N, theta_src, args.ldtype),
           "iters": det["iters"],
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": val, "unit": "s"},
           "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- GPU arm
def run_ours(args, rank, world, local):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2412_07127_gb300 import build, gicpcg as G
    from paper_2412_07127_gb300 import inputs as I

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    stream = torch.cuda.current_stream()
    h = G.Handle(local, stream)
    N = args.N
    seed = rank_seed(args.seed, rank)
    theta_np, theta_src = load_theta(I.N_PARAMS)
    theta = torch.from_numpy(theta_np).to(dev)
    ldt = G.GIC_F64 if args.ldtype == "f64" else G.GIC_F32

    E = torch.from_numpy(I.material_field(N, seed)).to(dev)
    b_np = I.rhs(3 * N * (N + 1) ** 2, seed)
    b = torch.from_numpy(b_np).to(dev)
    rowptr, col, valA = G.fem_hex_assemble(h, N, E)
    P = G.Pattern(h, rowptr, col)
    ws_pcg = G.workspace(h, P, G.GIC_WS_PCG, ldt)
    ws_gnn = G.gnn_workspace(h, P, 1, training=False)
    LIC = torch.empty(P.nnzL, dtype=torch.float64, device=dev)
    Lg = torch.empty_like(LIC)
    g = torch.empty(P.nnzL, dtype=torch.float32, device=dev)
    x = torch.empty_like(b)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    ws_pcg32 = G.workspace(h, P, G.GIC_WS_PCG, G.GIC_F32)

    def step(ldt_run):
        """IC(0), features + GNN + correction, PCG with the corrected factor,
        PCG with the plain IC(0) factor; factor precision ldt_run."""
        e = [ev() for _ in range(6)]
        wsp = ws_pcg if ldt_run == G.GIC_F64 else ws_pcg32
        e[0].record(stream)
        _, alpha, bad = G.ic0_auto(h, P, valA, out=LIC)
        e[1].record(stream)
        x9, e0, scale, _ = G.features(h, P, valA)
        G.gnn_forward(h, P, theta, x9, e0, ws=ws_gnn, g=g)
        _, ok = G.gnn_correct(h, P, LIC, g, scale, out=Lg)
        Luse = Lg if ok else LIC
        Lrun = Luse if ldt_run == G.GIC_F64 else G.to_f32(h, Luse)
        e[2].record(stream)
        x.zero_()
        r_g = G.pcg(h, P, valA, Lrun, b, x=x, ws=wsp)
        e[3].record(stream)
        L0 = LIC if ldt_run == G.GIC_F64 else G.to_f32(h, LIC)
        x.zero_()
        e[4].record(stream)
        r_i = G.pcg(h, P, valA, L0, b, x=x, ws=wsp)
        e[5].record(stream)
        return e, r_g, r_i, ok, alpha

    def phases(recs):
        ph = np.array([[r[0][k].elapsed_time(r[0][k + 1]) for k in range(5)] for r in recs]) / 1e3
        return ph.mean(0)

    for _ in range(args.warmup):
        step(ldt)
    sync_all(world, dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = G.launch_count(h)
    t_start, t_end = ev(), ev()
    torch.cuda.synchronize()
    t_start.record(stream)
    recs = [step(ldt) for _ in range(args.steps)]
    t_end.record(stream)
    sync_all(world, dev)
    launches = G.launch_count(h) - launches0
    clk = clocks.stop()
    # per-kernel times: the same steps once more with the library's CUDA
    # events around every launch (they add about 3.5% to a PCG, so the timed
    # steps above run without them)
    G.profile_enable(h, True)
    for _ in range(args.steps):
        step(ldt)
    torch.cuda.synchronize()
    prof = G.profile_read(h)
    G.profile_enable(h, False)
    total_ms = t_start.elapsed_time(t_end)
    ic0_s, gnn_s, cg_g_s, _, cg_i_s = phases(recs)
    value = ic0_s + gnn_s + cg_g_s
    total_ms, value = max_over_ranks([total_ms, value], world, dev)
    r_g, r_i = recs[-1][1], recs[-1][2]

    # the same steps with the FP32 preconditioner apply (FP64 CG), after the
    # timed region, with their own per-kernel profile
    other = None
    if args.ldtype == "f64" and not args.no_f32:
        for _ in range(2):
            step(G.GIC_F32)
        torch.cuda.synchronize()
        recs32 = [step(G.GIC_F32) for _ in range(args.steps)]
        torch.cuda.synchronize()
        G.profile_enable(h, True)
        for _ in range(args.steps):
            step(G.GIC_F32)
        torch.cuda.synchronize()
        prof32 = G.profile_read(h)
        G.profile_enable(h, False)
        a, b_, c, _, d = phases(recs32)
        kb32 = kernel_bytes(N, "f32")
        other = {"value_s": a + b_ + c, "phase_s": {"ic0": a, "features_gnn_correct": b_, "cg_gnn_ic": c, "cg_ic0": d,
                                                    "ic0_pcg_total": a + d},
                 "iters": {"gnn_ic": recs32[-1][1]["iters"], "ic0": recs32[-1][2]["iters"]},
                 "relres": {"gnn_ic": recs32[-1][1]["relres"], "ic0": recs32[-1][2]["relres"]},
                 "kernels": {k: {"launches": v["launches"], "avg_us": v["ms"] / v["launches"] * 1e3,
                                 "GB_s": kb32[k] / (v["ms"] / v["launches"] / 1e3) / 1e9}
                             for k, v in prof32.items() if v["launches"]}}

    # kernel classes: achieved GB/s from algorithmic bytes / mean launch time
    kb = kernel_bytes(N, args.ldtype)
    kern = {}
    for k, d in prof.items():
        if d["launches"]:
            avg = d["ms"] / d["launches"] / 1e3
            kern[k] = {"launches": d["launches"], "avg_us": avg * 1e6, "total_ms": d["ms"],
                       "GB_s": kb[k] / avg / 1e9}
    peak, peak_src = measured_peaks()
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    ach = kern[dom]["GB_s"]
    roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak, "peak_source": peak_src,
            "traffic": ncu_traffic(dom), "algorithmic_bytes_per_launch": kb[dom]}
    spmv_roof = None
    if "spmv" in kern:
        spmv_roof = {"achieved": kern["spmv"]["GB_s"], "frac": kern["spmv"]["GB_s"] / peak}

    out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.ldtype == "f64" else "f64+f32L",
           "data": "synthetic",
           "config": workload_config(N, theta_src, args.ldtype),
           "iters": {"gnn_ic": r_g["iters"], "ic0": r_i["iters"]},
           "phase_s": {"ic0": ic0_s, "features_gnn_correct": gnn_s, "cg_gnn_ic": cg_g_s, "cg_ic0": cg_i_s,
                       "ic0_pcg_total": ic0_s + cg_i_s},
           "relres": {"gnn_ic": r_g["relres"], "ic0": r_i["relres"]},
           "gnn_kept": bool(recs[-1][3]), "ic0_shift": recs[-1][4], "gnn_policy": gnn_policy(),
           "kernels": kern, "kernel_timing": "CUDA events on the library's stream around every launch, in a "
           "second pass of the same steps (the timed steps run without them: they add about 3.5% to a PCG)",
           "roofline": roof, "spmv_roofline": spmv_roof, "clocks": clk,
           "gpu_launches": launches,
           "schedule": {"chunks": P.nchunks, "multi_group_chunks": bool(P.chunked), "chunk_order": P.chunked, "sell_padding":
                        P.sell_nnz / P.nnzA - 1.0},
           "f32_apply": other}

    if not args.no_e2e:
        # end to end through the C-ABI with host buffers (pinned)
        A_rp = rowptr.cpu().pin_memory()
        A_c = col.cpu().pin_memory()
        A_v = valA.cpu().pin_memory()
        b_h = torch.from_numpy(b_np).pin_memory()
        x_h = torch.zeros(P.n, dtype=torch.float64).pin_memory()
        th_h = torch.from_numpy(theta_np).pin_memory()
        ws_h = G.solve_host_workspace(h, P.n, P.nnzA, True, ldt, device=local)
        rp_np, c_np, v_np, b_hn, x_hn, th_hn = (t.numpy() for t in (A_rp, A_c, A_v, b_h, x_h, th_h))
        G.solve_host(h, rp_np, c_np, v_np, b_hn, theta=th_hn, l_dtype=ldt, ws=ws_h, x=x_hn)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            re = G.solve_host(h, rp_np, c_np, v_np, b_hn, theta=th_hn, l_dtype=ldt, ws=ws_h, x=x_hn)
            ts.append(time.perf_counter() - t0)
        e2e = float(np.mean(ts))
        e2e = max_over_ranks([e2e], world, dev)[0]
        out["e2e"] = {"value": e2e, "unit": "s",
                      "h2d_bytes_per_step": int(A_rp.numel() * 4 + A_c.numel() * 4 + A_v.numel() * 8
                                                + b_h.numel() * 8 + th_h.numel() * 4),
                      "d2h_bytes_per_step": int(x_h.numel() * 8), "iters": re["iters"],
                      "call": "gic_solve_host (analysis, IC(0), GNN, correction, PCG, copies)"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, det = oracle_solve_seconds(N, seed, theta_np.astype(np.float64))
        out["cpu_baseline"] = {"value": cv, "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": (f"1 thread: IC(0), features, correction and full PCG "
                                          f"({det['iters']} iters, IC(0) factor) on the {N}^3 system; GNN forward "
                                          f"timed on 20^3 and scaled by edge count; "
                                          f"{det['cpu_work_s']:.1f} s of CPU work"),
                               "detail": det}
    if world > 1:
        dist.barrier()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
