"""Benchmark: GNN-corrected IC(0)-PCG against plain IC(0)-PCG to a 1e-8
relative residual on the synthetic hex elasticity system of 148^3 elements
(9,857,244 dofs, 787.7M nonzeros) on one GB300. A, b, x and every CG vector
and scalar are FP64; the factor is applied in FP64 (the headline) and in FP32
(beside it).

A step is one pass of the method over the system already resident in HBM:
IC(0) factorisation, graph features, GNN forward, correction of L (Eq. 2)
and PCG with the corrected factor (Supplementary Algorithm 1). `value` is
the mean seconds of that step. After the timed steps, and outside them:
plain IC(0)-PCG (the method's fallback), both again with the FP32 factor,
one more step with CUDA events around every launch (per-kernel times and the
roofline), `e2e` (the same solve through gic_solve_host: A and b copied from
pinned host memory, x copied back) and the CPU oracle timed on a bounded
sample of the same system (`cpu_baseline`).

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
    ap.add_argument("--N", type=int, default=148)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--ldtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-f32", action="store_true", help="skip the FP32-apply comparison")
    ap.add_argument("--mixed-N", type=int, default=69,
                    help="size of the mixed-precision side measurement (FP32 factor apply with the GNN "
                         "correction and IC(0) fallback against all-FP64 plain IC(0)-PCG); 0 skips it")
    ap.add_argument("--side-steps", type=int, default=2,
                    help="steps of each comparison run after the timed region")
    ap.add_argument("--pipeline", type=int, default=4,
                    help="triangular-solve kernels (GIC_TUNE_PIPELINE): 4 automatic, 3 level-sliced, "
                         "2 warp-specialised, 1 staged, 0 generic")
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
    """Algorithmic bytes per launch of each kernel class: the CSR of A or L
    read once (8- or 4-byte values and int32 columns, int32 row pointers) and
    the vectors read and written once (the backward sweep also reads r for
    the fused r^T z). FP32 apply: 4-byte factor values and solve vectors."""
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


def ncu_traffic(kernel, N, ldtype):
    """DRAM bytes per launch at this workload from the committed ncu summary,
    if its entry is for this kernel class, size and factor precision and the
    captured kernel's source is unchanged (else null)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    ent = json.load(open(p)).get(f"{kernel}/{ldtype}")
    if not ent or ent.get("N") != N:
        return None
    src = os.path.join(ROOT, "paper_2412_07127_gb300", "csrc", ent["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != ent.get("source_sha"):
        return None
    return ent.get("bytes_per_launch")


# ---------------------------------------------------------------- oracle timing
def host_cpu():
    """CPU model and core count of this host (for the baseline lines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


def principal_block(A, idx):
    """Rows and columns idx (sorted) of a CSR matrix: a principal submatrix."""
    import numpy as np
    import oracle as O
    pos = np.full(A.n, -1, np.int64)
    pos[idx] = np.arange(idx.size)
    starts, ends = A.rowptr[idx].astype(np.int64), A.rowptr[idx + 1].astype(np.int64)
    sel = np.concatenate([np.arange(a, e) for a, e in zip(starts, ends)])
    row = np.repeat(np.arange(idx.size), ends - starts)
    keep = pos[A.col[sel]] >= 0
    sel, row = sel[keep], row[keep]
    rp = np.zeros(idx.size + 1, np.int32)
    rp[1:] = np.cumsum(np.bincount(row, minlength=idx.size))
    return O.CSR(rp, pos[A.col[sel]].astype(np.int32), A.val[sel].copy())


def oracle_sample(N, seed, theta64, yrows, planes=3, pcg_iters=10, spmv_reps=5):
    """The CPU oracle on a bounded sample of the N^3 system: its principal
    block of the dofs of the nodes (x, y < yrows, z) of `planes` free node
    planes in the middle of the cube (all x). The cube's element layers from
    one below the first of those planes to the last hold every element that
    touches them, and a slab of just those layers, clamped at its bottom,
    numbers the nodes of its first `planes` planes as the block's rows in
    order; so the block is exactly the cube's. Times, single-threaded, IC(0),
    features, GNN forward and correction on the block, `pcg_iters` PCG
    iterations with the corrected factor, and one SpMV on one core and on
    all cores (OpenMP)."""
    import numpy as np
    import oracle as O
    from paper_2412_07127_gb300 import inputs as I
    E = I.material_field(N, seed)
    z1 = max(1, N // 2 - planes // 2)
    layers = E.reshape(N, N, N)[z1 - 1: z1 + planes].ravel()
    S = O.fem_box_assemble(N, N, planes + 1, 1.0 / N, layers)
    nodes = np.array([x + (N + 1) * (y + (N + 1) * z) for z in range(planes) for y in range(min(yrows, N + 1))
                      for x in range(N + 1)], np.int64)
    idx = (3 * nodes[:, None] + np.arange(3)[None, :]).ravel()
    B = principal_block(S, idx)
    k = B.n
    b = I.rhs(3 * N * (N + 1) ** 2, seed)[:k]
    T = O.lower(B)
    x = np.random.default_rng(1).standard_normal(k)
    O.spmv_threads(B, x)  # starts the thread pool
    t0 = time.perf_counter()
    L, alpha, bad = O.ic0_auto(B)
    t1 = time.perf_counter()
    x9, e0, sc = O.features(B)
    t2 = time.perf_counter()
    g = O.gnn_forward(T, x9, e0, theta64)
    t3 = time.perf_counter()
    Lc = O.correct(T, L.val, g * np.sqrt(sc))
    t4 = time.perf_counter()
    O.pcg(B, b, O.CSR(T.rowptr, T.col, Lc), tol=0.0, maxit=pcg_iters)  # runs all pcg_iters iterations
    t5 = time.perf_counter()
    for _ in range(spmv_reps):
        O.spmv(B, x)
    t6 = time.perf_counter()
    for _ in range(spmv_reps):
        O.spmv_threads(B, x)
    t7 = time.perf_counter()
    return dict(ic0_s=t1 - t0, features_s=t2 - t1, gnn_s=t3 - t2, correct_s=t4 - t3,
                pcg_iter_s=(t5 - t4) / pcg_iters, spmv_1_s=(t6 - t5) / spmv_reps,
                spmv_all_s=(t7 - t6) / spmv_reps, rows=k, nnzA=int(B.nnz), nnzL=int(T.nnz), work_s=t7 - t0,
                block=f"dofs of nodes (x, y < {min(yrows, N + 1)}, z) of free planes z = {z1}..{z1 + planes - 1}")


def oracle_estimate(N, smp, iters):
    """Seconds of the oracle's full GNN-IC solve of the N^3 system from a
    sample: the factor phases scale with nnz(L) (features with nnz(A)), a
    PCG iteration with nnz(A) (SpMV, two triangular solves over nnz(L) =
    (nnz(A) + n) / 2, vector updates), times the solve's iteration count.
    The all-core figure runs the SpMV on every core (OpenMP); IC(0), the
    GNN and the triangular solves stay sequential."""
    n, nnz, nnzL, _ = workload_sizes(N)
    fA, fL = nnz / smp["nnzA"], nnzL / smp["nnzL"]
    setup = (smp["ic0_s"] + smp["gnn_s"] + smp["correct_s"]) * fL + smp["features_s"] * fA
    it1 = smp["pcg_iter_s"] * fA
    itall = (smp["pcg_iter_s"] - smp["spmv_1_s"] + smp["spmv_all_s"]) * fA
    return setup + it1 * iters, setup + itall * iters, {"setup_s": setup, "pcg_iter_s_1core": it1,
                                                        "pcg_iter_s_allcores": itall}


def golden_iters(N):
    """The oracle's own IC(0)-PCG iteration count for the seed-0 N^3 system,
    if the stored oracle result exists (tests/golden, written by the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", f"pcg_hex{N}_seed0.json")
    if not os.path.exists(p):
        return None
    return json.load(open(p))["f64"]["iters"]


def run_reference(args, rank, world):
    """The base contract's reference arm: the CPU oracle, timed on the host
    cores, on a bounded sample of the workload per step (rank 0 only)."""
    import numpy as np
    from paper_2412_07127_gb300 import inputs as I
    if rank != 0:
        return
    theta, theta_src = load_theta(I.N_PARAMS)
    th64 = theta.astype(np.float64)
    N = args.N
    yrows = 12  # about 2 s of oracle work per step at 148^3
    iters = golden_iters(N)
    iters_src = "oracle's own IC(0)-PCG count (tests/golden)"
    if iters is None:
        iters, iters_src = 4 * N + 30, "4N + 30 (no stored oracle count for this size)"
    for _ in range(args.warmup):
        oracle_sample(N, args.seed, th64, yrows, pcg_iters=5, spmv_reps=2)
    vals, vall, ts = [], [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        smp = oracle_sample(N, args.seed, th64, yrows, pcg_iters=5, spmv_reps=2)
        ts.append(time.perf_counter() - t0)
        v1, va, det = oracle_estimate(N, smp, iters)
        vals.append(v1)
        vall.append(va)
    import oracle as O
    val = float(np.mean(vals))
    sample = (f"principal block of the {N}^3 system, {smp['block']} ({smp['rows']} rows, {smp['nnzA']} nnz): "
              f"IC(0), features, GNN forward, correction, 5 PCG iterations per step on one core; scaled to the "
              f"full system by nnz and to {iters} iterations ({iters_src})")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(ts)) * 1e3,
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": workload_config(N, theta_src, "f64"),
           "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": sample, "value": val, "unit": "s",
                            "allcores_spmv_value": float(np.mean(vall)), "allcores_threads": O.threads(),
                            "host": host_cpu(), "detail": det},
           "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- GPU arm
def mixed_precision(G, I, h, dev, stream, N, seed, theta, steps, pol):
    """The mixed-precision comparison at N^3 (about 1M dofs at 69^3), after
    the headline's timed steps: FP64 CG vectors and scalars with the factor
    applied in FP32, the GNN correction with the IC(0) fallback, against
    all-FP64 plain IC(0)-PCG on the same system. Each path is timed with CUDA
    events over `steps` runs after one untimed run."""
    import numpy as np
    import torch
    E = torch.from_numpy(I.material_field(N, seed)).to(dev)
    b = torch.from_numpy(I.rhs(3 * N * (N + 1) ** 2, seed)).to(dev)
    rp, c, v = G.fem_hex_assemble(h, N, E)
    P = G.Pattern(h, rp, c)
    ws = {d: G.workspace(h, P, G.GIC_WS_PCG, d) for d in (G.GIC_F64, G.GIC_F32)}
    wsg = G.gnn_workspace(h, P, 1, training=False)
    L = torch.empty(P.nnzL, dtype=torch.float64, device=dev)
    Lg = torch.empty_like(L)
    g = torch.empty(P.nnzL, dtype=torch.float32, device=dev)
    x = torch.empty_like(b)

    def run(path):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        G.ic0_auto(h, P, v, out=L)
        Lr, ldt, ok = L, G.GIC_F64, True
        if path == "gnn_ic_f32L":
            x9, e0_, scale, _ = G.features(h, P, v)
            G.gnn_forward(h, P, theta, x9, e0_, ws=wsg, g=g)
            _, ok = G.gnn_correct(h, P, L, g, scale, out=Lg)
            Lr = Lg if ok else L
        if path != "ic0_f64":
            Lr, ldt = G.to_f32(h, Lr), G.GIC_F32
        x.zero_()
        r = G.pcg(h, P, v, Lr, b, x=x, ws=ws[ldt])
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3, r, ok

    res = {}
    for path in ("gnn_ic_f32L", "ic0_f32L", "ic0_f64"):
        run(path)
        runs = [run(path) for _ in range(steps)]
        res[path] = {"value_s": float(np.mean([t for t, _, _ in runs])), "iters": runs[-1][1]["iters"],
                     "relres": runs[-1][1]["relres"]}
        if path == "gnn_ic_f32L":
            res[path]["gnn_kept"] = bool(runs[-1][2])
    chosen = "gnn_ic_f32L" if (pol and pol["use_gnn"]) else "ic0_f32L"
    out = {"workload": f"hex elasticity {N}^3 elements ({P.n} dofs, {P.nnzA} nnz), same generator and seed",
           "paths": res, "chosen": chosen,
           "speedup_vs_f64_ic0": res["ic0_f64"]["value_s"] / res[chosen]["value_s"],
           "iters_vs_f64_ic0": res[chosen]["iters"] / res["ic0_f64"]["iters"] - 1.0,
           "solve_kernels": {"f64": G.solve_kernels_chosen(h, P, G.GIC_F64),
                             "f32": G.solve_kernels_chosen(h, P, G.GIC_F32)},
           "steps": steps}
    del ws, wsg, P
    return out


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
    G.set_tuning(h, G.GIC_TUNE_PIPELINE, args.pipeline)
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
    ws = {d: G.workspace(h, P, G.GIC_WS_PCG, d) for d in (G.GIC_F64, G.GIC_F32)}
    ws_gnn = G.gnn_workspace(h, P, 1, training=False)
    LIC = torch.empty(P.nnzL, dtype=torch.float64, device=dev)
    Lg = torch.empty_like(LIC)
    g = torch.empty(P.nnzL, dtype=torch.float32, device=dev)
    x = torch.empty_like(b)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step_gnn(ldt_run):
        """One pass of the method: IC(0), features, GNN, correction (Eq. 2),
        PCG with the corrected factor in precision ldt_run."""
        e = [ev() for _ in range(4)]
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
        r = G.pcg(h, P, valA, Lrun, b, x=x, ws=ws[ldt_run])
        e[3].record(stream)
        return e, r, ok, alpha

    def step_ic0(ldt_run):
        """The fallback: IC(0), PCG with the plain factor."""
        e = [ev() for _ in range(3)]
        e[0].record(stream)
        G.ic0_auto(h, P, valA, out=LIC)
        Lrun = LIC if ldt_run == G.GIC_F64 else G.to_f32(h, LIC)
        e[1].record(stream)
        x.zero_()
        r = G.pcg(h, P, valA, Lrun, b, x=x, ws=ws[ldt_run])
        e[2].record(stream)
        return e, r

    def secs(recs, k0, k1):
        return float(np.mean([r[0][k0].elapsed_time(r[0][k1]) for r in recs])) / 1e3

    for _ in range(args.warmup):
        step_gnn(ldt)
    sync_all(world, dev)
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = G.launch_count(h)
    t_start, t_end = ev(), ev()
    t_start.record(stream)
    recs = [step_gnn(ldt) for _ in range(args.steps)]
    t_end.record(stream)
    sync_all(world, dev)
    launches = G.launch_count(h) - launches0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    ic0_s, gnn_s, cg_s, value = secs(recs, 0, 1), secs(recs, 1, 2), secs(recs, 2, 3), secs(recs, 0, 3)
    total_ms, value = max_over_ranks([total_ms, value], world, dev)
    r_g = recs[-1][1]

    # after the timed region: the fallback, the other factor precision, and
    # one step with per-kernel CUDA events
    K2 = max(1, args.side_steps)
    rec0 = [step_ic0(ldt) for _ in range(K2)]
    torch.cuda.synchronize()
    r_i = rec0[-1][1]
    G.profile_enable(h, True)
    step_gnn(ldt)
    torch.cuda.synchronize()
    prof = G.profile_read(h)
    G.profile_enable(h, False)
    other = None
    if args.ldtype == "f64" and not args.no_f32:
        recs32 = [step_gnn(G.GIC_F32) for _ in range(K2)]
        rec032 = [step_ic0(G.GIC_F32) for _ in range(K2)]
        G.profile_enable(h, True)
        step_gnn(G.GIC_F32)
        torch.cuda.synchronize()
        prof32 = G.profile_read(h)
        G.profile_enable(h, False)
        kb32 = kernel_bytes(N, "f32")
        it32, it0_32 = recs32[-1][1]["iters"], rec032[-1][1]["iters"]
        other = {"value_s": secs(recs32, 0, 3),
                 "phase_s": {"ic0": secs(recs32, 0, 1), "features_gnn_correct": secs(recs32, 1, 2),
                             "cg_gnn_ic": secs(recs32, 2, 3), "ic0_path_total": secs(rec032, 0, 2)},
                 "iters": {"gnn_ic": it32, "ic0": it0_32},
                 "iters_vs_f64": {"gnn_ic": it32 / r_g["iters"] - 1.0, "ic0": it0_32 / r_i["iters"] - 1.0},
                 "relres": {"gnn_ic": recs32[-1][1]["relres"], "ic0": rec032[-1][1]["relres"]},
                 "kernels": {k: {"launches": v["launches"], "avg_us": v["ms"] / v["launches"] * 1e3,
                                 "GB_s": kb32[k] / (v["ms"] / v["launches"] / 1e3) / 1e9}
                             for k, v in prof32.items() if v["launches"]},
                 "steps": K2}

    # kernel classes: achieved GB/s = algorithmic bytes / mean launch time
    kb = kernel_bytes(N, args.ldtype)
    kern = {}
    for k, d in prof.items():
        if d["launches"]:
            avg = d["ms"] / d["launches"] / 1e3
            kern[k] = {"launches": d["launches"], "avg_us": avg * 1e6, "total_ms": d["ms"], "GB_s": kb[k] / avg / 1e9}
    peak, peak_src = measured_peaks()
    dom = max(kern, key=lambda k: kern[k]["total_ms"])
    ach = kern[dom]["GB_s"]
    roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": peak_src, "traffic": ncu_traffic(dom, N, args.ldtype),
            "algorithmic_bytes_per_launch": kb[dom]}
    spmv_roof = None
    if "spmv" in kern:
        spmv_roof = {"achieved": kern["spmv"]["GB_s"], "frac": kern["spmv"]["GB_s"] / peak,
                     "traffic": ncu_traffic("spmv", N, args.ldtype)}
    pol = gnn_policy()
    cuts = r_g["iters"] < r_i["iters"]
    out = {"metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.ldtype == "f64" else "f64+f32L",
           "data": "synthetic",
           "config": workload_config(N, theta_src, args.ldtype),
           "iters": {"gnn_ic": r_g["iters"], "ic0": r_i["iters"]},
           "phase_s": {"ic0": ic0_s, "features_gnn_correct": gnn_s, "cg_gnn_ic": cg_s,
                       "ic0_path_total": secs(rec0, 0, 2), "cg_ic0": secs(rec0, 1, 2)},
           "relres": {"gnn_ic": r_g["relres"], "ic0": r_i["relres"]},
           "gnn_kept": bool(recs[-1][2]), "ic0_shift": recs[-1][3],
           "gnn_cuts_iterations": cuts,
           "policy": {"validation": pol, "chosen": ("gnn_ic" if pol and pol["use_gnn"] else "ic0"),
                      "chosen_value_s": value if (pol and pol["use_gnn"]) else secs(rec0, 0, 2)},
           "side_steps": K2,
           "kernels": kern, "kernel_timing": "CUDA events on the library's stream around every launch, in one "
           "more step after the timed ones (the timed steps run without them)",
           "roofline": roof, "spmv_roofline": spmv_roof, "clocks": clk,
           "gpu_launches": launches,
           "schedule": {"chunks": P.nchunks, "level_sliced": bool(P.level_sliced), "slices": P.slices,
                        "solve_kernels": G.solve_kernels_chosen(h, P, ldt),
                        "spmv": "3x3 node blocks" if P.node_blocks else "SELL-32",
                        "spmv_padding": P.spmv_entries / P.nnzA - 1.0},
           "f32_apply": other}

    if args.mixed_N > 0 and args.mixed_N != N:
        out["mixed_precision"] = mixed_precision(G, I, h, dev, stream, args.mixed_N, seed, theta,
                                                 max(1, args.side_steps), gnn_policy())

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
        for _ in range(K2):
            t0 = time.perf_counter()
            re = G.solve_host(h, rp_np, c_np, v_np, b_hn, theta=th_hn, l_dtype=ldt, ws=ws_h, x=x_hn)
            ts.append(time.perf_counter() - t0)
        e2e = float(np.mean(ts))
        e2e = max_over_ranks([e2e], world, dev)[0]
        out["e2e"] = {"value": e2e, "unit": "s",
                      "h2d_bytes_per_step": int(A_rp.numel() * 4 + A_c.numel() * 4 + A_v.numel() * 8
                                                + b_h.numel() * 8 + th_h.numel() * 4),
                      "d2h_bytes_per_step": int(x_h.numel() * 8), "iters": re["iters"], "steps": K2,
                      "call": "gic_solve_host (analysis, IC(0), GNN, correction, PCG, copies)"}
        del ws_h

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(N, seed, theta_np.astype(np.float64), 100)
        v1, vall, det = oracle_estimate(N, smp, r_g["iters"])
        import oracle as O
        out["cpu_baseline"] = {
            "value": v1, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": (f"principal block of the {N}^3 system, {smp['block']} ({smp['rows']} rows, {smp['nnzA']} "
                       f"nnz): IC(0), features, GNN forward, correction and 10 PCG iterations on one core, "
                       f"{smp['work_s']:.1f} s of CPU work; scaled to the full system by nnz and to this run's "
                       f"{r_g['iters']} GNN-IC iterations"),
            "allcores_spmv_value": vall, "allcores_threads": O.threads(), "host": host_cpu(),
            "detail": {**det, **{k: smp[k] for k in ("ic0_s", "features_s", "gnn_s", "correct_s", "pcg_iter_s",
                                                     "spmv_1_s", "spmv_all_s")}}}
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
