"""Benchmark of the FMM poroelastic DDM hot path on GB300.

Workload: randomly distributed pressurised fractures, 200 non-intersecting
cracks (seeded rejection sampling) in a 200 m x 200 m box, lengths U[2, 10] m,
orientations U[0, pi), 100 constant elements each: N = 20,000 elements,
60,000 unknowns.  G = 6 GPa, nu = 0.2, nu_u = 0.33, B = 0.8, k = 1e-18 m^2,
mu = 1e-3 Pa s; fracture pressure 10 MPa, sigma_H = 30 MPa, sigma_h = 25 MPa;
one time element of 10 s.  FMM with n = 8 Chebyshev nodes per dimension,
leaf size 32, FP32 pair/M2L arithmetic, FP64 Krylov.

A timed step is one FMM influence product y = [K(dt)] x over all N elements
(inputs resident in HBM; L2 flushed between steps); value = N / step time in
Melem/s.  The same run also reports the full time-step solve (tree build,
right-hand side, GMRES to 1e-5, SIFs) as solves/s with p50/p99 latency, the
dense on-the-fly product (conventional PDDM on the GPU), the error of the
FMM product against the FP64 CPU oracle on sampled rows, the roofline of
the dominant kernel and the oracle timed on the host cores.

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload (the method has no reference implementation to install).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM matvec Melem/s & solves/s vs dense GPU DDM at <=1e-3 rel err; p50/p99"
WORKLOAD = "random pressurised fractures: 200 cracks x 100 elements (N=20000), dt=10 s"
DT = 10.0
LOADS = dict(sigma_H=30e6, sigma_h=25e6, p_f=10e6, p0=0.0)
STAGE_KERNEL = {"leaf": "k_near2", "m2l": "k_m2l_tc", "up": "k_up", "down": "k_down"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n-cheb", type=int, default=8)
    ap.add_argument("--leaf", type=int, default=32)
    ap.add_argument("--solves", type=int, default=100)
    ap.add_argument("--orders", default="12,16", help="extra Chebyshev orders timed beside --n-cheb ('' = none)")
    ap.add_argument("--m2l", default="compressed", choices=["compressed", "full"],
                    help="M2L operators of the headline product and solves")
    ap.add_argument("--adaptive", type=int, default=1, help="time the adaptive and the uniform tree on the "
                    "clustered set (0 = skip)")
    ap.add_argument("--well-steps", type=int, default=100, help="time steps of the horizontal-well march (0 = skip)")
    ap.add_argument("--well-tol", type=float, default=3e-4, help="GMRES tolerance of the horizontal-well march "
                    "(its FP32 floor: 1.5e-5 at the first step, ~1.4e-4 from step ~40)")
    ap.add_argument("--oracle-rows", type=int, default=12)
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--hist-lags", type=int, default=10)
    ap.add_argument("--batch-problems", type=int, default=512)
    ap.add_argument("--batch-dense", type=int, default=1, help="time the dense GPU arm of the batch (step 1)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-nmax", type=int, default=200000)
    ap.add_argument("--serve-max-steps", type=int, default=100)
    ap.add_argument("--serve-dense-seconds", type=float, default=30.0,
                    help="window of the dense-DDM arm on the same request stream")
    ap.add_argument("--serve-rate", type=float, default=50.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def ncu_record():
    """DRAM traffic / flop counts from the committed ncu capture, valid only
    while the kernel sources are unchanged."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except Exception:
        return None, False
    csrc = os.path.join(ROOT, "paper_1812_05087_gb300", "csrc")
    ok = all(hashlib.sha1(open(os.path.join(csrc, f), "rb").read()).hexdigest() == h
             for f, h in rec["sources_sha1"].items())
    return rec, ok


def alu_peak_tflops(sm_mhz):
    """FP32 FMA peak: 152 SMs x 128 FP32 lanes x 2 flop x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def near_pair_flops(quad_near):
    """Algorithmic FP32 work of one element-integrated 4 x 3 kernel block
    (one near pair): ~150 flops for the elastic part plus ~60 per Gauss
    point of the transient part."""
    return 150 + 60 * quad_near


def well_march(ctx, tree, N, steps, half_length, torch, tol=3e-4):
    """Horizontal-well time march (paper Sec. 4/5): per step the history of
    all previous steps is subtracted from the right-hand side, then the RATE
    system is solved (x0 = previous solution).  Returns per-step (history
    ms, solve ms), the GMRES infos and the solutions (steps x 3N)."""
    from paper_1812_05087_gb300 import inputs
    hist = torch.zeros(steps, 3 * N, dtype=torch.float64, device="cuda")
    b0 = ctx.rhs(tree, system="rate", **inputs.WELL_LOADS)
    times = [inputs.WELL_DT * k for k in range(steps + 1)]
    x = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    x[2 * N:] = inputs.well_source(half_length)
    t_hist, t_solve, infos = [], [], []
    for h in range(1, steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b = b0.clone()
        if h > 1:
            ctx.history_apply(tree, hist[:h - 1], times[:h + 1], b)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        x, info = ctx.gmres_solve(tree, inputs.WELL_DT, b, x, system="rate", tol=tol, raise_on_notconv=False)
        hist[h - 1] = x
        torch.cuda.synchronize()
        t_hist.append(1e3 * (t1 - t0))
        t_solve.append(1e3 * (time.perf_counter() - t1))
        infos.append(info)
    return t_hist, t_solve, infos, hist


def oracle_sample(xy, x, rows_elems):
    import oracle
    mat = __import__("paper_1812_05087_gb300.inputs", fromlist=["x"]).material_tuple()
    N = xy.shape[1]
    rows = np.concatenate([rows_elems + b * N for b in range(3)])
    t0 = time.perf_counter()
    A = oracle.assemble_rows(mat, xy, DT, rows)
    dt = time.perf_counter() - t0
    return A @ x, rows, dt


def replica_seed(rank):
    """Seed of rank's own fracture set: the path shards only across
    independent problems (replicas, no data-path collective)."""
    from paper_1812_05087_gb300 import inputs
    return inputs.SEED + rank


def max_over_ranks(dist, vals, device):
    """Element-wise maximum of per-rank timings over all ranks (identity
    without a process group); device is where the collective's tensor lives
    ("cuda" for NCCL, "cpu" for gloo)."""
    if dist is None:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def whole_job_melem_s(world, n_per_rank, ms):
    """Elements of all ranks' products per second (Melem/s) at the slowest
    rank's time per product."""
    return world * n_per_rank / (ms * 1e-3) / 1e6


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1812_05087_gb300 import inputs
    xy, _ = inputs.random_fractures()
    N = xy.shape[1]
    x = inputs.unknowns(N, seed=99)
    rng = np.random.default_rng(0)
    k = max(1, args.oracle_rows // 3)
    oracle.build()
    for _ in range(args.warmup):
        oracle_sample(xy, x, rng.choice(N, 1, replace=False))
    times = []
    for _ in range(args.steps):
        _, _, dt = oracle_sample(xy, x, rng.choice(N, k, replace=False))
        times.append(dt)
    per_elem = sum(times) / (k * args.steps)
    v = 1.0 / per_elem / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Melem/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_rows_per_step": 3 * k},
            "cpu_baseline": {"value": v, "unit": "Melem/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{k} target elements (3 rows each) x {N} source elements per step"},
            "e2e": {"value": v, "unit": "Melem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


BUCKETS = ((100, 300), (300, 1000), (1000, 3000), (3000, 10000), (10000, 20001))


def run_batched(args, inputs, Context, torch, loads):
    """Config-4 workload: 512 uneven random fracture sets.  A project-written
    autotuner (ddm_autotune) picks the Chebyshev order, leaf size and tree kind per size
    bucket on a representative problem; every problem's tree takes its
    bucket's choice; the time steps (1-10 per problem) run as lockstep
    batched GMRES solves of the problems still marching (history of each
    problem subtracted first).  Also: the same problems' first step with the
    dense GPU product (conventional DDM), and sampled problems against the
    FP64 oracle."""
    from paper_1812_05087_gb300.ddm import DDMError
    probs = inputs.batch_problems(args.batch_problems)
    bctx = Context(inputs.MATERIAL, n_cheb=args.n_cheb, leaf_size=args.leaf)
    # autotune: representative problem per bucket, its largest (the deepest
    # tree for a leaf size, so the far field that the choice must serve is
    # in the test; the smaller problems of the bucket carry more of their
    # product in the exact near field).  The product error bound is a fifth of the GMRES
    # tolerance (1e-5), else the tolerance itself: a product less accurate
    # than the tolerance leaves the exact residual that the escalated solver
    # measures above it.
    table = []
    t0 = time.perf_counter()
    for lo, hi in BUCKETS:
        cand = [pr for pr in probs if lo <= pr["xy"].shape[1] < hi]
        if not cand:
            continue
        rep = max(cand, key=lambda pr: pr["xy"].shape[1])
        n = rep["xy"].shape[1]
        best = None
        for bound in (2e-6, 1e-5):            # the tighter bound where some candidate meets it
            try:
                best = bctx.autotune(torch.as_tensor(rep["xy"], device="cuda"),
                                     torch.as_tensor(inputs.unknowns(n, seed=n), device="cuda"), DT,
                                     orders=[4, 6, 8, 10, 12], leaves=[16, 32, 64], max_rel_err=bound)
                best["bound"] = bound
                break
            except DDMError:
                continue
        if best is None:
            raise RuntimeError(f"autotune: no candidate within 1e-5 for bucket {lo}-{hi}")
        table.append({"bucket": [lo, hi], "sample_N": n, **best})
    t_tune = time.perf_counter() - t0

    def params(n):
        for row in table:
            if row["bucket"][0] <= n < row["bucket"][1]:
                return row["n_cheb"], row["leaf_size"], row["adaptive"]
        return args.n_cheb, args.leaf, False

    # problems sorted by their number of steps (descending): the problems still
    # marching at step k are a prefix, so every step's batch shares the arenas
    order = sorted(range(len(probs)), key=lambda i: -probs[i]["steps"])
    probs = [probs[i] for i in order]
    t0 = time.perf_counter()
    btrees = [bctx.build_tree(torch.as_tensor(pr["xy"], device="cuda"), *params(pr["xy"].shape[1])) for pr in probs]
    torch.cuda.synchronize()
    t_trees = time.perf_counter() - t0
    sizes = [t.n for t in btrees]
    off = np.concatenate([[0], np.cumsum([3 * n for n in sizes])])
    rhs0 = torch.cat([bctx.rhs(t, system="pressure", **loads) for t in btrees])
    smax = max(pr["steps"] for pr in probs)
    active = [sum(1 for pr in probs if pr["steps"] >= k) for k in range(1, smax + 1)]
    batches = [bctx.batch(btrees[:m]) for m in active]
    hist = torch.zeros(smax, int(off[-1]), dtype=torch.float64, device="cuda")
    x = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
    times = [DT * k for k in range(smax + 1)]

    def march():
        x.zero_()
        infos_all, solves = [], 0
        for k in range(1, smax + 1):
            m, L3 = active[k - 1], int(off[active[k - 1]])
            rhs = rhs0[:L3].clone()
            if k > 1:
                for i in range(m):
                    lo_, hi_ = int(off[i]), int(off[i + 1])
                    bctx.history_apply(btrees[i], hist[:k - 1, lo_:hi_].contiguous(), times[:k + 1], rhs[lo_:hi_])
            xs, infos = batches[k - 1].gmres_solve(DT, rhs, x[:L3], tol=1e-5, raise_on_notconv=False)
            hist[k - 1, :L3] = x[:L3]
            infos_all.append(infos)
            solves += m
        return infos_all, solves

    march()                                    # capture + warm (caches, graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    infos_all, solves = march()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    conv = sum(int(i["converged"]) for infos in infos_all for i in infos)
    # step 1 alone, for the dense comparison on the same problems
    full = batches[0]
    t0 = time.perf_counter()
    xf, inf_f = full.gmres_solve(DT, rhs0, torch.zeros_like(rhs0), tol=1e-5, raise_on_notconv=False)
    torch.cuda.synchronize()
    t_step1 = time.perf_counter() - t0
    dense_step1 = None
    if args.batch_dense:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xd, inf_d = full.gmres_solve(DT, rhs0, torch.zeros_like(rhs0), tol=1e-5, mode="dense",
                                     raise_on_notconv=False)
        torch.cuda.synchronize()
        t_d = time.perf_counter() - t0
        dense_step1 = {"solves_per_s": len(btrees) / t_d, "s": t_d,
                       "converged": int(sum(i["converged"] for i in inf_d))}
        d = (xf - xd).abs().cpu().numpy()
        ref = xd.abs().cpu().numpy()
        dense_step1["max_rel_diff_fmm_vs_dense"] = float(max(
            d[off[i]:off[i + 1]].max() / max(ref[off[i]:off[i + 1]].max(), 1e-300) for i in range(len(btrees))))
    # sampled problems against the FP64 oracle (direct solve of step 1)
    err = None
    if not args.no_oracle:
        import oracle
        mat = inputs.material_tuple()
        small = [i for i in range(len(probs)) if sizes[i] <= 400][:6]
        e = []
        xs1 = xf.cpu().numpy()
        for i in small:
            g = probs[i]["xy"]
            ref = oracle.solve(oracle.assemble(mat, g, DT), oracle.rhs(g, system="pressure", **loads), sizes[i])
            seg = xs1[off[i]:off[i + 1]]
            e.append(max(np.abs(seg[b * sizes[i]:(b + 1) * sizes[i]] - ref[b * sizes[i]:(b + 1) * sizes[i]]).max()
                         / max(np.abs(ref[b * sizes[i]:(b + 1) * sizes[i]]).max(), 1e-4 * np.abs(ref).max())
                         for b in range(3)))
        err = {"problems": len(small), "max_block_rel_err_vs_oracle": float(max(e)) if e else None}
    res = {"problems": len(btrees), "elements": int(sum(sizes)), "steps_total": solves,
           "autotune": table, "autotune_s": t_tune, "tree_build_s": t_trees,
           "march_s": t_batch, "batched_solves_per_s": solves / t_batch,
           "converged": conv, "step1_solves_per_s": len(btrees) / t_step1,
           "step1_converged": int(sum(i["converged"] for i in inf_f)),
           "max_iterations": int(max(i["iterations"] for infos in infos_all for i in infos)),
           "dense_step1": dense_step1, "error": err}
    for bt in batches:
        bt.close()
    for t in btrees:
        t.close()
    bctx.close()
    return res


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1812_05087_gb300 import inputs
    from paper_1812_05087_gb300.ddm import Context

    xy, segs = inputs.random_fractures(seed=replica_seed(rank))
    N = xy.shape[1]
    tips = inputs.tips_of(segs)
    stream = torch.cuda.current_stream()
    ctx = Context(inputs.MATERIAL, n_cheb=args.n_cheb, leaf_size=args.leaf)
    # M2L operators: SVD-compressed (mode 1, default rank) or the full ones
    ctx.set_m2l_compression(1 if args.m2l == "compressed" else 0)
    d_xy = torch.as_tensor(xy, dtype=torch.float64, device="cuda")
    tree = ctx.build_tree(d_xy)
    info = tree.info()
    x_h = inputs.unknowns(N, seed=99)
    x = torch.as_tensor(x_h, device="cuda")
    y = torch.empty_like(x)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, K, W):
        for _ in range(W):
            fn()
        barrier()
        ts = []
        for _ in range(K):
            flush.add_(1.0)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            ts.append((a, b))
        barrier()
        return [a.elapsed_time(b) for a, b in ts]

    # ---------------- FMM product (value)
    fmm = lambda: ctx.matvec(tree, x, 0.0, DT, mode="fmm", out=y)
    ctx.profile_read()
    with Clocks(local) as clk:
        t_fmm = timed(fmm, args.steps, args.warmup)
    launches = ctx.profile_read()
    n_launch_fmm = sum(v[1] for v in launches.values())
    per_matvec_launches = n_launch_fmm / (args.steps + args.warmup)
    # stage breakdown with events (separate pass)
    ctx.profile(True)
    for _ in range(3):
        fmm()
    stages = ctx.profile_read()
    ctx.profile(False)
    ms_fmm = float(np.mean(t_fmm))
    y_fmm = y.cpu().numpy()
    # building the per-window operators of a new time window (M2L operator
    # set, own-element blocks): once per window, cached on the tree; the
    # timed product above reuses the cached window
    ctx.profile(True)
    ctx.matvec(tree, x, 0.0, 1.1 * DT, mode="fmm", out=torch.empty_like(y))
    wst = ctx.profile_read()
    ctx.profile(False)
    window_setup = {"m2l_ops_ms": wst["m2l_ops"][0], "self_blocks_ms": wst["self_blocks"][0],
                    "note": "per new time window, cached on the tree (excluded from the timed product): the M2L "
                            "operator set and, when compressed, its bases and cores; the own-element blocks"}

    # ---------------- other Chebyshev orders (same workload, own context and
    # tree), each with the full and the compressed M2L operators
    orders = {}
    extra = [int(v) for v in args.orders.split(",") if v.strip()]
    for nn in [args.n_cheb] + [v for v in extra if v != args.n_cheb]:
        octx = Context(inputs.MATERIAL, n_cheb=nn, leaf_size=args.leaf)
        otree = octx.build_tree(d_xy)
        oy = torch.empty_like(y)
        ofn = lambda: octx.matvec(otree, x, 0.0, DT, mode="fmm", out=oy)

        def order_stages():
            octx.profile_read()
            octx.profile(True)
            for _ in range(3):
                ofn()
            ost = octx.profile_read()
            octx.profile(False)
            return {k: v[0] / 3 for k, v in ost.items() if v[1] > 0}

        oinfo = otree.info()
        rec = {"depth": oinfo["depth"], "m2l_pairs": oinfo["n_m2l_pairs"], "p2p_pairs": oinfo["n_p2p_pairs"]}
        if nn != args.n_cheb or args.m2l == "compressed":
            octx.set_m2l_compression(0)
            oms = float(np.mean(timed(ofn, args.steps, args.warmup)))
            rec.update({"ms_per_matvec": oms, "melem_s": world * N / (oms * 1e-3) / 1e6,
                        "stages_ms_per_matvec": order_stages(), "y": oy.cpu().numpy()})
        if nn >= 8 and (nn != args.n_cheb or args.m2l == "full"):
            octx.set_m2l_compression(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ofn()
            torch.cuda.synchronize()
            first = (time.perf_counter() - t0) * 1e3
            cms = float(np.mean(timed(ofn, args.steps, args.warmup)))
            rec["compressed_m2l"] = {"rank": 64 + 4 * (nn - 8), "ms_per_matvec": cms,
                                     "melem_s": world * N / (cms * 1e-3) / 1e6,
                                     "first_product_ms": first, "stages_ms_per_matvec": order_stages(),
                                     "note": "SVD-compressed M2L (ddm_set_m2l_compression mode 1); first product "
                                             "includes the set-up of the window's bases and cores",
                                     "y": oy.cpu().numpy()}
        orders[nn] = rec
        otree.close()
        octx.close()

    # ---------------- adaptive tree (the quadtree of paper Sec. 3.1 as stated:
    # cells of more than leaf_size elements split, leaves at any level)
    # against the uniform tree on a strongly clustered set; products and
    # solves on both, errors against the GPU dense product (and, on rank 0,
    # the oracle's sampled rows)
    adaptive_res = None
    if args.adaptive:
        cxy, _ = inputs.clustered_fractures(seed=inputs.SEED + 6 + 100 * rank)
        cN = cxy.shape[1]
        d_cxy = torch.as_tensor(cxy, device="cuda")
        cx_h = inputs.unknowns(cN, seed=98)
        cx = torch.as_tensor(cx_h, device="cuda")
        cy = torch.empty_like(cx)
        actx = Context(inputs.MATERIAL, n_cheb=args.n_cheb, leaf_size=args.leaf)
        actx.set_m2l_compression(1 if args.m2l == "compressed" else 0)
        dtree = actx.build_tree(d_cxy)
        actx.matvec(dtree, cx, 0.0, DT, mode="dense", out=cy)
        cy_dense = cy.cpu().numpy()
        dtree.close()
        adaptive_res = {"workload": "clustered fractures: 4 swarms x 100 cracks of 0.4-1.5 m x 20 elements in "
                                    "12 m squares + 20 cracks of 10-40 m x 100 elements over 400 m (N=10000)",
                        "N": cN, "xy": cxy, "x": cx_h}
        for kind, ad in (("uniform", False), ("adaptive", True)):
            tr = actx.build_tree(d_cxy, adaptive=ad)
            ti = tr.info()
            afn = lambda: actx.matvec(tr, cx, 0.0, DT, mode="fmm", out=cy)
            ams = float(np.mean(timed(afn, args.steps, args.warmup)))
            yk = cy.cpu().numpy()
            e = max(np.abs(yk[b * cN:(b + 1) * cN] - cy_dense[b * cN:(b + 1) * cN]).max() /
                    np.abs(cy_dense[b * cN:(b + 1) * cN]).max() for b in range(3))
            b_ = actx.rhs(tr, system="pressure", **LOADS)
            sts, sinf = [], None
            for i in range(4):                    # the first builds the tree's window caches
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, sinf = actx.gmres_solve(tr, DT, b_, system="pressure", tol=1e-5, mode="fmm",
                                           raise_on_notconv=False)
                torch.cuda.synchronize()
                if i:
                    sts.append((time.perf_counter() - t0) * 1e3)
            adaptive_res[kind] = {"depth": ti["depth"], "leaf_level_min": ti["leaf_level_min"],
                                  "cells": ti["n_cells"], "leaves": ti["n_leaves"], "m2l_pairs": ti["n_m2l_pairs"],
                                  "p2p_pairs": ti["n_p2p_pairs"], "max_leaf_records": ti["max_leaf_records"],
                                  "ms_per_matvec": ams, "melem_s": cN / (ams * 1e-3) / 1e6,
                                  "rel_err_vs_gpu_dense": e, "solve_ms": sorted(sts)[len(sts) // 2],
                                  "gmres_iterations": sinf["iterations"], "converged": bool(sinf["converged"]),
                                  "y": yk}
            tr.close()
        adaptive_res["product_speedup_adaptive_vs_uniform"] = (adaptive_res["uniform"]["ms_per_matvec"] /
                                                              adaptive_res["adaptive"]["ms_per_matvec"])
        # adaptive = "auto": the kind the library's cost model keeps on each set
        auto = {}
        for name, g in (("clustered", d_cxy), ("random_fractures_20k", d_xy)):
            at = actx.build_tree(g, adaptive="auto")
            auto[name] = "adaptive" if at.info()["adaptive"] else "uniform"
            at.close()
        adaptive_res["auto_kind"] = auto
        # the headline workload (random fractures, N = 20,000) on an adaptive tree
        mtree = actx.build_tree(d_xy, adaptive=True)
        mi = mtree.info()
        my_ = torch.empty_like(y)
        mms = float(np.mean(timed(lambda: actx.matvec(mtree, x, 0.0, DT, mode="fmm", out=my_), args.steps,
                                  args.warmup)))
        adaptive_res["random_fractures_20k_adaptive"] = {
            "depth": mi["depth"], "leaf_level_min": mi["leaf_level_min"], "leaves": mi["n_leaves"],
            "p2p_pairs": mi["n_p2p_pairs"], "m2l_pairs": mi["n_m2l_pairs"], "ms_per_matvec": mms,
            "melem_s": N / (mms * 1e-3) / 1e6}
        mtree.close()
        actx.close()

    # ---------------- dense product on the GPU (conventional PDDM)
    dense = lambda: ctx.matvec(tree, x, 0.0, DT, mode="dense", out=y)
    t_dense = timed(dense, max(2, args.steps // 5), 2)
    y_dense = y.cpu().numpy()
    ms_dense = float(np.mean(t_dense))

    # ---------------- full time-step solves
    def solve(mode):
        tr = ctx.build_tree(d_xy)
        b = ctx.rhs(tr, system="pressure", **LOADS)
        sol, inf = ctx.gmres_solve(tr, DT, b, system="pressure", tol=1e-5, mode=mode, raise_on_notconv=False)
        ctx.sif(tr, sol, tips)
        tr.close()
        return inf

    # a solve builds its own tree and window: the automatic compression
    # policy (compress a window once it has served 128 products) leaves a
    # single ~35-product solve on the full operators, which is cheaper than
    # a compression set-up per solve
    ctx.set_m2l_compression(2)
    lat, infos = [], []
    for i in range(args.solves + 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos.append(solve("fmm"))
        torch.cuda.synchronize()
        if i >= 2:
            lat.append(time.perf_counter() - t0)
    lat_ms = sorted(1e3 * v for v in lat)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dinfo = solve("dense")
    torch.cuda.synchronize()
    dense_solve_ms = 1e3 * (time.perf_counter() - t0)

    # ---------------- end to end through the C ABI with host buffers
    xh = torch.as_tensor(x_h).pin_memory()
    yh = torch.empty_like(xh).pin_memory()

    def e2e():
        x.copy_(xh, non_blocking=True)
        ctx.matvec(tree, x, 0.0, DT, mode="fmm", out=y)
        yh.copy_(y, non_blocking=True)

    t_e2e = timed(e2e, args.steps, args.warmup)
    ms_e2e = float(np.mean(t_e2e))

    # ---------------- history sum (time marching): H past steps of dt
    H = args.hist_lags
    hist = torch.as_tensor(np.stack([inputs.unknowns(N, seed=300 + k) for k in range(H)]), device="cuda")
    times = [DT * k for k in range(H + 2)]
    rhs_h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t_hist = timed(lambda: ctx.history_apply(tree, hist, times, rhs_h), 3, 1)
    ms_hist = float(np.mean(t_hist))

    # ---------------- horizontal-well march (10 x 2,000 elements, 60 s steps)
    well_res = None
    if args.well_steps > 0:
        wxy, _ = inputs.parallel_fractures(n_frac=10, spacing=20.0, half_length=100.0, elems=2000)
        wN = wxy.shape[1]
        wtree = ctx.build_tree(torch.as_tensor(wxy, device="cuda"))
        th, ts, winf, wh = well_march(ctx, wtree, wN, args.well_steps, 100.0, torch, tol=args.well_tol)
        lags = args.well_steps * (args.well_steps - 1) // 2
        tot = sum(th) + sum(ts)
        well_res = {"workload": "10 parallel fractures x 2000 elements (N=20000), RATE system, 60 s steps, "
                                f"GMRES to {args.well_tol:g}",
                    "steps": args.well_steps, "ms_per_step": tot / args.well_steps,
                    "history_ms_per_step": sum(th) / args.well_steps, "history_share": sum(th) / tot,
                    "solve_ms_per_step": sum(ts) / args.well_steps,
                    "history_melem_lags_per_s": wN * lags / (sum(th) * 1e-3) / 1e6 if lags else None,
                    "converged": int(sum(i["converged"] for i in winf)),
                    "gmres_iterations_mean": float(np.mean([i["iterations"] for i in winf]))}
        # the same march with the time-compressed history sum (8 exact steps,
        # 8 nodes per block of ratio 2), against the exact march
        ctx.set_history_compression(8, 8, 2.0)
        th2, ts2, winf2, wh2 = well_march(ctx, wtree, wN, args.well_steps, 100.0, torch, tol=args.well_tol)
        ctx.set_history_compression(0)
        tips = torch.as_tensor(np.array([f * 2000 + e for f in range(10) for e in (0, 1999)]), device="cuda")
        KI, KII = ctx.sif(wtree, wh[-1].contiguous(), tips)
        KI2, KII2 = ctx.sif(wtree, wh2[-1].contiguous(), tips)
        kscale = float(KI.abs().max())
        tot2 = sum(th2) + sum(ts2)
        d_last = (wh2[-1] - wh[-1]).abs().cpu().numpy()
        r_last = wh[-1].abs().cpu().numpy()
        well_res["compressed_history"] = {
            "exact_steps": 8, "nodes": 8, "ratio": 2.0, "ms_per_step": tot2 / args.well_steps,
            "history_ms_per_step": sum(th2) / args.well_steps, "history_share": sum(th2) / tot2,
            "converged": int(sum(i["converged"] for i in winf2)),
            "last_step_max_rel_diff_vs_exact": float(max(d_last[b * wN:(b + 1) * wN].max() /
                                                         max(r_last[b * wN:(b + 1) * wN].max(), 1e-300)
                                                         for b in range(2))),
            "sif_max_rel_diff_vs_exact": float(max((KI2 - KI).abs().max(), (KII2 - KII).abs().max()) / kscale)}
        wtree.close()

    # ---------------- batched uneven problems: autotuned per size bucket,
    # one work-list launch per stage, 1-10 time steps per problem
    batch_res = None
    if args.batch_problems > 0:
        batch_res = run_batched(args, inputs, Context, torch, LOADS)

    # ---------------- serving: Poisson arrivals, continuous batching.  The
    # stated trace (50/s for 60 s, N log-uniform in [1e3, 2e5], 1-100 steps)
    # offers far more work than one GPU does in 60 s: the window measures the
    # sustained throughput of a saturated server; at its end the unfinished
    # requests are cancelled.  Geometries are generated just before their
    # arrival (not inside the server's work).
    serve_res = None
    if args.serve_seconds > 0:
        from paper_1812_05087_gb300.ddm import Server

        def serve(mode, seconds):
            """Replay the trace's first `seconds` of arrivals against a server
            in the given product mode; unfinished requests are cancelled at
            the end of the window."""
            trace = inputs.serving_trace(duration=seconds, rate=args.serve_rate, nmin=1000, nmax=args.serve_nmax)
            ctx.set_history_compression(8, 8, 2.0)       # the server's context takes it over
            srv = Server(ctx, budget_bytes=160 << 30, max_active=32, tol=1e-5)
            ctx.set_history_compression(0)
            srv.set_mode(mode)
            tickets, keep, steps_req, sizes_req = [], [], [], []
            t0 = time.perf_counter()
            for rq in trace:
                g = torch.as_tensor(inputs.serving_geometry(rq["N"], rq["seed"]), device="cuda")
                o = torch.zeros(3 * (g.numel() // 4), dtype=torch.float64, device="cuda")
                st_ = 1 + (rq["steps"] - 1) % args.serve_max_steps
                while time.perf_counter() - t0 < rq["t"]:
                    time.sleep(0.0005)
                tickets.append(srv.submit(g, o, DT, st_, **LOADS))
                keep.append((g, o))
                steps_req.append(st_)
                sizes_req.append(g.numel() // 4)
            while time.perf_counter() - t0 < seconds:
                time.sleep(0.01)
            t_win = time.perf_counter() - t0
            snap = [srv.poll(tk) for tk in tickets]
            sstats = srv.stats()
            srv.cancel()
            t1 = time.perf_counter()
            while any(srv.poll(tk)["poll"] == 6 for tk in tickets) and time.perf_counter() - t1 < 300:
                time.sleep(0.01)
            srv.close()
            done = [k for k, r in enumerate(snap) if r["poll"] == 0]
            lats = sorted(snap[k]["latency_ms"] for k in done)
            solves = int(sum(r["steps_done"] for r in snap))
            elem_steps = float(sum(r["steps_done"] * n for r, n in zip(snap, sizes_req)))
            res = {"mode": mode, "requests_arrived": len(tickets), "completed_in_window": len(done),
                   "offered_time_step_solves": int(sum(steps_req)),
                   "offered_solves_per_s": sum(steps_req) / seconds,
                   "time_step_solves_in_window": solves, "window_s": t_win,
                   "solves_per_s": solves / t_win, "element_steps_per_s": elem_steps / t_win,
                   "p50_ms": lats[len(lats) // 2] if lats else None,
                   "p99_ms": lats[min(len(lats) - 1, int(0.99 * len(lats)))] if lats else None,
                   "server_time_ms": sstats}
            return res, done, keep, steps_req, sizes_req

        serve_res, done, keep, steps_req, sizes_req = serve("fmm", args.serve_seconds)
        serve_res["history"] = "time-compressed (8 exact steps, 8 nodes, ratio 2)"
        serve_res["trace"] = (f"Poisson {args.serve_rate}/s for {args.serve_seconds} s, N log-uniform [1e3, "
                              f"{args.serve_nmax:g}], 1-{args.serve_max_steps} steps; saturated: the unfinished "
                              f"requests are cancelled at the end of the window")
        # served results against the exact operator: completed one-step
        # requests of <= 20,000 elements, the oracle's rows of A(dt) at 6
        # sampled elements (3 rows each) against the right-hand side
        if not args.no_oracle:
            import oracle
            mat = inputs.material_tuple()
            chk = [k for k in done if steps_req[k] == 1 and sizes_req[k] <= 20000][:3]
            errs = []
            rng_o = np.random.default_rng(17)
            for k in chk:
                g, o = keep[k]
                xy_k = g.cpu().numpy().reshape(4, -1)
                n_k = xy_k.shape[1]
                el = rng_o.choice(n_k, 6, replace=False)
                rows = np.concatenate([el + c * n_k for c in range(3)])
                Ar = oracle.assemble_rows(mat, xy_k, DT, rows)
                b = oracle.rhs(xy_k, system="pressure", **LOADS)[rows]
                errs.append(float(np.abs(Ar @ o.cpu().numpy() - b).max() / np.abs(b).max()))
            serve_res["oracle_residual"] = {"requests": len(chk), "max_rel_residual": max(errs) if errs else None,
                                            "note": "completed one-step requests of <= 20,000 elements: |A(dt) x - b| "
                                                    "on 18 oracle rows, relative to max |b| (GMRES tolerance 1e-5)"}
        # the conventional dense DDM on the same request stream (a shorter window)
        dres, _, _, _, _ = serve("dense", args.serve_dense_seconds)
        serve_res["dense_arm"] = dres

    # ---------------- roofline of the dominant kernel
    st = {k: v for k, v in stages.items() if v[1] > 0 and k in ("leaf", "m2l")}
    dom = max(st, key=lambda k: st[k][0])
    dom_ms = st[dom][0] / max(1, st[dom][1])
    n = args.n_cheb
    clocks = clk.summary()
    sm_mhz = clocks["sm_mhz"] or peaks().get("sm_max_mhz", 2070.0)
    rec, rec_ok = ncu_record()
    kname = "k_tc_group" if dom == "m2l" and args.m2l == "compressed" else STAGE_KERNEL[dom]
    bound, peak, peak_note = "alu", alu_peak_tflops(sm_mhz), \
        f"FP32 peak 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz (median SM clock sampled under load)"
    exe = None
    if dom == "m2l":
        flop = 2.0 * (4 * n * n) ** 2 * info["n_m2l_pairs"]
        flop_note = "2 (4n^2)^2 flops per interaction pair (the 3xTF32 split issues 3x this on the tensor cores)"
        bound = "tensor"
        bf16 = peaks().get("bf16_tflops")
        peak = (bf16 or 1900.0) * 0.5
        peak_note = ("TF32 dense = measured" if bf16 else "TF32 dense = fallback") + \
            " bf16 GEMM peak x 0.5 (nominal TF32/BF16 ratio)"
    else:
        fpp = near_pair_flops(6)
        flop = float(info["n_p2p_pairs"]) * fpp
        flop_note = (f"{fpp} algorithmic FP32 flops per near pair (one element-integrated 4x3 kernel block: "
                     f"~150 elastic + 60 per Gauss point x 6 transient points)")
        if rec and kname in rec and "fp32_flops_per_pair" in rec[kname]:
            exe = {"flops_per_pair": rec[kname]["fp32_flops_per_pair"],
                   "achieved": float(info["n_p2p_pairs"]) * rec[kname]["fp32_flops_per_pair"] / (dom_ms * 1e-3) / 1e12,
                   "note": f"ncu-counted FP32 flops of {kname} per pair (fadd + 2 ffma + fmul)"}
    achieved = flop / (dom_ms * 1e-3) / 1e12
    roof = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": (rec[kname]["dram_bytes"] if (rec and rec_ok and kname in rec) else None),
            "flops_per_launch": flop, "flop_note": flop_note, "executed": exe,
            "peak_note": peak_note,
            "ms_per_launch": dom_ms}

    # ---------------- accuracy + CPU baseline (oracle on sampled rows)
    err = cpu = None
    if rank == 0 and not args.no_oracle:
        rng = np.random.default_rng(1)
        k = max(1, args.oracle_rows // 3)
        elems = rng.choice(N, k, replace=False)
        ref, rows, dt_or = oracle_sample(xy, x_h, elems)
        e_f = np.abs(y_fmm[rows] - ref)
        e_d = np.abs(y_dense[rows] - ref)
        scale = [np.abs(ref[b * k:(b + 1) * k]).max() for b in range(3)]
        err = {"fmm_vs_oracle": max(e_f[b * k:(b + 1) * k].max() / scale[b] for b in range(3)),
               "dense_vs_oracle": max(e_d[b * k:(b + 1) * k].max() / scale[b] for b in range(3)),
               "rows": int(rows.size)}
        for nn, o in orders.items():
            for rec in (o, o.get("compressed_m2l", {})):
                if "y" in rec:
                    e_o = np.abs(rec["y"][rows] - ref)
                    rec["error_vs_oracle"] = max(e_o[b * k:(b + 1) * k].max() / scale[b] for b in range(3))
        if adaptive_res is not None:                 # the clustered set's sampled rows
            ca = adaptive_res
            celems = rng.choice(ca["N"], k, replace=False)
            cref, crows, _ = oracle_sample(ca["xy"], ca["x"], celems)
            cscale = [np.abs(cref[b * k:(b + 1) * k]).max() for b in range(3)]
            for kind in ("uniform", "adaptive"):
                e_c = np.abs(ca[kind]["y"][crows] - cref)
                ca[kind]["error_vs_oracle"] = max(e_c[b * k:(b + 1) * k].max() / cscale[b] for b in range(3))
        import oracle
        cpu = {"value": k / dt_or / 1e6, "unit": "Melem/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"{k} target elements (3 rows each) x {N} sources, FP64 adaptive element quadrature"}

    # ---------------- max over ranks
    tot_ms, ms_e2e = max_over_ranks(dist, [ms_fmm, ms_e2e], "cuda")
    if rank != 0:
        return
    value = whole_job_melem_s(world, N, tot_ms)
    solves_s = 1e3 / float(np.mean(lat_ms))
    line = {
        "metric": METRIC, "value": value, "unit": "Melem/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "n_cheb": n, "leaf": args.leaf, "depth": info["depth"],
                   "m2l_pairs": info["n_m2l_pairs"], "p2p_pairs": info["n_p2p_pairs"],
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}",
                   "m2l": (f"SVD-compressed operators, rank {64 + 4 * (n - 8)}" if args.m2l == "compressed" and n >= 8
                           else "full operators")},
        "solves_per_s": world * solves_s, "solves_timed": len(lat_ms), "solve_p50_ms": lat_ms[len(lat_ms) // 2],
        "solve_p99_ms": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))],
        "gmres_iterations": infos[-1]["iterations"], "gmres_rel_residual": infos[-1]["rel_residual"],
        "dense_melem_s": world * N / (ms_dense * 1e-3) / 1e6, "dense_ms_per_matvec": ms_dense,
        "dense_solve_ms": dense_solve_ms, "dense_gmres_iterations": dinfo["iterations"],
        "fmm_speedup_vs_dense": ms_dense / ms_fmm,
        "history": {"lags": H, "ms": ms_hist, "melem_lags_per_s": N * H / (ms_hist * 1e-3) / 1e6},
        "window_setup": window_setup,
        "orders": {str(nn): {k: ({kk: vv for kk, vv in v.items() if kk != "y"} if isinstance(v, dict) else v)
                             for k, v in o.items() if k != "y"} for nn, o in orders.items()},
        "adaptive_tree": ({k: ({kk: vv for kk, vv in v.items() if kk != "y"} if isinstance(v, dict) else v)
                           for k, v in adaptive_res.items() if k not in ("xy", "x")} if adaptive_res else None),
        "well": well_res,
        "batched": batch_res, "serving": serve_res,
        "error": err,
        "stages_ms_per_matvec": {k: v[0] / 3 for k, v in stages.items() if v[1] > 0},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": whole_job_melem_s(world, N, ms_e2e), "unit": "Melem/s",
                "h2d_bytes_per_step": int(x.numel() * 8), "d2h_bytes_per_step": int(y.numel() * 8)},
        "gpu_launches": int(round(per_matvec_launches * args.steps)),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
