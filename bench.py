"""Benchmark of the DABS bulk local search on GB300.

Default workload: the sparse Max-Cut-shaped QUBO (G(n=800, p=0.06), edge
weights +-1, seed 1) with 1024 concurrent searches, 4 pools x 100 packets,
tabu 8, s = 1/10, b = 10, Straight seeding, one instance per launch.  One step
is one generation: offspring -> batch search (every search flips >= b*n bits)
-> pool merge -> finalise, all in the CUDA library.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dabs|reference]

Prints one JSON line.  --impl reference times the plain C oracle (the CPU
restatement of the method) on the host cores, one generation per step.
Under torchrun (N > 1) every rank runs an independent replica (weak scaling,
no collective on the data path); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2207_03069_gb300 import workloads as wl  # noqa: E402

WORKLOADS = {
    "maxcut800": dict(desc="sparse Max-Cut QUBO G(n=800,p=0.06) w=+-1 seed 1", n=800,
                      searches=1024, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(10, 1),
                      seed_mode=0),
    "dense64": dict(desc="dense QUBO n=64 W~U[-100,100] seed 0", n=64, searches=32, pools=4,
                    pool_cap=64, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0),
    "tsp32": dict(desc="TSP one-hot 32 cities (1024 bits) grid 1000 seed 2", n=1024,
                  searches=2048, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0),
    "qasp5627": dict(desc="QASP-shaped sparse Ising r=256, 5627 nodes 40279 random edges, seed 6",
                     n=5627, searches=1024, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1),
                     seed_mode=0),
}


def make_W(name):
    if name == "maxcut800":
        return wl.maxcut_qubo(800, 0.06, seed=1)
    if name == "dense64":
        return wl.dense_qubo(64, -100, 100, seed=0)
    if name == "tsp32":
        return wl.tsp_qubo(32, 1000, seed=2)[0]
    if name == "qasp5627":
        return wl.sparse_ising_qubo(5627, 40279, 256, seed=6)
    raise ValueError(name)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def search_profile():
    """DRAM traffic of the batch-search kernel from the committed ncu summary,
    valid only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "search_maxcut800.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        prof = json.load(f)
    h = hashlib.sha256()
    for fn in ("search.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2207_03069_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    if prof.get("kernel_sha256") != h.hexdigest():
        return None
    return prof


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.th:
            self.th.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_copy_gbs(torch, dev):
    """Read+write bandwidth of a 32 MiB device copy that stays in L2 (context)."""
    a = torch.empty(8 << 20, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(5):
        b.copy_(a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 200
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    torch.cuda.synchronize()
    return 2 * a.numel() * 4 * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9


def recompute_rate(torch, dabs, dev, n=4096, count=256, reps=20):
    """Tensor-core recompute of Delta/E (tcgen05, bf16 limbs) for `count`
    vectors of a dense n x n instance: the batched-seeding step of the batched
    workload.  Returns timing and the tensor FLOP rate (2 limbs x 2 S n^2)."""
    W = wl.dense_qubo(n, -1000, 1000, seed=3)
    ctx = dabs.Context(W, searches=count, pools=1, pool_cap=1)
    rng = np.random.default_rng(3)
    X = torch.from_numpy(wl.pack_bits((rng.random((count, n)) < 0.5).astype(np.uint8))
                         .view(np.int32)).to(dev)
    E = torch.zeros(count, dtype=torch.int64, device=dev)
    dl = torch.zeros((count, ctx.ld), dtype=torch.int32, device=dev)
    st = torch.cuda.Stream(device=dev)
    ctx.set_stream(st)
    for _ in range(3):
        ctx.recompute_dev(X, E, dl)
    ctx.kernel_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(st)
    for _ in range(reps):
        ctx.recompute_dev(X, E, dl)
    ev[1].record(st)
    ctx.kernel_status()
    ms = ev[0].elapsed_time(ev[1]) / reps
    flops = 4.0 * count * n * n
    ctx.close()
    return {"n": n, "vectors": count, "ms": ms, "tensor_tflops": flops / (ms * 1e-3) / 1e12,
            "note": "bf16 limbs on tcgen05.mma kind::f16, exact; includes bit->bf16 expansion"}


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(np.ceil(q / 100.0 * len(xs))) - 1))
    return xs[k]


def row_roofline(row_bytes_per_s):
    """The flip kernel's algorithmic row traffic (2 n bytes per flip) as a
    fraction of the measured HBM copy peak (whole-run rates, host timing)."""
    hbm, kind = peaks()
    return {"row_gbs": row_bytes_per_s / 1e9, "frac_of_hbm": row_bytes_per_s / 1e9 / hbm,
            "peak": f"{kind} HBM copy {hbm:.0f} GB/s"}


def tsp_ttt(dabs, seeds=32, generations=30):
    """TSP-shaped QUBO (32 cities, one-hot 1024 bits, 2048 searches, b = 1,
    s = 1/10): per seed the target is the best energy that seed's solve reaches
    in `generations` generations; time-to-target = wall time of the solve with
    that target (host API, results back on the host)."""
    W, dist, p = wl.tsp_qubo(32, 1000, seed=2)
    kw = dict(searches=2048, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0)
    ctx = dabs.Context(W, **kw, max_generations=generations)
    ttt, flips, feasible = [], 0, 0
    ctx.solve(10**12, seed=10**6)  # warm
    for sd in range(seeds):
        X, target, _ = ctx.solve(10**12, seed=sd)
        t0 = time.perf_counter()
        X2, E2, F2 = ctx.solve(10**12, seed=sd, target=target)
        ttt.append(time.perf_counter() - t0)
        flips += F2
        assert E2 == target
        M = X2.reshape(32, 32)  # one-hot feasible: every position and city used once
        feasible += int((M.sum(0) == 1).all() and (M.sum(1) == 1).all())
    ctx.close()
    return {"workload": "TSP 32 cities one-hot n=1024, 2048 searches, b=1, s=1/10",
            "seeds": seeds, "target": f"best energy of the same seed after {generations} generations",
            "ttt_p50_s": pct(ttt, 50), "ttt_p99_s": pct(ttt, 99), "flips_per_s": flips / sum(ttt),
            "feasible_targets": feasible, "roofline": row_roofline(flips / sum(ttt) * 2 * 1024)}


def batched_vs_plain(dabs, count=64, generations=3):
    """64 dense QUBOs, n log-uniform in [256, 4096] (seed 3), W ~ U[-1000, 1000],
    256 searches each, recompute seeding on the tensor cores: one batched solve
    vs one solve per instance (one instance per launch), same seeds."""
    ns = wl.batched_sizes(count, 256, 4096, seed=3)
    kw = dict(searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1,
              max_generations=generations)
    Ws = [wl.dense_qubo(int(n), -1000, 1000, seed=1000 + i) for i, n in enumerate(ns)]
    ctxs = [dabs.Context(W, **kw) for W in Ws]
    seeds = list(range(count))
    big = [10**12] * count
    dabs.batch_solve(ctxs[:2], big[:2], seeds[:2])  # warm
    for c in ctxs[:2]:
        c.solve(10**12, seed=0)
    torch_sync()
    t0 = time.perf_counter()
    bout = dabs.batch_solve(ctxs, big, seeds)
    tb = time.perf_counter() - t0
    t0 = time.perf_counter()
    pout = [c.solve(10**12, seed=sd) for c, sd in zip(ctxs, seeds)]
    tp = time.perf_counter() - t0
    same = all(b[1] == q[1] and b[2] == q[2] and np.array_equal(b[0], q[0])
               for b, q in zip(bout, pout))
    fl = sum(b[2] for b in bout)
    row_bytes = sum(b[2] * 2 * int(n) for b, n in zip(bout, ns))
    # time to target: every instance's target is the energy it reaches alone in
    # `generations` generations; all 64 arrive at t = 0.  Plain: one solve after
    # another (an instance waits for those before it); served: submitted at once
    # to the continuous-batching server.
    targets = [int(q[1]) for q in pout]
    for c in ctxs:
        c.close()
    t0 = time.perf_counter()
    plain_ttt = []
    for W, sd, tg in zip(Ws, seeds, targets):  # context set-up counted, as the server's is
        c = dabs.Context(W, **kw)
        c.solve(10**12, seed=sd, target=tg)
        c.close()
        plain_ttt.append(time.perf_counter() - t0)
    params = dabs.default_params(**kw)
    srv = dabs.Server(60 << 30)
    tickets = [srv.submit(W, params, 10**12, sd, target=tg) for W, sd, tg in zip(Ws, seeds, targets)]
    while srv.step(1):
        pass
    served_ttt, reached = [], True
    for t, tg in zip(tickets, targets):
        st, X, E, F, L = srv.poll(t)
        served_ttt.append(L)
        reached = reached and E <= tg
    srv.close()
    return {"workload": f"{count} dense QUBOs n log-uniform [256,4096], 256 searches each, "
                        f"{generations} generations, tensor-core recompute seeding",
            "batched_flips_per_s": fl / tb, "plain_flips_per_s": fl / tp,
            "speedup": tp / tb, "identical_results": bool(same), "flips": fl,
            "roofline_batched": row_roofline(row_bytes / tb),
            "ttt": {"target": f"the energy each instance reaches alone in {generations} generations; "
                              f"all {count} arrive at t = 0",
                    "plain_p50_s": pct(plain_ttt, 50), "plain_p99_s": pct(plain_ttt, 99),
                    "served_p50_s": pct(served_ttt, 50), "served_p99_s": pct(served_ttt, 99),
                    "targets_reached": bool(reached)}}


def small_graphs(dabs, generations=200, reps=3):
    """The small dense workload (n = 64, W ~ U[-100, 100] seed 0, 32 searches,
    4 pools x 64, b = 1, s = 1/10) solved for 200 generations through
    dabs_solve, with generations replayed from the captured CUDA graph and
    launched kernel by kernel; best of `reps`, same seed, identical results."""
    W = wl.dense_qubo(64, -100, 100, seed=0)
    kw = dict(searches=32, pools=4, pool_cap=64, tabu=8, s=(1, 10), b=(1, 1), seed_mode=0,
              max_generations=generations)
    out, res = {}, {}
    for graphs in (True, False):
        ctx = dabs.Context(W, **kw)
        ctx.set_graphs(graphs)
        ctx.solve(10**12, seed=0)  # warm (and capture)
        best = None
        for _ in range(reps):
            torch_sync()
            t0 = time.perf_counter()
            X, E, f = ctx.solve(10**12, seed=1)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        res[graphs] = (X.tobytes(), E, f)
        out["graphs" if graphs else "kernel_by_kernel"] = {"flips_per_s": f / best,
                                                           "ms_per_generation": best * 1e3 / generations}
        ctx.close()
    out["identical_results"] = res[True] == res[False]
    out["roofline"] = row_roofline(out["graphs"]["flips_per_s"] * 2 * 64)
    out["speedup"] = out["kernel_by_kernel"]["ms_per_generation"] / out["graphs"]["ms_per_generation"]
    out["workload"] = "dense n=64, 32 searches, 200 generations x >= 64 flips per search"
    return out


def serving(dabs, seconds=4.0, rate=50.0, generations=20, sizes=(512, 1024, 2048, 4096, 8192),
            budget_gb=60, plain=True, big=16384):
    """Poisson arrivals (seed 4) of dense QUBOs, n uniform in `sizes`, plus one
    n = `big` instance mid-trace, 256 searches, 20 generations each, recompute
    seeding; served with continuous batching under an HBM budget, and (plain)
    one request at a time on the same trace.  Latency = completion - arrival."""
    rng = np.random.default_rng(4)
    arr = wl.poisson_arrivals(rate, seconds, seed=4)
    reqs = [(float(t), int(rng.choice(sizes)), 5000 + i) for i, t in enumerate(arr)]
    if big:  # the one n = 16384 instance (512 MB of int16 W), arriving mid-trace
        reqs.append((seconds / 2, big, 9999))
        reqs.sort()
    kw = dict(searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1,
              max_generations=generations)
    params = dabs.default_params(**kw)
    Wcache = {}

    def W_of(n, sd):
        key = (n, sd)
        if key not in Wcache:
            Wcache[key] = wl.dense_qubo(n, -1000, 1000, seed=sd)
        return Wcache[key]

    for _, n, sd in reqs:  # instances are prepared before the clock starts
        W_of(n, sd)
    out = {"workload": f"Poisson {rate}/s for {seconds}s, n in {list(sizes)}"
                       + (f" plus one n={big} instance" if big else "")
                       + f", 256 searches, {generations} generations, recompute seeding",
           "requests": len(reqs)}
    srv = dabs.Server(budget_gb << 30)
    t0 = time.perf_counter()
    tickets, i, pending = [], 0, 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            _, n, sd = reqs[i]
            tickets.append(srv.submit(W_of(n, sd), params, 10**12, sd))
            i += 1
        if srv.info()[1] + srv.info()[2] == 0:
            time.sleep(0.001)
            pending = 0
            continue
        pending = srv.step(1)
    wall = time.perf_counter() - t0
    lat, fl, rb = [], 0, 0
    for t, (_, n, _) in zip(tickets, reqs):
        st, X, E, F, L = srv.poll(t)
        lat.append(L)
        fl += F
        rb += F * 2 * n
        if n == big:
            out["served_big_latency_s"] = L
    srv.close()
    out.update({"served_p50_s": pct(lat, 50), "served_p99_s": pct(lat, 99),
                "served_flips_per_s": fl / wall, "served_wall_s": wall,
                "roofline_served": row_roofline(rb / wall)})
    if plain:
        t0 = time.perf_counter()
        lat2, free_at = [], 0.0
        for (ta, n, sd) in reqs:
            start = max(ta, free_at)
            now = time.perf_counter() - t0
            if now < start:
                time.sleep(start - now)
            c = dabs.Context(W_of(n, sd), **kw)
            c.solve(10**12, seed=sd)
            c.close()
            free_at = time.perf_counter() - t0
            lat2.append(free_at - ta)
        out.update({"plain_p50_s": pct(lat2, 50), "plain_p99_s": pct(lat2, 99),
                    "plain_flips_per_s": fl / (time.perf_counter() - t0)})
    return out


def torch_sync():
    import torch
    torch.cuda.synchronize()


def oracle_rate(Wm, spec, seed, seconds, threads):
    """Oracle (plain C, as it stands) on the same workload: whole generations on
    `threads` host threads until `seconds` have passed.  Returns (flips/s, gens)."""
    from oracle import oracle as orc
    p = orc.make_params(searches=spec["searches"], pools=spec["pools"], pool_cap=spec["pool_cap"],
                        tabu=spec["tabu"], s=spec["s"], b=spec["b"], seed_mode=spec["seed_mode"])
    so = orc.Solver(Wm, p, seed)
    t0 = time.perf_counter()
    flips, gens = 0, 0
    while True:
        flips += so.generation(threads)
        gens += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return flips / (time.perf_counter() - t0), gens


def aggregate(pg, seconds, flips):
    """Whole-job figures over replicas: the slowest rank's time and the sum of
    all ranks' flips (host-side gloo reduction; no collective on the data path)."""
    if pg is None:
        return seconds, flips
    import torch
    t = torch.tensor([seconds, flips], dtype=torch.float64)
    tmax = t.clone()
    pg.all_reduce(tmax, op=pg.ReduceOp.MAX)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    lrank = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        pg = dist
    return ws, rank, lrank, pg


def run_reference(args, ws, rank, pg):
    spec = WORKLOADS[args.workload]
    if rank != 0:
        return
    Wm = make_W(args.workload)
    from oracle import oracle as orc
    threads = os.cpu_count() or 1
    p = orc.make_params(searches=spec["searches"], pools=spec["pools"], pool_cap=spec["pool_cap"],
                        tabu=spec["tabu"], s=spec["s"], b=spec["b"], seed_mode=spec["seed_mode"])
    so = orc.Solver(Wm, p, args.seed)
    for _ in range(args.warmup):
        so.generation(threads)
    t0 = time.perf_counter()
    flips = 0
    for _ in range(args.steps):
        flips += so.generation(threads)
    dt = time.perf_counter() - t0
    v = flips / dt
    line = {"impl": "reference", "metric": "bit flips/s", "value": v, "unit": "flips/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": spec["desc"], "n": spec["n"], "searches": spec["searches"],
                       "pools": spec["pools"], "pool_cap": spec["pool_cap"],
                       "tabu": spec["tabu"], "s": "%d/%d" % spec["s"], "b": "%d/%d" % spec["b"],
                       "seeding": "straight" if spec["seed_mode"] == 0 else "recompute",
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": v, "unit": "flips/s", "cores": threads, "kind": "oracle",
                             "sample": f"{args.steps} whole generations after {args.warmup} "
                                       f"warm-up generations, {spec['searches']} searches"},
            "e2e": {"value": v, "unit": "flips/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dabs", choices=["dabs", "reference"])
    ap.add_argument("--workload", default="maxcut800", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-recompute", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the TSP time-to-target, batched and serving measurements")
    ap.add_argument("--trace-seconds", type=float, default=4.0)
    ap.add_argument("--variant", default="", help="force warps x chunks, e.g. 4x1")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, lrank, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
        if pg:
            pg.barrier()
        return

    import torch
    from paper_2207_03069_gb300 import build, dabs

    build.build()
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    spec = WORKLOADS[args.workload]
    Wm = make_W(args.workload)
    n = Wm.shape[0]
    kw = {k: spec[k] for k in ("searches", "pools", "pool_cap", "tabu", "s", "b", "seed_mode")}
    ctx = dabs.Context(Wm, **kw)
    stream = torch.cuda.Stream(device=dev)
    ctx.set_stream(stream)
    sweep = {}
    if args.variant:
        ctx.set_variant_name(args.variant)
    elif not args.no_autotune:
        tuned = ctx.autotune(3)  # untimed: picks warps x chunks and the row format
        sweep = {"chosen": ctx.variant_name(), "ns_per_flip": tuned[3]}
    seed = args.seed + 1000 * rank
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    # ---------------- device-resident timing: one generation per step
    ctx.solve_begin(seed)
    for _ in range(args.warmup):
        ctx.solve_generations(1)
    st0 = ctx.solve_status()
    sampler = ClockSampler(lrank)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)  # untimed: evict L2 between timed steps
        e = ev[k]
        e[0].record(stream)
        ctx.run_stage(dabs.STAGE_OFFSPRING)
        e[1].record(stream)
        ctx.run_stage(dabs.STAGE_SEARCH)
        e[2].record(stream)
        ctx.run_stage(dabs.STAGE_MERGE)
        ctx.run_stage(dabs.STAGE_FINALIZE)
        e[3].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    st1 = ctx.solve_status()
    step_ms = [e[0].elapsed_time(e[3]) for e in ev]
    search_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_s = sum(step_ms) * 1e-3
    flips = st1["flips"] - st0["flips"]
    total_s, flips = aggregate(pg, total_s, flips)
    value = flips / total_s
    flips_rank = st1["flips"] - st0["flips"]

    # ---------------- roofline of the batch-search kernel
    hbm, peak_kind = peaks()
    algo_bytes = flips_rank * 2 * n / args.steps  # int16 row of W per flip, per launch
    launch_s = sum(search_ms) * 1e-3 / args.steps
    achieved = algo_bytes / launch_s / 1e9
    prof = search_profile()
    info = ctx.info()
    vkey = "%dx%d" % (info["warps"], info["chunks"])
    traffic = prof["dram_bytes_per_launch"].get(vkey) if prof else None
    l2 = l2_copy_gbs(torch, dev)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_kind": f"{peak_kind} HBM copy",
                "traffic": traffic, "traffic_source": "profiles/search_maxcut800.json" if traffic else None,
                "kernel": "k_batch_search", "algorithmic_bytes_per_launch": algo_bytes,
                "launch_ms": launch_s * 1e3, "search_share_of_step": sum(search_ms) / sum(step_ms),
                "l2_copy_gbs_measured": l2, "frac_of_l2_copy": achieved / l2}
    # integer-ALU ceiling beside the memory roofline: the ALU pipe (integer
    # compare, min, select, logic) issues 16 lanes per scheduler, 4 schedulers
    # per SM; the ncu capture gives the ALU instructions the kernel spends per flip
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 4 * 16 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    rate = flips_rank / (sum(step_ms) * 1e-3)  # this GPU's flips/s
    alu = {"pipe": "ALU (integer compare/min/select/logic), 64 lanes per SM",
           "peak_lane_ops_per_s": alu_peak, "algorithmic_lane_ops_per_flip": 2 * n,
           "frac_algorithmic": rate * 2 * n / alu_peak}
    pv = prof["variants"].get(vkey) if prof else None
    if pv and "alu_warp_inst_per_flip_est" in pv:
        per_flip = pv["alu_warp_inst_per_flip_est"]
        alu.update({"executed_warp_inst_per_flip_ncu": per_flip,
                    "ceiling_flips_per_s": alu_peak / (32 * per_flip),
                    "frac_of_ceiling": rate * 32 * per_flip / alu_peak,
                    "alu_pct_of_peak_ncu": pv.get("alu_pct_of_peak_active")})
    roofline["alu"] = alu

    # ---------------- end to end through the C ABI with host buffers
    Wpin = torch.empty((n, n), dtype=torch.int16, pin_memory=True).numpy()
    Wpin[:] = Wm
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    ctx.set_stream(None)
    ctx.solve(1, seed=seed)  # warm
    t0 = time.perf_counter()
    e2e_flips = 0
    for k in range(e2e_steps):
        ctx.load_weights(Wpin)              # H2D of the step's input
        X, E, f = ctx.solve(1, seed=seed + k)  # one generation, best X/E back to the host
        e2e_flips += f
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_flips / e2e_s, "unit": "flips/s", "h2d_bytes_per_step": 2 * n * n,
           "d2h_bytes_per_step": n + 8,
           "call": "dabs_load_weights + dabs_solve(budget=1 generation) per step"}

    rec = recompute_rate(torch, dabs, dev) if not args.no_recompute else None
    extra = {}
    if not args.no_extra and ws == 1:
        extra["small_graphs"] = small_graphs(dabs)
        extra["time_to_target"] = tsp_ttt(dabs)
        extra["batched"] = batched_vs_plain(dabs)
        extra["serving"] = serving(dabs, seconds=args.trace_seconds)
    if rec:
        mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
        pk = json.load(open(mp))["bf16_tflops"] if os.path.exists(mp) else 1900.0
        rec["peak_tflops"] = pk
        rec["frac"] = rec["tensor_tflops"] / pk

    # ---------------- CPU baseline: the oracle as it stands, bounded sample
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, gens = oracle_rate(Wm, spec, seed, args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": "flips/s", "cores": threads, "kind": "oracle",
               "sample": f"first {gens} generation(s) of the same workload ({spec['searches']} "
                         f"searches), about {args.cpu_seconds:.0f} s"}
        # the same oracle on one thread, over a smaller solve of the same W and
        # parameters (one generation of 64 searches: about 1/16 of the work)
        one = dict(spec, searches=64)
        r1, g1 = oracle_rate(Wm, one, seed, 0.0, 1)
        cpu["single_thread"] = {"value": r1, "unit": "flips/s", "cores": 1,
                                "sample": f"{g1} generation(s) of 64 searches, same W and parameters"}

    if rank == 0:
        line = {"metric": "bit flips/s", "value": value, "unit": "flips/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": spec["desc"], "n": n, "searches": spec["searches"],
                           "pools": spec["pools"], "pool_cap": spec["pool_cap"],
                           "tabu": spec["tabu"], "s": "%d/%d" % spec["s"],
                           "b": "%d/%d" % spec["b"],
                           "seeding": "straight" if spec["seed_mode"] == 0 else "recompute",
                           "variant": "%d warp(s) x %d chunk(s)" % (ctx.info()["warps"],
                                                                    ctx.info()["chunks"]),
                           "l2": "flushed (256 MiB write) between timed steps",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "delta_updates_per_s": value * n, "autotune": sweep, "gpu_launches": 5 * args.steps,
                "clocks": clocks, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu,
                "recompute_tensor": rec, **extra}
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.barrier()


if __name__ == "__main__":
    main()
