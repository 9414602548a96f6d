"""Benchmark of the DABS bulk local search on GB300.

Default workload (the metric's "batched vs plain"): 64 dense QUBOs with n
log-uniform in [256, 4096] (seed 3), W ~ U[-1000, 1000] (seed 1000 + i), 256
searches each, 4 pools x 100 packets, tabu 8, s = 1/10, b = 1, recompute
seeding on the tensor cores.  One step is one generation of every instance:
offspring -> recompute -> batch search (every search flips >= b*n bits) ->
pool merge -> finalise, all in the CUDA library, in the batched form (one
batch-search launch per kernel variant for all instances).  The same instances
and seeds are also timed in the plain form (one instance per launch) and must
give identical results.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl dabs|reference]
                    [--workload batched64|maxcut800|tsp32|dense64|qasp5627]

Prints one JSON line.  --impl reference times the plain C oracle (the CPU
restatement of the method) on the host cores, one generation of a bounded
sample of the workload per step.  Under torchrun (N > 1) every rank runs an
independent replica (weak scaling, no collective on the data path); rank 0
prints the aggregate.
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
    "batched64": dict(desc="64 dense QUBOs, n log-uniform in [256,4096] (seed 3), W~U[-1000,1000] "
                           "(seed 1000+i), 256 searches each", kind="batched", count=64, n_lo=256,
                      n_hi=4096, searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1),
                      seed_mode=1, sample_searches=16),
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


def batched_instances(spec):
    ns = wl.batched_sizes(spec["count"], spec["n_lo"], spec["n_hi"], seed=3)
    return [wl.dense_qubo(int(n), -1000, 1000, seed=1000 + i) for i, n in enumerate(ns)]


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


def search_profile(fname="search_maxcut800.json"):
    """DRAM traffic of the batch-search kernel from a committed ncu summary,
    valid only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", fname)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        prof = json.load(f)
    if prof.get("kernel_sha256") != kernel_hash():
        return None
    return prof


def kernel_hash():
    """sha256 of the search kernel's source (search.cuh, common.cuh) without
    its // comments and blank lines: a capture stays valid across comment
    edits, not across code changes."""
    h = hashlib.sha256()
    for fn in ("search.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2207_03069_gb300", "csrc", fn), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


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


def rows_from_l2(wset, l2_size, traffic, row_bytes):
    """Where the flip kernel's rows come from: the L2 when W and -W fit it, or
    when the captured DRAM traffic of the search launches (bytes, None when
    no capture matches the kernel) is under a quarter of the row bytes they
    read (the instances searched at one time fit the L2 together)."""
    return wset <= l2_size or (traffic is not None and traffic < 0.25 * row_bytes)


def l2_read_gbs(torch, dev, mib=64, reps=20):
    """Read bandwidth of a buffer that stays in L2 (64 MiB of the 129 MB L2),
    measured by the library's read kernel (dabs_measure_read_gbs): the L2 peak
    the flip kernel's row reads are compared with when W fits the L2."""
    from paper_2207_03069_gb300 import dabs
    a = torch.randint(-1000, 1000, ((mib << 20) // 4,), dtype=torch.int32, device=dev)
    return dabs.measure_read_gbs(a, reps)


def recompute_rate(torch, dabs, dev, n=4096, count=256, reps=20):
    """Tensor-core recompute of Delta/E (tcgen05) for `count` vectors of a
    dense n x n instance with W ~ U[-1000, 1000] (the batched workload's
    weights): the batched-seeding step.  Returns timing and the rate of the
    contraction D W in FLOP/s (2 S n^2 per call; with |W| <= 2048 the kernel
    multiplies by W itself as one fp16 operand)."""
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
    flops = 2.0 * count * n * n
    ctx.close()
    return {"n": n, "vectors": count, "ms": ms, "tensor_tflops": flops / (ms * 1e-3) / 1e12,
            "flops_per_call": flops,
            "note": "tcgen05.mma kind::f16 (W as one fp16 operand, exact for |W| <= 2048), "
                    "M = 256 vectors per CTA; includes the bit -> fp16 expansion kernel"}


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


_T0 = time.perf_counter()


def progress(msg):
    """A progress line on stderr (the JSON line alone goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}\n")
    sys.stderr.flush()


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


def run_reference_batched(args, ws, rank, pg):
    """The oracle on the batched workload's sample (every instance, with
    sample_searches searches each): one generation of all instances per step."""
    spec = WORKLOADS[args.workload]
    if rank != 0:
        return
    Ws = batched_instances(spec)
    ns = [W.shape[0] for W in Ws]
    from oracle import oracle as orc
    threads = os.cpu_count() or 1
    p = orc.make_params(searches=spec["sample_searches"], pools=spec["pools"],
                        pool_cap=spec["pool_cap"], tabu=spec["tabu"], s=spec["s"], b=spec["b"],
                        seed_mode=spec["seed_mode"])
    sos = [orc.Solver(W, p, args.seed + i) for i, W in enumerate(Ws)]
    for _ in range(args.warmup):
        for so in sos:
            so.generation(threads)
    t0 = time.perf_counter()
    flips = 0
    for _ in range(args.steps):
        for so in sos:
            flips += so.generation(threads)
    dt = time.perf_counter() - t0
    v = flips / dt
    line = {"impl": "reference", "metric": "bit flips/s (batched vs plain, bit-exact)", "value": v,
            "unit": "flips/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": spec["desc"], "instances": len(Ws), "n_min": min(ns),
                       "n_max": max(ns), "searches": spec["searches"], "pools": spec["pools"],
                       "pool_cap": spec["pool_cap"], "tabu": spec["tabu"],
                       "s": "%d/%d" % spec["s"], "b": "%d/%d" % spec["b"],
                       "seeding": "recompute", "parallelism": "host threads"},
            "cpu_baseline": {"value": v, "unit": "flips/s", "cores": threads, "kind": "oracle",
                             "sample": f"per step one generation of all {len(Ws)} instances with "
                                       f"{spec['sample_searches']} of their {spec['searches']} "
                                       f"searches (same W and parameters)"},
            "e2e": {"value": v, "unit": "flips/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, ws, rank, pg):
    spec = WORKLOADS[args.workload]
    if spec.get("kind") == "batched":
        return run_reference_batched(args, ws, rank, pg)
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


# ------------------------------------------------------------------ batched workload
def oracle_batched_rate(Ws, spec, seed, seconds, threads, gens=None):
    """The oracle (plain C, as it stands) on a bounded sample of the batched
    workload: every instance with `sample_searches` searches (same W and
    parameters), whole generations of all instances until `seconds` have
    passed (or `gens` generations).  Returns (flips/s, generations)."""
    from oracle import oracle as orc
    p = orc.make_params(searches=spec["sample_searches"], pools=spec["pools"],
                        pool_cap=spec["pool_cap"], tabu=spec["tabu"], s=spec["s"], b=spec["b"],
                        seed_mode=spec["seed_mode"])
    sos = [orc.Solver(W, p, seed + i) for i, W in enumerate(Ws)]
    t0 = time.perf_counter()
    flips, g = 0, 0
    while True:
        for so in sos:
            flips += so.generation(threads)
        g += 1
        if (gens is not None and g >= gens) or (gens is None and time.perf_counter() - t0 >= seconds):
            break
    return flips / (time.perf_counter() - t0), g


SERVE_SIZES = (512, 1024, 2048, 4096, 8192)
SERVE_CATALOG = 16  # distinct instances per size (W ~ U[-1000, 1000], seed 5000 + 16 size + j)


def serve_requests(rate, seconds, seed, sizes=SERVE_SIZES, big=0):
    """Poisson arrivals (rate per s for `seconds`, seed) of dense QUBOs with n
    uniform in `sizes`: request i solves instance j = i mod 16 of its size
    with solve seed 20000 + i; plus one n = `big` instance mid-trace.  The
    same seed gives request i the same size at every rate.  Returns a list of
    (arrival s, n, instance seed, solve seed) sorted by arrival."""
    rng = np.random.default_rng(seed)
    arr = wl.poisson_arrivals(rate, seconds, seed=seed)
    reqs = []
    for i, t in enumerate(arr):
        n = int(rng.choice(sizes))
        reqs.append((float(t), n, 5000 + 16 * sizes.index(n) + i % SERVE_CATALOG, 20000 + i))
    if big:
        reqs.append((seconds / 2, big, 9999, 9999))
        reqs.sort()
    return reqs


def serve_kw(generations):
    return dict(searches=256, pools=4, pool_cap=100, tabu=8, s=(1, 10), b=(1, 1), seed_mode=1,
                max_generations=generations)


def served_trace(dabs, reqs, generations, budget_gb=60, targets=None, Wcache=None):
    """Serves `reqs` (serve_requests) with continuous batching: 256 searches,
    a flip budget of 256 x generations x n and at most `generations`
    generations, recompute seeding.  With `targets` ((n, instance, solve
    seed) -> energy), each request stops at its target; latency = completion
    - arrival.  Returns (results, latencies, flips, wall seconds)."""
    Wcache = {} if Wcache is None else Wcache
    for _, n, inst, _ in reqs:  # instances are prepared before the clock starts
        if (n, inst) not in Wcache:
            Wcache[(n, inst)] = wl.dense_qubo(n, -1000, 1000, seed=inst)
    params = dabs.default_params(**serve_kw(generations))
    srv = dabs.Server(budget_gb << 30)
    t0 = time.perf_counter()
    tickets, i, pending = [], 0, 0
    while i < len(reqs) or pending:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i][0] <= now:
            _, n, inst, sd = reqs[i]
            tg = None if targets is None else targets[(n, inst, sd)]
            tickets.append(srv.submit(Wcache[(n, inst)], params, 256 * generations * n, sd, target=tg))
            i += 1
        if srv.info()[1] + srv.info()[2] == 0:
            time.sleep(0.0005)
            pending = 0
            continue
        pending = srv.step(1)
    wall = time.perf_counter() - t0
    res, lat, fl = {}, [], 0
    for t, (_, n, inst, sd) in zip(tickets, reqs):
        st, X, E, F, L = srv.poll(t)
        res[(n, inst, sd)] = (X.tobytes(), E, F)
        lat.append(L)
        fl += F
    srv.close()
    return res, lat, fl, wall


def serving(dabs, seconds=2.0, rate=50.0, sweep=(5.0, 10.0, 25.0), generations=4, big=0):
    """The served workload with per-request targets: every request's target
    is the energy it reaches alone (computed before the clock, in batched form,
    whose results equal the alone ones); the trace at `rate` is served with
    continuous batching and, on the same arrivals, one request at a time (the
    plain form); every request's (X, E, flips) must be identical in both.  The
    same requests are also served at the `sweep` rates (p50/p99 per rate)."""
    Wcache = {}
    kw = serve_kw(generations)
    traces = {r: serve_requests(r, seconds, 4, big=big if r == rate else 0)
              for r in (rate,) + tuple(sweep)}
    keys = sorted({q[1:] for rq in traces.values() for q in rq})  # (n, instance, solve seed)
    for n, inst, _ in keys:
        if (n, inst) not in Wcache:
            Wcache[(n, inst)] = wl.dense_qubo(n, -1000, 1000, seed=inst)
    targets = {}
    t0 = time.perf_counter()
    for c0 in range(0, len(keys), 48):  # untimed: the energies each reaches alone
        chunk = keys[c0:c0 + 48]
        ctxs = [dabs.Context(Wcache[k[:2]], **kw) for k in chunk]
        out = dabs.batch_solve(ctxs, [256 * generations * k[0] for k in chunk], [k[2] for k in chunk])
        for k, o in zip(chunk, out):
            targets[k] = o[1]
        for c in ctxs:
            c.close()
    t_targets = time.perf_counter() - t0
    progress(f"serving: {len(keys)} targets in {t_targets:.1f}s")
    reqs = traces[rate]
    res, lat, fl, wall = served_trace(dabs, reqs, generations, targets=targets, Wcache=Wcache)
    out = {"workload": f"Poisson {rate}/s for {seconds}s (seed 4), n uniform in "
                       f"{{512,...,8192}} ({SERVE_CATALOG} instances per size, one solve seed "
                       f"per request)" + (f" plus one n={big}" if big else "")
                       + f", 256 searches, budget 256 x {generations} x n flips, at most "
                         f"{generations} generations, recompute seeding",
           "target": "the energy each request reaches alone under the same limits",
           "requests": len(reqs), "served_p50_s": pct(lat, 50), "served_p99_s": pct(lat, 99),
           "served_flips_per_s": fl / wall, "served_wall_s": wall,
           "targets_precompute_s": t_targets}
    progress(f"serving: served {len(reqs)} requests in {wall:.1f}s")
    # plain: one request at a time on the same arrivals
    t0 = time.perf_counter()
    lat2, free_at, same = [], 0.0, True
    fl2 = 0
    for (ta, n, inst, sd) in reqs:
        start = max(ta, free_at)
        now = time.perf_counter() - t0
        if now < start:
            time.sleep(start - now)
        c = dabs.Context(Wcache[(n, inst)], **kw)
        X, E, F = c.solve(256 * generations * n, seed=sd, target=targets[(n, inst, sd)])
        c.close()
        free_at = time.perf_counter() - t0
        lat2.append(free_at - ta)
        fl2 += F
        same = same and res[(n, inst, sd)] == (X.tobytes(), E, F)
    out.update({"plain_p50_s": pct(lat2, 50), "plain_p99_s": pct(lat2, 99),
                "plain_flips_per_s": fl2 / (time.perf_counter() - t0),
                "plain_wall_s": time.perf_counter() - t0,
                "identical_results": bool(same)})
    progress("serving: plain done")
    rates = {}
    for r in sweep:
        rs, lt, f3, w3 = served_trace(dabs, traces[r], generations, targets=targets, Wcache=Wcache)
        ok = all(rs[k] == res[k] for k in rs if k in res)
        rates[str(r)] = {"requests": len(traces[r]), "p50_s": pct(lt, 50), "p99_s": pct(lt, 99),
                         "flips_per_s": f3 / w3, "identical_results": bool(ok)}
        progress(f"serving: rate {r}/s done")
    out["rate_sweep"] = rates
    return out


def run_batched(args, ws, rank, lrank, pg):
    import torch
    from paper_2207_03069_gb300 import build, dabs

    build.build()
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    # the L2 read peak, measured before the workload's buffers exist (later in
    # the run the same measurement has read about a third of it)
    l2 = l2_read_gbs(torch, dev)
    spec = WORKLOADS[args.workload]
    Ws = batched_instances(spec)
    ns = [W.shape[0] for W in Ws]
    kw = {k: spec[k] for k in ("searches", "pools", "pool_cap", "tabu", "s", "b", "seed_mode")}
    seed0 = args.seed + 1000 * rank
    seeds = [seed0 + i for i in range(len(Ws))]
    big = [10**15] * len(Ws)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > L2 (129 MB)

    def flips_of(ctxs):
        return [c.solve_status()["flips"] for c in ctxs]

    progress(f"batched: {len(Ws)} instances ready")
    # ---------------- batched form: one generation of every instance per step
    ctxs = [dabs.Context(W, **kw) for W in Ws]
    bt = dabs.Batch(ctxs, stream)
    bt.begin(big, seeds)
    for _ in range(args.warmup):
        bt.generations(1)
    info0 = bt.info()
    f0 = flips_of(ctxs)
    sampler = ClockSampler(lrank)
    sampler.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)  # untimed: evict L2 between timed steps
        ev[k][0].record(stream)
        bt.generations(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    info1 = bt.info()
    f1 = flips_of(ctxs)
    step_ms = [e[0].elapsed_time(e[1]) for e in ev]
    per_inst = [b - a for a, b in zip(f0, f1)]
    flips = sum(per_inst)
    total_s, flips_all = aggregate(pg, sum(step_ms) * 1e-3, flips)
    value = flips_all / total_s
    launches = info1["launches"] - info0["launches"]
    search_ms = (info1["search_ms"] - info0["search_ms"]) / args.steps
    best_b = [c.solve_best() for c in ctxs]
    bt.close()

    progress(f"batched: {value / 1e6:.1f} M flips/s")
    # ---------------- plain form: the same instances, one instance per launch
    plain = [dabs.Context(W, **kw) for W in Ws]
    for c in plain:
        c.set_stream(stream)
    for c, sd in zip(plain, seeds):
        c.solve_begin(sd, budget=10**15)
    for _ in range(args.warmup):
        for c in plain:
            c.solve_generations(1)
    torch.cuda.synchronize()
    pev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        pev[k][0].record(stream)
        for c in plain:
            c.solve_generations(1)
        pev[k][1].record(stream)
    torch.cuda.synchronize()
    plain_s = sum(e[0].elapsed_time(e[1]) for e in pev) * 1e-3
    fp = flips_of(plain)
    best_p = [c.solve_best() for c in plain]
    identical = all(a[1] == b[1] and np.array_equal(a[0], b[0]) for a, b in zip(best_b, best_p)) \
        and fp == f1
    assert identical, "batched and plain forms disagree"
    plain_value = flips / plain_s
    for c in plain:
        c.close()
    for c in ctxs:
        c.close()

    progress(f"plain: {plain_value / 1e6:.1f} M flips/s, identical={identical}")
    # ---------------- roofline of the batch-search phase (the dominant kernel)
    hbm, peak_kind = peaks()
    row_bytes = sum(f * 2 * n for f, n in zip(per_inst, ns)) / args.steps  # per generation
    achieved = row_bytes / (search_ms * 1e-3) / 1e9
    wset = sum(4 * n * n for n in ns)  # W and -W: the rows one flip may read
    l2_size = torch.cuda.get_device_properties(dev).L2_cache_size
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = sms * 4 * 16 * (clocks.get("sm_max_mhz") or 2070.0) * 1e6
    prof = search_profile("search_batched64.json")
    traffic = prof.get("dram_bytes_per_generation") if prof else None
    from_l2 = rows_from_l2(wset, l2_size, traffic, row_bytes)
    bound = "l2" if from_l2 else "hbm"
    peak = l2 if from_l2 else hbm
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "peak_kind": "measured L2-resident read (64 MiB buffer, library read kernel, "
                             "before the workload's buffers are allocated)"
                             if from_l2 else f"{peak_kind} HBM copy",
                "traffic": traffic,
                "traffic_source": "profiles/search_batched64.json" if prof else None,
                "traffic_per": "generation (all search launches), dram read + write",
                "kernel": "k_batch_search (multi-instance launches, one per variant group)",
                "algorithmic_bytes_per_launch": row_bytes,
                "algorithmic_bytes": "flips x 2n per flip (the int16 row of sigma(x_i) W), summed over instances",
                "launch_ms": search_ms, "search_share_of_step": search_ms / (sum(step_ms) / args.steps),
                "working_set_bytes": wset, "l2_bytes": l2_size,
                "frac_of_hbm": achieved / hbm, "l2_read_gbs_measured": l2, "frac_of_l2": achieved / l2,
                "alu": {"pipe": "ALU (integer compare/min/select/logic), 64 lanes per SM",
                        "peak_lane_ops_per_s": alu_peak,
                        "algorithmic_lane_ops_per_flip": "2n (Step 1 compare, Eq. (4) multiply-add)",
                        "frac_algorithmic": sum(f * 2 * n for f, n in zip(per_inst, ns))
                        / (sum(step_ms) * 1e-3) / alu_peak}}
    cap8 = (prof or {}).get("capture_8x2_full") or {}
    if cap8.get("pipe_pct_of_peak"):
        # the dominant launch's pipe use from the same capture: the bound that binds
        roofline["alu"]["alu_pipe_pct_of_peak_ncu"] = cap8["pipe_pct_of_peak"].get("alu")
        roofline["alu"]["ncu_launch"] = "k_batch_search<8, 2> (2048 < n <= 4096), one launch"

    # ---------------- end to end through the C ABI with host buffers
    pinned = []
    for W in Ws:
        t = torch.empty(W.shape, dtype=torch.int16, pin_memory=True).numpy()
        t[:] = W
        pinned.append(t)
    kw1 = dict(kw, max_generations=1)
    e2e_ctx = [dabs.Context(W, **kw1) for W in Ws]
    dabs.batch_solve(e2e_ctx, big, seeds)  # warm
    e2e_steps = max(3, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_flips = 0
    for k in range(e2e_steps):
        for c, Wp in zip(e2e_ctx, pinned):
            c.load_weights(Wp)  # H2D of the step's inputs
        out = dabs.batch_solve(e2e_ctx, big, [sd + k for sd in seeds])  # best X, E back on the host
        e2e_flips += sum(o[2] for o in out)
    e2e_s = time.perf_counter() - t0
    for c in e2e_ctx:
        c.close()
    e2e = {"value": e2e_flips / e2e_s, "unit": "flips/s",
           "h2d_bytes_per_step": int(sum(2 * n * n for n in ns)),
           "d2h_bytes_per_step": int(sum(n + 8 + 8 for n in ns)),
           "call": "dabs_load_weights for all 64 instances + dabs_batch_solve (one generation) "
                   "per step, best X/E/flips of every instance read back"}

    progress("e2e done")
    extra = {}
    if not args.no_extra and ws == 1:
        extra["time_to_target"] = batched_ttt(dabs, Ws, kw, seeds)
        progress("time to target done")
        if args.trace_seconds > 0:
            extra["serving"] = serving(dabs, seconds=args.trace_seconds, big=args.serve_big,
                                       generations=args.serve_generations,
                                       sweep=tuple(args.serve_sweep))
            progress("serving done")
        rec = recompute_rate(torch, dabs, dev) if not args.no_recompute else None
        if rec:
            mp = os.path.join(ROOT, "MEASURED_PEAKS.json")
            pk = json.load(open(mp))["bf16_tflops"] if os.path.exists(mp) else 1900.0
            rec["peak_tflops"] = pk
            rec["frac"] = rec["tensor_tflops"] / pk
            extra["recompute_tensor"] = rec
        extra["maxcut800"] = single_summary(dabs, torch, dev, "maxcut800", clocks, l2)
        progress("maxcut800 done")
        extra["small_graphs"] = small_graphs(dabs)
        extra["tsp_time_to_target"] = tsp_ttt(dabs, seeds=8)
        progress("small and tsp done")

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, g = oracle_batched_rate(Ws, spec, seed0, args.cpu_seconds, threads)
        cpu = {"value": r, "unit": "flips/s", "cores": threads, "kind": "oracle",
               "sample": f"{g} generation(s) of all {len(Ws)} instances with "
                         f"{spec['sample_searches']} searches each (same W and parameters), "
                         f"about {args.cpu_seconds:.0f} s"}

    if rank == 0:
        line = {"metric": "bit flips/s (batched vs plain, bit-exact)", "value": value,
                "unit": "flips/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": sum(step_ms) / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": spec["desc"], "instances": len(Ws), "n_min": min(ns),
                           "n_max": max(ns), "searches": spec["searches"], "pools": spec["pools"],
                           "pool_cap": spec["pool_cap"], "tabu": spec["tabu"],
                           "s": "%d/%d" % spec["s"], "b": "%d/%d" % spec["b"],
                           "seeding": "recompute (tensor cores)",
                           "form": "batched: one search launch per variant group",
                           "l2": "flushed (256 MiB write) between timed steps; W+(-W) "
                                 f"{wset / 2**20:.0f} MiB > L2",
                           "parallelism": "replicas" if ws > 1 else "single GPU"},
                "plain": {"value": plain_value, "unit": "flips/s", "speedup": value / plain_value,
                          "identical_results": bool(identical),
                          "form": "one instance per launch (its generation as a CUDA graph)"},
                "delta_updates_per_s": sum(f * n for f, n in zip(per_inst, ns)) / (sum(step_ms) * 1e-3),
                "gpu_launches": launches, "launches_per_step": launches / args.steps,
                "clocks": clocks, "roofline": roofline, "e2e": e2e, "cpu_baseline": cpu, **extra}
        print(json.dumps(line), flush=True)
    if pg:
        pg.barrier()


def batched_ttt(dabs, Ws, kw, seeds, generations=3):
    """Time to target, batched vs plain: every instance's target is the energy
    it reaches alone in `generations` generations; all arrive at t = 0.  Plain:
    one solve after another (an instance waits for those before it); batched:
    submitted at once to the continuous-batching server.  Context set-up is
    counted on both sides."""
    kwg = dict(kw, max_generations=generations)
    ctxs = [dabs.Context(W, **kwg) for W in Ws]
    targets = [o[1] for o in dabs.batch_solve(ctxs, [10**15] * len(Ws), seeds)]
    for c in ctxs:
        c.close()
    torch_sync()
    t0 = time.perf_counter()
    plain_ttt = []
    for W, sd, tg in zip(Ws, seeds, targets):
        c = dabs.Context(W, **kwg)
        c.solve(10**15, seed=sd, target=tg)
        c.close()
        plain_ttt.append(time.perf_counter() - t0)
    params = dabs.default_params(**kwg)
    srv = dabs.Server(60 << 30)
    tickets = [srv.submit(W, params, 10**15, sd, target=tg) for W, sd, tg in zip(Ws, seeds, targets)]
    while srv.step(1):
        pass
    served, reached = [], True
    for t, tg in zip(tickets, targets):
        st, X, E, F, L = srv.poll(t)
        served.append(L)
        reached = reached and E <= tg
    srv.close()
    return {"target": f"the energy each instance reaches alone in {generations} generations; "
                      f"all {len(Ws)} arrive at t = 0",
            "plain_p50_s": pct(plain_ttt, 50), "plain_p99_s": pct(plain_ttt, 99),
            "served_p50_s": pct(served, 50), "served_p99_s": pct(served, 99),
            "targets_reached": bool(reached)}


def single_summary(dabs, torch, dev, name, clocks, l2, steps=10):
    """One single-instance workload (autotuned, one generation per step): flips/s,
    ns per flip and the flip kernel against the L2-resident read bandwidth."""
    spec = WORKLOADS[name]
    Wm = make_W(name)
    n = Wm.shape[0]
    kw = {k: spec[k] for k in ("searches", "pools", "pool_cap", "tabu", "s", "b", "seed_mode")}
    ctx = dabs.Context(Wm, **kw)
    st = torch.cuda.Stream(device=dev)
    ctx.set_stream(st)
    ctx.autotune(3)
    ctx.solve_begin(1)
    for _ in range(3):
        ctx.solve_generations(1)
    s0 = ctx.solve_status()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(steps)]
    for k in range(steps):
        ctx.run_stage(dabs.STAGE_OFFSPRING)
        ev[k][0].record(st)
        ctx.run_stage(dabs.STAGE_SEARCH)
        ev[k][1].record(st)
        ctx.run_stage(dabs.STAGE_MERGE)
        ctx.run_stage(dabs.STAGE_FINALIZE)
    torch.cuda.synchronize()
    s1 = ctx.solve_status()
    ms = sum(e[0].elapsed_time(e[1]) for e in ev) / steps
    fl = (s1["flips"] - s0["flips"]) / steps
    ach = fl * 2 * n / (ms * 1e-3) / 1e9
    out = {"workload": spec["desc"], "variant": ctx.variant_name(), "keyed": ctx.keyed()[0],
           "search_flips_per_s": fl / (ms * 1e-3), "ns_per_flip": ms * 1e6 / fl,
           "roofline": {"bound": "l2" if 4 * n * n < torch.cuda.get_device_properties(dev).L2_cache_size else "hbm",
                        "achieved_gbs": ach, "l2_read_gbs_measured": l2, "frac_of_l2": ach / l2}}
    ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dabs", choices=["dabs", "reference"])
    ap.add_argument("--workload", default="batched64", choices=sorted(WORKLOADS))
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-recompute", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the TSP time-to-target, batched and serving measurements")
    ap.add_argument("--trace-seconds", type=float, default=2.0)
    ap.add_argument("--serve-big", type=int, default=0,
                    help="add one instance of this n (e.g. 16384) mid-trace to the served workload")
    ap.add_argument("--serve-generations", type=int, default=4,
                    help="generation limit of every served request (budget 256 x this x n flips)")
    ap.add_argument("--serve-sweep", type=float, nargs="*", default=[5.0, 10.0, 25.0],
                    help="arrival rates (req/s) of the served trace's rate sweep")
    ap.add_argument("--variant", default="", help="force warps x chunks, e.g. 4x1")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, lrank, pg = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
        if pg:
            pg.barrier()
        return

    if WORKLOADS[args.workload].get("kind") == "batched":
        run_batched(args, ws, rank, lrank, pg)
        return
    import torch
    from paper_2207_03069_gb300 import build, dabs

    build.build()
    torch.cuda.set_device(lrank)
    dev = torch.device("cuda", lrank)
    l2 = l2_read_gbs(torch, dev)  # before the workload's buffers exist
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
    l2c = l2_copy_gbs(torch, dev)
    # W and -W (the rows one flip may read) against the L2: rows are L2 hits
    # when they fit (the capture confirms it: DRAM traffic is the search state)
    from_l2 = 4 * n * n <= torch.cuda.get_device_properties(dev).L2_cache_size
    peak = l2 if from_l2 else hbm
    roofline = {"bound": "l2" if from_l2 else "hbm", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": "measured L2-resident read (64 MiB buffer, library read kernel)"
                             if from_l2 else f"{peak_kind} HBM copy",
                "traffic": traffic, "traffic_source": "profiles/search_maxcut800.json" if traffic else None,
                "kernel": "k_batch_search", "algorithmic_bytes_per_launch": algo_bytes,
                "launch_ms": launch_s * 1e3, "search_share_of_step": sum(search_ms) / sum(step_ms),
                "frac_of_hbm": achieved / hbm, "l2_read_gbs_measured": l2,
                "l2_copy_gbs_measured": l2c, "frac_of_l2_copy": achieved / l2c}
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
