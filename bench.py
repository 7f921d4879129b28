"""Benchmark of the D2-clustering assignment step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one hierarchical clustering job of the image-like workload
(N=200,000 bags of 8-16 supports in d=6, Dirichlet(0.5) weights, FP32;
K=64 centroids of 16 supports per segment; segments of 5,000 bags; 10
rounds of (assign, location update) per segment; then the 2,560 segment
centroids are clustered to 64 with 10 more rounds).  Every assign solves
the exact Mallows LP for each (bag, centroid) pair of its segment, so the
unit is one pair LP: 200000*64*10 + 2560*64*10 pair LPs per step.

Prints one JSON line (rank 0).  `value` is device-timed pairs/s with the
inputs resident in HBM; `e2e` is the same through the C-ABI with pinned
host buffers (inputs copied in and labels/centroids copied out inside the
timed region).  `roofline` reports the dominant kernel (k_assign) against
the FP32/INT issue peak; `cpu_baseline` times the FP64 CPU oracle on a
bounded sample on this host's cores.

--impl reference times that oracle itself as the comparison arm.
Multi-GPU (torchrun): every rank clusters its own copy of the workload
(independent problems, no data-path collective) -> weak scaling.
"""
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

WORKLOAD = dict(name="image_like", N=200_000, K=64, seg=5000, iters=10, n=16, d=6)
METRIC = "exact Mallows pairs/s at rel err<=1e-6 vs FP64 oracle"
UNIT = "pairs/s"
L2_BYTES = 129 * 1024 * 1024
ALU_LANES_PER_SM = 128


def pairs_per_step(N, K, seg, iters):
    """Pair LPs solved by the assign steps of one clustering job."""
    total = 0
    n_l = N
    while True:
        M = 1 if n_l <= seg else -(-n_l // seg)
        total += n_l * K * max(iters, 1)
        if M == 1:
            return total
        n_l = M * K


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(step_seconds, pairs_per_rank_step, steps, ws):
    """Whole-job throughput over ranks: max of the ranks' timed totals,
    units all ranks processed (weak scaling: each rank its own workload)."""
    t = reduce_max(float(sum(step_seconds)), ws)
    return pairs_per_rank_step * steps * ws / t, t


def reduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = max(sm)
        loaded = [s for s in sm if s >= 0.5 * hi] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    """Hash of the sources of the screening kernel's translation unit
    (k_screen<32,1> is instantiated in d2_npl1.cu from these files)."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_1302_0435_gb300", "csrc")
    for f in ("d2_npl1.cu", "d2_solve.cuh", "d2_solver.cuh", "d2_internal.h"):
        with open(os.path.join(cs, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per k_assign launch from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "k_assign_image_like.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        prof = json.load(f)
    if prof.get("source_hash") != kernel_source_hash():
        return None
    return prof.get("dram_bytes_per_launch_full")


# ---------------------------------------------------------------- oracle --

def cpu_sample(objs, cents, target_s, seed=7):
    """Time the FP64 oracle on random (object, centroid) pairs of the
    workload, in batches on all host cores, until about target_s seconds."""
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    K = cents.count
    batch = 2048 * cores
    npairs, dt, piv_all, pi_all, pj_all = 0, 0.0, [], [], []
    while dt < target_s and npairs < 20_000_000:
        pi = rng.integers(0, objs.count, size=batch)
        pj = rng.integers(0, K, size=batch)
        t0 = time.perf_counter()
        _, piv = oracle.mallows_pairs(objs, cents, pi, pj, nthreads=cores, return_pivots=True)
        dt += time.perf_counter() - t0
        npairs += batch
        piv_all.append(piv)
        pi_all.append(pi)
        pj_all.append(pj)
    piv = np.concatenate(piv_all)
    pi = np.concatenate(pi_all)
    pj = np.concatenate(pj_all)
    sizes = np.diff(objs.off)[pi]
    ncent = np.diff(cents.off)[pj]
    d = objs.dim
    ops = 2.0 * sizes * ncent * d + piv * (sizes * ncent + 4.0 * (sizes + ncent))
    return dict(value=npairs / dt, unit=UNIT, cores=cores, kind="oracle",
                sample="%d random (bag, centroid) pairs of the workload's first segment set "
                       "(FP64 transportation simplex, %d threads)" % (npairs, cores),
                seconds=dt, mean_pivots=float(piv.mean()), ops_per_pair=float(ops.mean()))


def run_reference(args):
    """The comparison arm: the FP64 oracle itself, on host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1302_0435_gb300 import synth
    objs, cents = synth.image_like(N=WORKLOAD["N"], K=WORKLOAD["K"])
    import oracle
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(11)
    # size one step to about 4 s of oracle work on this host
    cal = 256 * cores
    t0 = time.perf_counter()
    oracle.mallows_pairs(objs, cents, rng.integers(0, objs.count, size=cal),
                         rng.integers(0, cents.count, size=cal), nthreads=cores)
    step_pairs = int(max(cal, 4.0 * cal / max(time.perf_counter() - t0, 1e-3)))

    def step():
        pi = rng.integers(0, objs.count, size=step_pairs)
        pj = rng.integers(0, cents.count, size=step_pairs)
        oracle.mallows_pairs(objs, cents, pi, pj, nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    v = step_pairs * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d random pairs per step of the image_like workload" % step_pairs},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config():
    w = WORKLOAD
    return {"workload": "image_like: N=%d bags, 8-16 supports, d=%d, Dirichlet(0.5), FP32; K=%d "
                        "centroids of %d supports per segment; segments of %d; %d rounds per level; "
                        "top-level merge" % (w["N"], w["d"], w["K"], w["n"], w["seg"], w["iters"]),
            "N": w["N"], "K": w["K"], "seg_size": w["seg"], "iters": w["iters"],
            "pairs_per_step": pairs_per_step(w["N"], w["K"], w["seg"], w["iters"]),
            "l2": "flushed between steps (256 MiB write), not timed"}


# ------------------------------------------------------------------ ours --

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1302_0435_gb300 import build, d2, synth
    build.build()
    d2.load()
    w = WORKLOAD
    objs, cents = synth.image_like(N=w["N"], K=w["K"], seed=1002 + rank)
    ctx = d2.Context(dev.index)
    stream = torch.cuda.current_stream(dev)
    d2.d2_set_stream(ctx, stream)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device=dev))
    ob = d2.bags_from_synth(objs, device=dev)
    T = cents.loc.shape[0]
    out_loc = torch.empty((T, w["d"]), dtype=torch.float64, device=dev)
    out_w = torch.empty(w["K"], dtype=torch.float64, device=dev)
    labels = torch.empty(w["N"], dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    ppstep = pairs_per_step(w["N"], w["K"], w["seg"], w["iters"])

    def step():
        d2.d2_cluster_level(ctx, ob, w["K"], w["seg"], w["iters"], out_loc, out_w, labels)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    launches0 = d2.d2_get_stats()["kernel_launches"]
    barrier(ws)
    torch.cuda.synchronize(dev)
    times = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1) / 1e3)
    torch.cuda.synchronize(dev)
    barrier(ws)
    launches = d2.d2_get_stats()["kernel_launches"] - launches0
    clk = clocks.stop()
    value, t_total = aggregate(times, ppstep, args.steps, ws)

    # dominant kernel: k_assign over the full bag set against one segment's K centroids
    lab1 = torch.empty(w["N"], dtype=torch.int32, device=dev)
    dd1 = torch.empty(w["N"], dtype=torch.float64, device=dev)
    d2.d2_assign(ctx, ob, lab1, dd1)
    torch.cuda.synchronize(dev)
    kt = []
    for _ in range(3):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d2.d2_assign(ctx, ob, lab1, dd1)
        e1.record(stream)
        e1.synchronize()
        kt.append(e0.elapsed_time(e1) / 1e3)
    k_sec = statistics.median(kt)
    k_pairs = w["N"] * w["K"]

    # end to end through the C-ABI with pinned host buffers
    hb = d2.bags_from_synth(objs, pinned=True)
    h_loc = torch.empty((T, w["d"]), dtype=torch.float64).pin_memory()
    h_w = torch.empty(w["K"], dtype=torch.float64).pin_memory()
    h_lab = torch.empty(w["N"], dtype=torch.int32).pin_memory()
    bi = hb.loc.numel() * hb.loc.element_size() + hb.w.numel() * hb.w.element_size() + \
        hb.off.numel() * 8
    bo = h_loc.numel() * 8 + h_w.numel() * 8 + h_lab.numel() * 4
    e2e_steps = max(1, min(args.steps, 2))
    d2.d2_cluster_level(ctx, hb, w["K"], w["seg"], w["iters"], h_loc, h_w, h_lab)
    torch.cuda.synchronize(dev)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d2.d2_cluster_level(ctx, hb, w["K"], w["seg"], w["iters"], h_loc, h_w, h_lab)
    torch.cuda.synchronize(dev)
    e2e_t = reduce_max(time.perf_counter() - t0, ws)
    e2e_v = ppstep * e2e_steps * ws / e2e_t

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0

    cpu = cpu_sample(objs, cents, target_s=args.cpu_seconds) if not args.skip_cpu else None
    serve = None
    if not args.skip_serve:
        serve = serve_measure(dev)
    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu_peak = sms * ALU_LANES_PER_SM * mhz * 1e6 / 1e12  # T lane-ops/s
    roof = None
    if cpu is not None:
        achieved = k_pairs * cpu["ops_per_pair"] / k_sec / 1e12
        roof = {"bound": "alu", "kernel": "k_screen+k_exact (cold d2_assign)", "achieved": achieved,
                "peak": alu_peak,
                "unit": "T lane-ops/s", "frac": achieved / alu_peak,
                "traffic": profiled_traffic(),
                "peak_source": "%d SMs x %d FP32/INT lanes x %.0f MHz (median SM clock under load); "
                               "HBM/bf16 peaks %s in MEASURED_PEAKS.json are not the bound"
                               % (sms, ALU_LANES_PER_SM, mhz, peak_kind),
                "ops_per_pair": cpu["ops_per_pair"], "mean_oracle_pivots": cpu["mean_pivots"],
                "launch_seconds": k_sec, "pairs_per_launch": k_pairs}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 pivots + f64 certify",
        "data": "synthetic", "config": workload_config(),
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)},
        "gpu_launches": int(launches), "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
        "serve": serve,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def serve_measure(dev, n_requests=150, lam_fracs=(0.8,), n_sat=24, seed=1005):
    """Serving workload: Poisson arrivals of assignment requests (log-uniform
    1-4096 bags of 4-64 supports, d=32) against K=1024 resident centroids of
    32 supports, through the continuous-batching server.  Saturated
    throughput comes from a burst of n_sat requests; then requests arrive at
    lam_frac of the saturated request rate and each one's submit-to-done
    latency is recorded.  The plain one-pair-per-launch GPU form
    (d2_mallows_batch with one pair per call) is timed beside it."""
    import threading
    import torch
    from paper_1302_0435_gb300 import d2, synth
    cents, means = synth.serving_centroids(K=1024, seed=seed)
    ctx = d2.Context(dev.index)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device=dev))
    rng = np.random.default_rng(seed + 1)
    K = cents.count
    srv = d2.Server(ctx, slots=8)
    # warm the slots' buffers
    warm = [d2.bags_from_synth(synth.serving_request(rng, means, size=4096)) for _ in range(2)]
    for t in [srv.submit(b) for b in warm]:
        srv.poll(t)
    burst = [d2.bags_from_synth(synth.serving_request(rng, means)) for _ in range(n_sat)]
    t0 = time.perf_counter()
    ts = [srv.submit(b) for b in burst]
    for t in ts:
        srv.poll(t)
    sat_dt = time.perf_counter() - t0
    sat_pairs = sum(b.count for b in burst) * K / sat_dt
    # the request law's mean size (log-uniform on [1, 4096]) sets the
    # request rate that offers a given fraction of the saturated pairs/s
    mean_bags = (4096.0 - 1.0) / np.log(4096.0)
    sat_rps = sat_pairs / (mean_bags * K)
    out = {"workload": "serving: K=1024 resident centroids (n=32, d=32), requests log-uniform "
                       "1-4096 bags of 4-64 supports", "slots": 8,
           "saturated_pairs_per_s": sat_pairs, "saturated_requests_per_s": sat_rps, "levels": []}
    for frac in lam_fracs:
        lam = frac * sat_rps
        reqs = [d2.bags_from_synth(synth.serving_request(rng, means)) for _ in range(n_requests)]
        offered = sum(b.count for b in reqs) * K
        gaps = rng.exponential(1.0 / lam, size=n_requests)
        lat = []
        tickets = []
        done = threading.Event()

        def poller():
            i = 0
            while i < n_requests:
                while len(tickets) <= i:
                    time.sleep(0.0002)
                rc, _, _, ms = srv.poll(tickets[i])
                lat.append(ms)
                i += 1
            done.set()
        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t_start = time.perf_counter()
        nxt = t_start
        for b, gap in zip(reqs, gaps):
            nxt += gap
            wait = nxt - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            tickets.append(srv.submit(b))
        done.wait()
        wall = time.perf_counter() - t_start
        lat = np.array(lat)
        out["levels"].append({"lambda_frac": frac, "requests": n_requests,
                              "offered_pairs": int(offered), "lambda_per_s": lam,
                              "p50_ms": float(np.percentile(lat, 50)),
                              "p99_ms": float(np.percentile(lat, 99)),
                              "pairs_per_s": sum(b.count for b in reqs) * K / wall})
    srv.close()
    # plain form: one pair per launch
    one = synth.serving_request(rng, means, size=64)
    ob = d2.bags_from_synth(one, device=dev)
    po = torch.zeros(1, dtype=torch.int64, device=dev)
    pc = torch.zeros(1, dtype=torch.int64, device=dev)
    dd = torch.empty(1, dtype=torch.float64, device=dev)
    calls = 300
    d2.d2_mallows_batch(ctx, ob, po, pc, dd)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for c in range(calls):
        po.fill_(c % one.count)
        pc.fill_(c % K)
        d2.d2_mallows_batch(ctx, ob, po, pc, dd)
    d2.d2_sync(ctx)
    plain_dt = time.perf_counter() - t0
    out["plain_one_pair_per_launch"] = {"pairs_per_s": calls / plain_dt,
                                        "ms_per_pair": 1e3 * plain_dt / calls}
    ctx.close()
    return out


def run_profile_case(args):
    """Small case for ncu captures: two d2_assign launches, device buffers,
    of the image-like law (N=20,000 bags against K=64 centroids) or of the
    high-dimension law (BF16 d=128 descriptors against K=512 centroids of 64
    supports: the screen reads tensor-core cost tiles)."""
    import torch
    from paper_1302_0435_gb300 import build, d2, synth
    build.build()
    d2.load()
    if args.profile_workload == "image_level":
        # the benchmark step's level driver on profile_n bags (segments of
        # 5,000, 10 rounds): k_screen launches after the first are warm
        # rounds replayed from the CUDA graph
        objs, cents = synth.image_like(N=args.profile_n, K=WORKLOAD["K"])
        ctx = d2.Context(0)
        d2.d2_set_stream(ctx, torch.cuda.current_stream())
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        ob = d2.bags_from_synth(objs, device="cuda:0")
        K = WORKLOAD["K"]
        out_loc = torch.empty((cents.loc.shape[0], objs.dim), dtype=torch.float64, device="cuda:0")
        out_w = torch.empty(K, dtype=torch.float64, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        rc = d2.d2_cluster_level(ctx, ob, K, WORKLOAD["seg"], WORKLOAD["iters"], out_loc, out_w, lab)
        d2.d2_sync(ctx)
        ctx.close()
        print("profile case done: cluster_level rc=%d on %d bags" % (rc, objs.count))
        return 0 if rc == 0 else 1
    if args.profile_workload == "joint_weights":
        # Alg. 1 Step 1 on the image-like law: the bags' nearest-centroid
        # clusters, then the cutting-plane rounds of d2_update_weights
        import time
        objs, cents = synth.image_like(N=args.profile_n, K=WORKLOAD["K"])
        ctx = d2.Context(0)
        d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
        ob = d2.bags_from_synth(objs, device="cuda:0")
        lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
        dd = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
        d2.d2_assign(ctx, ob, lab, dd)
        its = torch.zeros(WORKLOAD["K"], dtype=torch.int32, device="cuda:0")
        d2.d2_sync(ctx)
        s0 = d2.d2_get_stats()
        t0 = time.perf_counter()
        rc = d2.d2_update_weights(ctx, ob, lab, max_iter=1000, tol=1e-9, iters=its)
        d2.d2_sync(ctx)
        dt = time.perf_counter() - t0
        s1 = d2.d2_get_stats()
        ctx.close()
        pe = s1["pairs_exact"] - s0["pairs_exact"]
        print("profile case done: joint weights rc=%d on %d bags, %.3f s, %d rounds, %d master "
              "pivots, %d member solves, %.1f pivots per solve"
              % (rc, objs.count, dt, int(its.max()),
                 s1["joint_master_pivots"] - s0["joint_master_pivots"], pe,
                 (s1["pivots_exact"] - s0["pivots_exact"]) / max(pe, 1)))
        return 0 if rc == 0 else 1
    if args.profile_workload == "high_dim":
        objs, cents = synth.high_dim(N=args.profile_n, K=512)
        ctx = d2.Context(0, tile_budget_mib=1024)  # keep a capture to about 1 GB of tiles
    else:
        objs, cents = synth.image_like(N=args.profile_n, K=WORKLOAD["K"])
        ctx = d2.Context(0)
    d2.d2_set_centroids(ctx, d2.bags_from_synth(cents, device="cuda:0"))
    ob = d2.bags_from_synth(objs, device="cuda:0")
    lab = torch.empty(objs.count, dtype=torch.int32, device="cuda:0")
    dd = torch.empty(objs.count, dtype=torch.float64, device="cuda:0")
    for _ in range(2):
        d2.d2_assign(ctx, ob, lab, dd)
    d2.d2_sync(ctx)
    print("profile case done: %d x %d pairs" % (objs.count, cents.count))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-serve", action="store_true")
    ap.add_argument("--serve-full", action="store_true",
                    help="serving sweep at 0.5/0.8/0.95 of saturation (own JSON line)")
    ap.add_argument("--profile", action="store_true", help="small k_assign case for ncu")
    ap.add_argument("--profile-n", type=int, default=20000)
    ap.add_argument("--profile-workload", default="image_like",
                    choices=["image_like", "image_level", "high_dim", "joint_weights"])
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args)
    if args.serve_full:
        import torch
        from paper_1302_0435_gb300 import build, d2
        build.build()
        d2.load()
        res = serve_measure(torch.device("cuda", 0), n_requests=200, lam_fracs=(0.5, 0.8, 0.95))
        print(json.dumps({"metric": "serve p50/p99 ms", "serve": res}), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
