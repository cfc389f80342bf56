#!/usr/bin/env python
"""Throughput of the GB300 lattice FMM on the uniform 2^20-source / 2^20-target workload.

One step = the whole hot path for one problem: lfmm_plan_create (root box, leaf
level, leaf buckets, cached model-box operators) + lfmm_eval (P2M, M2M, M2L+L2L,
P2P+L2P, binary64 final sum), i.e. (N_src + N_tgt) points solved.  value is
Mpoints/s over the timed steps with inputs resident in device memory; e2e is the
same through the C ABI with pinned host buffers (copies inside the timed region).
L2 (129 MB) is flushed between timed steps by writing a 256 MB buffer.

--impl reference times the CPU oracle (brute force, all host cores) on a bounded
sample of the same workload and reports the same metric, extrapolated.
Multi-GPU (torchrun): independent replicas, one problem per GPU, no collective in
the data path; value = points of all ranks / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpoints/s at rel err≤1e-6 (mixed vs plain FP64 on GPU); serve p50/p99 ms"
WORKLOAD = "uniform_1m: 2^20 distinct sources + 2^20 distinct targets uniform in [0,4096)^2, seed 1"
L2_FLUSH_BYTES = 256 << 20
SM_COUNT = 152
TC_MIN_LEVEL = 6            # library default: levels >= 6 of the fp32 path on the tensor cores
TF32_PER_BF16 = 1.1 / 2.25  # nominal dense tf32 : bf16 tensor throughput


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["lfmm", "reference"], default="lfmm")
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--no-extras", action="store_true", help="skip fp64 comparison, oracle checks, cpu baseline, serving")
    ap.add_argument("--serve-requests", type=int, default=20000,
                    help="requests of the serving stream replayed at their arrival times (0: skip)")
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-pool", type=int, default=1024, help="distinct request contents generated for the replay")
    ap.add_argument("--serve-budget-ms", type=float, default=50.0,
                    help="server overload policy: shed a request after this long waiting for admission")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic work
def near_pairs(src, tgt, info) -> int:
    """Source-target pairs in the same or adjacent leaves (eq. 2.2) of the plan's tree."""
    x0, y0, s, L = info["x0"], info["y0"], info["leaf_side"], info["L"]
    n = 1 << L
    def counts(p):
        bx = (p[:, 0].astype(np.int64) - x0) // s
        by = (p[:, 1].astype(np.int64) - y0) // s
        c = np.zeros((n + 2, n + 2), dtype=np.int64)
        np.add.at(c, (by + 1, bx + 1), 1)
        return c
    cs, ct = counts(src), counts(tgt)
    nb = sum(np.roll(np.roll(cs, dy, 0), dx, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1))
    return int((nb * ct).sum())


def m2l_flops(info, P, levels=None) -> int:
    """Useful flops of M2L (+ fused L2L): 2 P^2 per (target box, interaction-list box) pair over
    levels 2..L (Def. 6.1 lists, truncated at the root boundary), plus 2 P^2 per box for L2L."""
    total = 0
    for lvl in (levels if levels is not None else range(2, info["L"] + 1)):
        n = 1 << lvl
        x = np.arange(n)
        # per axis: number of valid source coordinates for each offset o in [-3, 3]
        valid = {o: ((x + o >= 0) & (x + o < n)) for o in range(-3, 4)}
        pairs = 0
        for px in (0, 1):
            for py in (0, 1):
                mx = (x % 2) == px
                for oy in range(-2 - py, 4 - py):
                    for ox in range(-2 - px, 4 - px):
                        if abs(ox) <= 1 and abs(oy) <= 1:
                            continue
                        cx = int((valid[ox] & mx).sum())
                        cy = int((valid[oy] & ((x % 2) == py)).sum())
                        pairs += cx * cy
        total += 2 * P * P * pairs
        if lvl >= 3:
            total += 2 * P * P * n * n
    return total


def m2l_tc_roofline(info, P, tc_levels, phases, n_prof, peaks, peak_src):
    """Tensor-core M2L (+ fused L2L) of the step's tensor-core levels: useful flops per
    level over the phase's device time per level (which also holds each level's TF32
    split launch, so the fraction is a lower bound for the kernel itself)."""
    ms_level = phases["m2l_tc"][0] / n_prof / max(1, len(tc_levels))
    flops = m2l_flops(info, P, tc_levels) // max(1, len(tc_levels))
    achieved = flops / (ms_level * 1e-3) / 1e12
    peak = float(peaks["bf16_tflops"]) * TF32_PER_BF16
    return {"kernel": "m2l_tma_kernel", "bound": "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_for("m2l_tma_kernel"),
            "peak_basis": f"tf32 dense = measured bf16 burst {peaks['bf16_tflops']} x {TF32_PER_BF16:.3f} "
                          f"(nominal 1.1 / 2.25 PFLOP/s) ({peak_src}); useful flops only, the 3xTF32 split "
                          f"issues 3 MMAs per useful product",
            "levels": tc_levels, "units_per_launch": flops, "ms_per_launch": ms_level,
            "time_basis": "tensor-core phase per level, TF32 split launch included"}


# ---------------------------------------------------------------- reference arm (oracle)
def reference_arm(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_1105_3505_gb300 import workloads
    oracle.build.build_oracle()
    prob = workloads.uniform_1m()
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    rng = np.random.default_rng(2024)
    sample = 256
    for _ in range(args.warmup):
        oracle.lattice_sum(prob.src, prob.f, prob.tgt[rng.choice(nt, 16, replace=False)])
    times = []
    for _ in range(args.steps):
        idx = rng.choice(nt, sample, replace=False)
        t0 = time.perf_counter()
        oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    pairs_per_s = sample * ns / t
    full_s = ns * nt / pairs_per_s
    value = (ns + nt) / full_s / 1e6
    out = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": WORKLOAD, "step": f"oracle brute force on {sample} sampled targets x all sources, "
                                                    "extrapolated to the full solve"},
           "cpu_baseline": {"value": value, "unit": "Mpoints/s", "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"{sample} of {nt} targets x {ns} sources per step"},
           "e2e": {"value": value, "unit": "Mpoints/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def cpu_baseline(prob, budget_s=12.0):
    import oracle
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    rng = np.random.default_rng(77)
    t0 = time.perf_counter()
    oracle.lattice_sum(prob.src, prob.f, prob.tgt[rng.choice(nt, 32, replace=False)])
    per_tgt = (time.perf_counter() - t0) / 32
    m = int(min(nt, max(64, budget_s / max(per_tgt, 1e-9))))
    idx = rng.choice(nt, m, replace=False)
    t0 = time.perf_counter()
    oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    dt = time.perf_counter() - t0
    pairs_per_s = m * ns / dt
    full_s = ns * nt / pairs_per_s
    return {"value": (ns + nt) / full_s / 1e6, "unit": "Mpoints/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{m} of {nt} targets x all {ns} sources ({dt:.1f} s), "
                                        f"extrapolated to the full {ns}x{nt} solve",
            "pairs_per_s": pairs_per_s}


def traffic_for(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    e = d.get(kernel)
    if not e:
        return None
    names = e["source"] if isinstance(e["source"], list) else [e["source"]]
    h = hashlib.sha256()
    for name in names:  # the kernel's file and the headers it includes
        with open(os.path.join(ROOT, "paper_1105_3505_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return e["bytes_per_launch"] if h.hexdigest()[:16] == e.get("source_sha256_16") else None


# ---------------------------------------------------------------- equal-accuracy binary64 arm
def fp64_equal_accuracy(lfmm, timed, s_d, t_d, f_d, u_d, idx, ref, ns, nt, value_mixed, steps):
    """The plain all-binary64 path at the metric's accuracy bar: the smallest p in 5..9
    whose sampled max-norm error is <= 1e-6 at leaf size 64, then that p timed (plan
    create + eval, L2 flushed) at leaf sizes 64, 128 and 256; the best is reported."""
    scale = np.abs(ref).max()
    chosen, errs = None, {}
    for p in range(5, 10):
        ms, _ = timed(s_d, t_d, f_d, u_d, lfmm.make_opts(lfmm.LFMM_FP64, p, 64, 32, 64), 1, 0, sync_ranks=False)
        errs[p] = float(np.abs(u_d.cpu().numpy()[idx] - ref).max() / scale)
        if errs[p] <= 1e-6:
            chosen = p
            break
    if chosen is None:
        return {"error": "no p in 5..9 met 1e-6", "rel_err_by_p": errs}
    rows = {}
    for leaf in (64, 128, 256):
        ms, _ = timed(s_d, t_d, f_d, u_d, lfmm.make_opts(lfmm.LFMM_FP64, chosen, leaf, 32, 64), steps, 1,
                      sync_ranks=False)
        rows[leaf] = {"ms_per_step": ms, "Mpoints_per_s": (ns + nt) / (ms * 1e-3) / 1e6,
                      "rel_err": float(np.abs(u_d.cpu().numpy()[idx] - ref).max() / scale)}
    best = min(rows, key=lambda k: rows[k]["ms_per_step"])
    return {"p": chosen, "leaf_size": best, "value": rows[best]["Mpoints_per_s"], "unit": "Mpoints/s",
            "ms_per_step": rows[best]["ms_per_step"], "rel_err": rows[best]["rel_err"], "by_leaf": rows,
            "rel_err_by_p_leaf64": errs, "mixed_over_fp64": value_mixed / rows[best]["Mpoints_per_s"],
            "note": "plan create + eval, inputs resident, L2 flushed; smallest p meeting rel err <= 1e-6 on the "
                    "128 sampled targets, best leaf size"}


def cold_plan_create(lfmm, s_d, t_d, ns, nt, stream, p):
    """Plan creation with the model-box operators built in the call (fresh cache keys)."""
    import torch
    ts = []
    for ppe in (63, 62, 61):
        o = lfmm.make_opts(lfmm.LFMM_MIXED, p, 64, 32, ppe)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = lfmm.lfmm_plan_create(s_d, ns, t_d, nt, o, stream)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
        lfmm.lfmm_plan_destroy(h)
    return {"median_ms": float(np.median(ts)), "samples_ms": ts,
            "note": "host wall clock of lfmm_plan_create with a cold operator cache (skeletons, T_ofs, M2M/L2L, "
                    "T_ifo and their device images built in the call); the timed step reuses the cache"}


def _timed_steps(fn, steps, warmup, stream, flush):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    evs = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in evs]))


def uniform_4k_leg(lfmm, steps: int = 20, warmup: int = 3):
    """The plain-method case: 4,096 distinct points from [0,256)^2, targets = sources
    (seed 0); plan create + eval per step, binary64 at p = 16 and mixed at p = 8, each
    checked against the full oracle."""
    import torch
    import oracle
    from paper_1105_3505_gb300 import workloads
    prob = workloads.uniform_4k()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    u_d = torch.empty(prob.tgt.shape[0], dtype=torch.float64, device=dev)
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt)
    res = {"workload": "uniform_4k: 4,096 distinct points from [0,256)^2, targets = sources, seed 0"}
    for name, prec, p in (("fp64_p16", lfmm.LFMM_FP64, 16), ("mixed_p8", lfmm.LFMM_MIXED, 8)):
        o = lfmm.make_opts(prec, p, 64, 32, 64)

        def step():
            h = lfmm.lfmm_plan_create(s_d, ns, t_d, nt, o, stream)
            lfmm.lfmm_eval(h, f_d, u_d, stream)
            lfmm.lfmm_plan_destroy(h)

        ms = _timed_steps(step, steps, warmup, stream, flush)
        err = float(np.abs(u_d.cpu().numpy() - ref).max() / np.abs(ref).max())
        res[name] = {"ms_per_step": ms, "Mpoints_per_s": (ns + nt) / (ms * 1e-3) / 1e6, "rel_err_full_oracle": err}
    return res


def clustered_leg(lfmm, steps: int = 5, warmup: int = 2):
    """The clustered workload (4,194,304 points in 64 Gaussian clusters plus 16 segments,
    targets = sources, seed 2) on the pruned tree, mixed at p = 8: plan create + eval per
    step (L2 flushed), the tree build's share of a serial pass, and 256 sampled targets
    against the oracle."""
    import torch
    import oracle
    from paper_1105_3505_gb300 import workloads
    prob = workloads.clustered_4m()
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
    u_d = torch.empty(prob.tgt.shape[0], dtype=torch.float64, device=dev)
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    o = lfmm.make_opts(lfmm.LFMM_MIXED, 8, 64, 32, 64)

    def step():
        h = lfmm.lfmm_plan_create(s_d, ns, t_d, nt, o, stream)
        lfmm.lfmm_eval(h, f_d, u_d, stream)
        lfmm.lfmm_plan_destroy(h)

    ms = _timed_steps(step, steps, warmup, stream, flush)
    u = u_d.cpu().numpy()
    lfmm.lfmm_profile_enable(True)
    lfmm.lfmm_profile_read(reset=True)
    os_ = lfmm.make_opts(lfmm.LFMM_MIXED, 8, 64, 32, 64, serial=True)
    h = lfmm.lfmm_plan_create(s_d, ns, t_d, nt, os_, stream)
    lfmm.lfmm_eval(h, f_d, u_d, stream)
    info = lfmm.lfmm_plan_get_info(h)
    torch.cuda.synchronize()
    lfmm.lfmm_plan_destroy(h)
    ph = lfmm.lfmm_profile_read(reset=True)
    lfmm.lfmm_profile_enable(False)
    total = sum(v[0] for v in ph.values())
    idx = np.random.default_rng(321).choice(nt, 256, replace=False)
    ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
    return {"workload": "clustered_4m: 4,194,304 points, 64 Gaussian clusters (sigma 200) + 1% on 16 segments, "
                        "targets = sources, seed 2",
            "ms_per_step": ms, "Mpoints_per_s": (ns + nt) / (ms * 1e-3) / 1e6, "tree": info["tree"],
            "levels": info["L"], "leaf_side": info["leaf_side"], "boxes": info["n_boxes"],
            "phases_ms_serial": {k: v[0] for k, v in ph.items()},
            "tree_share_serial": ph["tree"][0] / total if total > 0 else None,
            "rel_err_256_sampled": float(np.abs(u[idx] - ref).max() / np.abs(ref).max())}


# ---------------------------------------------------------------- serving leg
def _serve_gen(task):
    seed, n, i = task
    from paper_1105_3505_gb300 import workloads
    return workloads.serve_request(workloads.serve_schedule(seed=seed, n_requests=n), i)


def serve_leg(lfmm, n_requests: int, slots: int, pool_size: int = 1024, budget_ms: float = 50.0,
              check: int = 24):
    """Replays the serving stream against an lfmm server: n_requests Poisson arrivals at
    2,000 req/s (the whole 20,000-request stream by default), each submitted at its
    arrival time; latency = submit -> result in host memory.  Request contents (N_src
    log-uniform in [1e3, 1e6], uniform or four clusters, N_tgt = N_src/4, tolerance 1e-6
    or 1e-10) are the first pool_size requests of the stream, generated once and reused
    in turn (request i carries request i mod pool_size's points, charges and tolerance),
    so that the replay needs seconds of host time rather than minutes.  The server runs
    its overload policy with a latency budget of budget_ms: a request whose predicted wait
    exceeds it is refused at submit, and one that waits longer anyway is shed (both
    LFMM_EBUSY)."""
    import multiprocessing as mp
    import threading
    import oracle
    from paper_1105_3505_gb300 import workloads
    seed = 4
    pool_size = min(pool_size, n_requests)
    sched = workloads.serve_schedule(seed=seed, n_requests=n_requests)
    t_gen = time.perf_counter()
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        reqs = pool.map(_serve_gen, [(seed, pool_size, i) for i in range(pool_size)], chunksize=4)
        warm = pool.map(_serve_gen, [(seed + 101, 24, i) for i in range(24)], chunksize=2)
    t_gen = time.perf_counter() - t_gen
    # requests arrive in page-locked host buffers (as a serving front end would hand
    # them over): their copies are then asynchronous DMA instead of staged pageable copies
    import torch
    t_pin = time.perf_counter()
    pinned = []
    for r in reqs:
        pr = r.problem
        pinned.append((torch.from_numpy(pr.src).pin_memory(), torch.from_numpy(pr.tgt).pin_memory(),
                       torch.from_numpy(pr.f).pin_memory(),
                       torch.empty(pr.tgt.shape[0], dtype=torch.float64).pin_memory()))
    t_pin = time.perf_counter() - t_pin
    arrival = sched["arrival_s"]
    rng = np.random.default_rng(7)
    checked_idx = set(int(i) for i in rng.choice(n_requests, min(4 * check, n_requests), replace=False))
    with lfmm.Server(n_slots=slots) as sv:
        # warm start: model-box operators of both precisions at the leaf sides that occur
        for r in warm:
            sv.wait(sv.submit(r.problem.src, r.problem.tgt, r.problem.f, r.tol))
        sv.set_limits(max_pending=0, max_queue_ms=budget_ms)
        tickets = [None] * n_requests
        stats = [None] * n_requests
        done = [threading.Event() for _ in range(n_requests)]
        kept = {}
        submit_err = [0]

        def waiter():
            for i in range(n_requests):
                while tickets[i] is None:
                    time.sleep(0.0002)
                if tickets[i] < 0:
                    stats[i] = {"status": -tickets[i]}
                else:
                    u, st = sv.wait_stats(tickets[i])
                    stats[i] = st
                    if u is not None and i in checked_idx:
                        kept[i] = u.numpy().copy()
                done[i].set()

        th = threading.Thread(target=waiter)
        th.start()
        t0 = time.perf_counter()
        for i in range(n_requests):
            k = i % pool_size
            if i >= pool_size:
                done[i - pool_size].wait()  # its output buffer is reused
            delay = t0 + arrival[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            r, (ps, pt, pf, pu) = reqs[k], pinned[k]
            try:
                tickets[i] = sv.submit(ps, pt, pf, r.tol, out=pu)
            except lfmm.LfmmError as e:
                submit_err[0] += 1
                tickets[i] = -e.status
        th.join()
        t_end = time.perf_counter()
    codes = np.array([st["status"] for st in stats])
    ok = codes == lfmm.LFMM_OK
    tol = np.array([reqs[i % pool_size].tol for i in range(n_requests)])
    pts_all = np.array([reqs[i % pool_size].problem.n_points for i in range(n_requests)])
    served = np.nonzero(ok)[0]
    lat = np.array([stats[i]["total_ms"] for i in served])
    qms = np.array([stats[i]["queue_ms"] for i in served])
    rms = np.array([stats[i]["run_ms"] for i in served])
    tight = tol[served] < 1e-6
    span = t_end - t0
    errs = []
    for i in sorted(kept)[:check]:
        r = reqs[i % pool_size]
        idx = np.random.default_rng(int(i)).choice(r.problem.tgt.shape[0], min(64, r.problem.tgt.shape[0]),
                                                   replace=False)
        ref = oracle.lattice_sum(r.problem.src, r.problem.f, r.problem.tgt[idx])
        errs.append((r.tol, float(np.abs(kept[i][idx] - ref).max() / np.abs(ref).max())))

    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else None

    return {"requests": n_requests, "served": int(ok.sum()), "shed": int((codes == lfmm.LFMM_EBUSY).sum()),
            "failed_other": int((~ok & (codes != lfmm.LFMM_EBUSY)).sum()), "refused_at_submit": submit_err[0],
            "served_1e-6": int((ok & (tol >= 1e-6)).sum()), "served_1e-10": int((ok & (tol < 1e-6)).sum()),
            "offered_1e-6": int((tol >= 1e-6).sum()), "offered_1e-10": int((tol < 1e-6).sum()),
            "rate_req_per_s": 2000.0, "slots": slots, "latency_budget_ms": budget_ms,
            "arrival_span_s": float(arrival[-1]), "completion_span_s": span,
            "offered_Mpoints_per_s": float(pts_all.sum() / arrival[-1] / 1e6),
            "served_Mpoints_per_s": float(pts_all[served].sum() / span / 1e6),
            "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99),
            "p50_ms_mixed": pct(lat[~tight], 50), "p99_ms_mixed": pct(lat[~tight], 99),
            "p50_ms_df": pct(lat[tight], 50), "p99_ms_df": pct(lat[tight], 99),
            "queue_p50_ms": pct(qms, 50), "queue_p99_ms": pct(qms, 99),
            "run_p50_ms_mixed": pct(rms[~tight], 50), "run_p50_ms_df": pct(rms[tight], 50),
            "run_p99_ms_mixed": pct(rms[~tight], 99), "run_p99_ms_df": pct(rms[tight], 99),
            "checked": len(errs), "max_rel_err_1e-6_requests": max([e for t, e in errs if t >= 1e-6], default=None),
            "max_rel_err_1e-10_requests": max([e for t, e in errs if t < 1e-6], default=None),
            "generation_s": t_gen, "pin_s": t_pin, "pool": pool_size,
            "note": f"the whole {n_requests}-request stream (seed 4) submitted at its arrival times; contents of "
                    f"the first {pool_size} requests reused in turn; overload policy with a {budget_ms} ms latency "
                    "budget (refused at submit when the predicted wait exceeds it, shed when the wait does); tol "
                    "1e-6 -> mixed path p = 8, tol 1e-10 -> float-float path p = 16 (leaf 192)"}


# ---------------------------------------------------------------- batched forest leg
def forest_leg(lfmm, steps: int = 5, warmup: int = 2):
    """The batched workload: 4,096 independent problems (N_src log-uniform in [512, 8192],
    box side 4 sqrt(N), targets = sources) in one forest plan, mixed path with p and the
    leaf size from the autotuner (rel. error <= 1e-6); one step = lfmm_forest_create +
    lfmm_eval with inputs resident in device memory, L2 flushed before each step; also
    the evaluation alone, eager and as a recorded CUDA graph; 24 problems checked in
    full against the oracle."""
    import torch
    import oracle
    from paper_1105_3505_gb300 import workloads
    t_gen = time.perf_counter()
    probs = workloads.forest_4096()
    t_gen = time.perf_counter() - t_gen
    src = np.ascontiguousarray(np.concatenate([p.src for p in probs]))
    tgt = np.ascontiguousarray(np.concatenate([p.tgt for p in probs]))
    f = np.concatenate([p.f for p in probs])
    so = np.concatenate([[0], np.cumsum([p.src.shape[0] for p in probs])]).astype(np.int64)
    to = np.concatenate([[0], np.cumsum([p.tgt.shape[0] for p in probs])]).astype(np.int64)
    dev = torch.device("cuda:0")
    s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (src, tgt, f))
    u_d = torch.empty(tgt.shape[0], dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # p, leaf size and M2L path picked by the autotuner for rel. error <= 1e-6
    t_tune = time.perf_counter()
    opts, tune = lfmm.autotune(s_d, t_d, 1e-6, so, to, stream=stream)
    t_tune = time.perf_counter() - t_tune

    def step():
        h = lfmm.lfmm_forest_create(s_d, so, t_d, to, opts, stream)
        lfmm.lfmm_eval(h, f_d, u_d, stream)
        return h

    for _ in range(warmup):
        lfmm.lfmm_plan_destroy(step())
    torch.cuda.synchronize()
    evs = []
    for k in range(steps):
        flush.fill_(k & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        h = step()
        b.record(stream)
        lfmm.lfmm_plan_destroy(h)
        evs.append((a, b))
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    h = step()
    info = lfmm.lfmm_plan_get_info(h)
    torch.cuda.synchronize()
    u = u_d.cpu().numpy()
    # evaluation alone on the built forest: eager launches (one per level and sweep step),
    # the recorded CUDA graph, and one persistent launch per sweep for comparison
    ev_ms = {}
    for mode in ("eager", "graph", "persistent"):
        lfmm.lfmm_plan_set_flags(h, {"eager": 0, "graph": lfmm.LFMM_FLAG_GRAPH,
                                     "persistent": lfmm.LFMM_FLAG_PERSISTENT}[mode])
        for _ in range(2):
            lfmm.lfmm_eval(h, f_d, u_d, stream)
        torch.cuda.synchronize()
        evs2 = []
        for k in range(steps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lfmm.lfmm_eval(h, f_d, u_d, stream)
            b.record(stream)
            evs2.append((a, b))
        torch.cuda.synchronize()
        ev_ms[mode] = float(np.median([a.elapsed_time(b) for a, b in evs2]))
    lfmm.lfmm_plan_destroy(h)
    err = 0.0
    for i in np.random.default_rng(11).choice(len(probs), 24, replace=False):
        ref = oracle.lattice_sum(probs[i].src, probs[i].f, probs[i].tgt)
        err = max(err, float(np.abs(u[to[i]:to[i + 1]] - ref).max() / np.abs(ref).max()))
    pts = int(src.shape[0] + tgt.shape[0])
    return {"workload": "forest_4096: 4,096 problems, N log-uniform in [512, 8192], side 4 sqrt(N), targets = sources, seed 3",
            "points": pts, "ms_per_step": ms, "Mpoints_per_s": pts / (ms * 1e-3) / 1e6,
            "leaf_side": info["leaf_side"], "boxes": info["n_boxes"], "max_rel_err_24_problems": err,
            "step": "lfmm_forest_create + lfmm_eval", "generation_s": t_gen,
            "autotune": {"p": tune["p"], "leaf_size": tune["leaf_size"], "candidates": tune["candidates"],
                         "tuned_rel_err": tune["rel_err"], "seconds": t_tune},
            "eval_only_ms": ev_ms}


def eval_leg(lfmm, steps: int = 20, warmup: int = 3):
    """Evaluation alone (plan built once, outside the timed region), eager launches vs
    the plan's recorded CUDA graph (LFMM_FLAG_GRAPH), on uniform_1m (mixed, p = 8) and
    uniform_4k (binary64, p = 16); L2 flushed before every timed evaluation."""
    import torch
    from paper_1105_3505_gb300 import workloads
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    res = {}
    for name, prob, prec, p in (("uniform_1m_mixed_p8", workloads.uniform_1m(), lfmm.LFMM_MIXED, 8),
                                ("uniform_4k_fp64_p16", workloads.uniform_4k(), lfmm.LFMM_FP64, 16)):
        s_d, t_d, f_d = (torch.from_numpy(a).to(dev) for a in (prob.src, prob.tgt, prob.f))
        u_d = torch.empty(prob.tgt.shape[0], dtype=torch.float64, device=dev)
        pts = prob.src.shape[0] + prob.tgt.shape[0]
        row = {}
        ref = None
        for mode in ("eager", "graph"):
            o = lfmm.make_opts(prec, p, 64, 32, 64, graph=(mode == "graph"))
            h = lfmm.lfmm_plan_create(s_d, prob.src.shape[0], t_d, prob.tgt.shape[0], o, stream)
            for _ in range(warmup):
                lfmm.lfmm_eval(h, f_d, u_d, stream)
            torch.cuda.synchronize()
            evs = []
            for k in range(steps):
                flush.fill_(k & 0xFF)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                lfmm.lfmm_eval(h, f_d, u_d, stream)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
            lfmm.lfmm_plan_destroy(h)
            ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
            u = u_d.cpu().numpy()
            if ref is None:
                ref = u
            row[mode] = {"ms": ms, "Mpoints_per_s": pts / (ms * 1e-3) / 1e6}
        # two plans of the same points may order a leaf's points differently
        row["max_rel_diff"] = float(np.abs(ref - u).max() / np.abs(ref).max())
        res[name] = row
    return res


def multi_leg(lfmm, k: int = 8, steps: int = 10, warmup: int = 2):
    """k charge vectors on the uniform_1m plan (mixed, p = 8): lfmm_eval_multi against k
    calls of lfmm_eval (plan built once, L2 flushed before each timed call), and the
    near-field time per vector of the batched pass against the single-vector kernel."""
    import torch
    from paper_1105_3505_gb300 import workloads
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    prob = workloads.uniform_1m()
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    rng = np.random.default_rng(5)
    F = np.stack([workloads.zero_sum(rng.standard_normal(ns)) for _ in range(k)])
    s_d, t_d, F_d = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (prob.src, prob.tgt, F))
    U_d = torch.empty((k, nt), dtype=torch.float64, device=dev)
    o = lfmm.make_opts(lfmm.LFMM_MIXED, 8, 64, 32, 64)
    h = lfmm.lfmm_plan_create(s_d, ns, t_d, nt, o, stream)

    def timed(fn):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        evs = []
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return float(np.median([a.elapsed_time(b) for a, b in evs]))

    def multi():
        lfmm.load().lfmm_eval_multi(h, F_d.data_ptr(), k, U_d.data_ptr(), stream.cuda_stream)

    def singles():
        for r in range(k):
            lfmm.lfmm_eval(h, F_d[r], U_d[r], stream)

    ms_multi, ms_single = timed(multi), timed(singles)
    # near-field device time per vector: batched pass vs single-vector kernel (serial order)
    lfmm.lfmm_plan_set_flags(h, lfmm.LFMM_FLAG_SERIAL)
    lfmm.lfmm_profile_enable(True)
    lfmm.lfmm_profile_read(reset=True)
    multi()
    torch.cuda.synchronize()
    ph_m = lfmm.lfmm_profile_read(reset=True)
    lfmm.lfmm_eval(h, F_d[0], U_d[0], stream)
    torch.cuda.synchronize()
    ph_s = lfmm.lfmm_profile_read(reset=True)
    lfmm.lfmm_profile_enable(False)
    lfmm.lfmm_plan_destroy(h)
    pairs = 150228790  # near-field pairs of uniform_1m (per vector)
    p2p_m = ph_m["p2p"][0] / k
    return {"k": k, "ms_eval_multi": ms_multi, "ms_k_evals": ms_single, "speedup": ms_single / ms_multi,
            "Mpoints_per_s_per_vector_multi": k * (ns + nt) / (ms_multi * 1e-3) / 1e6,
            "near_field_us_per_vector": {"batched": p2p_m * 1e3, "single": ph_s["p2p"][0] * 1e3},
            "near_field_Gpair_fma_per_s": pairs * k / (ph_m["p2p"][0] * 1e-3) / 1e9,
            "note": "evaluation only; four vectors per near-field pass share each phi table lookup"}


def solvers_leg(lfmm):
    """The two solvers built on the lattice FMM, wall clock (host-driven GMRES):
    a Dirichlet problem on a digital disk of radius 1500 (about 7.07e6 nodes, 8.5e3
    boundary nodes; data x^2 - y^2 + 3 x y, scaled) and a lattice with 10^4 changed bars in
    a 2048^2 box; both with the float-float path at p = 16.  Also the GPU quadrature of
    phi near the origin (binary64) for radii 8, 16 and 32."""
    import time
    import torch
    from paper_1105_3505_gb300.bvp import LatticeDirichlet
    from paper_1105_3505_gb300.inclusions import LatticeInclusions
    res = {}
    r = 1500
    x, y = np.meshgrid(np.arange(-r, r + 1), np.arange(-r, r + 1), indexing="ij")
    keep = x * x + y * y <= r * r
    nodes = np.stack([x[keep], y[keep]], axis=1)
    t0 = time.perf_counter()
    bv = LatticeDirichlet(nodes)
    t1 = time.perf_counter()
    gx, gy = bv.gamma[:, 0].astype(np.float64), bv.gamma[:, 1].astype(np.float64)
    bv.solve((gx * gx - gy * gy + 3.0 * gx * gy) / r ** 2, tol=1e-12)
    t2 = time.perf_counter()
    u = bv.potential()
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    ox, oy = bv.omega[:, 0].astype(np.float64), bv.omega[:, 1].astype(np.float64)
    err = float(np.abs(u - (ox * ox - oy * oy + 3.0 * ox * oy) / r ** 2).max())
    res["dirichlet_disk_r1500"] = {"interior_nodes": int(bv.omega.shape[0]), "boundary_nodes": int(bv.gamma.shape[0]),
                                   "setup_ms": (t1 - t0) * 1e3, "gmres_iterations": bv.iterations,
                                   "solve_ms": (t2 - t1) * 1e3, "ms_per_iteration": (t2 - t1) * 1e3 / bv.iterations,
                                   "interior_eval_ms": (t3 - t2) * 1e3, "residual": bv.residual,
                                   "max_abs_err_vs_harmonic_data": err}
    bv.close()
    rng = np.random.default_rng(11)
    seen, bars, delta = set(), [], []
    while len(bars) < 10000:
        x0, y0 = (int(v) for v in rng.integers(0, 2048, size=2))
        horiz = bool(rng.integers(0, 2))
        key = (x0, y0, x0 + horiz, y0 + (not horiz))
        if key in seen:
            continue
        seen.add(key)
        bars.append(key)
        delta.append(-1.0 if rng.random() < 0.5 else float(rng.uniform(0.5, 3.0)))
    t0 = time.perf_counter()
    li = LatticeInclusions(np.array(bars), np.array(delta))
    t1 = time.perf_counter()
    li.solve(1.0, 0.5, tol=1e-12)
    t2 = time.perf_counter()
    res["inclusions_10k_bars"] = {"nodes": int(li.nodes.shape[0]), "setup_ms": (t1 - t0) * 1e3,
                                  "gmres_iterations": li.iterations, "solve_ms": (t2 - t1) * 1e3,
                                  "ms_per_iteration": (t2 - t1) * 1e3 / li.iterations, "residual": li.residual}
    li.close()
    # phi near the origin by the 2-D quadrature (binary64), 5-point and anisotropic operators
    for name, offs, w in (("phi_quadrature_5point", [[1, 0], [0, 1]], [1.0, 1.0]),
                          ("phi_quadrature_anisotropic_1_20", [[1, 0], [0, 1]], [1.0, 20.0])):
        row = {}
        for R in (8, 16, 32):
            lfmm.lfmm_phi_quadrature(offs, w, 2)  # warm-up
            t0 = time.perf_counter()
            lfmm.lfmm_phi_quadrature(offs, w, R)
            dt = time.perf_counter() - t0
            row[f"R{R}"] = {"entries": (2 * R + 1) ** 2, "ms": dt * 1e3}
        res[name] = row
    return res


# ---------------------------------------------------------------- replicas
def replica_throughput(ms_local, points_per_rank: int, world: int, device=None):
    """Whole-job throughput of `world` independent replicas: every rank solved
    points_per_rank points per step; the job's step time is the slowest rank's
    (max over ranks), so value = world * points / max_ms.  Returns (max ms list,
    Mpoints/s list)."""
    import torch
    import torch.distributed as dist
    ms = [float(m) for m in ms_local]
    if world > 1:
        t = torch.tensor(ms, dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = [float(v) for v in t.tolist()]
    return ms, [world * points_per_rank / (m * 1e-3) / 1e6 for m in ms]


# ---------------------------------------------------------------- main arm
def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    from paper_1105_3505_gb300 import build as lbuild
    if rank == 0:
        lbuild.build()
    if world > 1:
        dist.barrier()
    from paper_1105_3505_gb300 import lfmm, workloads
    lfmm.load()

    prob = workloads.uniform_1m()
    ns, nt = prob.src.shape[0], prob.tgt.shape[0]
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    s_d = torch.from_numpy(prob.src).to(dev)
    t_d = torch.from_numpy(prob.tgt).to(dev)
    f_d = torch.from_numpy(prob.f).to(dev)
    u_d = torch.empty(nt, dtype=torch.float64, device=dev)
    s_h = torch.from_numpy(prob.src).pin_memory()
    t_h = torch.from_numpy(prob.tgt).pin_memory()
    f_h = torch.from_numpy(prob.f).pin_memory()
    u_h = torch.empty(nt, dtype=torch.float64).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    opts = lfmm.make_opts(lfmm.LFMM_MIXED, args.p, 64, 32, 64)

    def step(src, tgt, f, u, o):
        h = lfmm.lfmm_plan_create(src, ns, tgt, nt, o, stream)
        lfmm.lfmm_eval(h, f, u, stream)
        return h

    def solve_step(src, tgt, f, u, o):
        lfmm.lfmm_solve(src, tgt, f, u, o, stream)
        return None

    def timed(src, tgt, f, u, o, steps, warmup, sync_ranks=True, fn=None):
        fn = fn or step
        for _ in range(warmup):
            h = fn(src, tgt, f, u, o)
            if h is not None:
                lfmm.lfmm_plan_destroy(h)
        torch.cuda.synchronize()
        if world > 1 and sync_ranks:
            dist.barrier()
        torch.cuda.synchronize()
        evs = []
        launches0 = lfmm.lfmm_launch_count()
        for k in range(steps):
            flush.fill_(k & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            h = fn(src, tgt, f, u, o)
            b.record(stream)
            if h is not None:
                lfmm.lfmm_plan_destroy(h)
            evs.append((a, b))
        torch.cuda.synchronize()
        launches = lfmm.lfmm_launch_count() - launches0
        if world > 1 and sync_ranks:
            dist.barrier()
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        return ms, launches

    # device-resident inputs (the value)
    sampler = ClockSampler(local_rank) if rank == 0 else None
    ms, launches = timed(s_d, t_d, f_d, u_d, opts, args.steps, args.warmup)
    clocks = sampler.stop() if sampler else None
    # e2e through host buffers: the one-shot call (f uploads beside the tree build)
    ms_e2e, _ = timed(s_h, t_h, f_h, u_h, opts, args.steps, max(1, args.warmup // 2), fn=solve_step)
    (ms, ms_e2e), (value, value_e2e) = replica_throughput([ms, ms_e2e], ns + nt, world, dev)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # per-phase device time: CUDA events the library records on `stream` around each
    # phase, over a second pass of the same timed loop (L2 flushed before every step)
    # (serial order, so that each phase's kernels are timed alone on the device)
    lfmm.lfmm_profile_enable(True)
    lfmm.lfmm_profile_read(reset=True)
    n_prof = max(3, min(args.steps, 10))
    opts_serial = lfmm.make_opts(lfmm.LFMM_MIXED, args.p, 64, 32, 64, serial=True)
    for _ in range(n_prof):
        flush.fill_(1)
        lfmm.lfmm_plan_destroy(step(s_d, t_d, f_d, u_d, opts_serial))
    phases = lfmm.lfmm_profile_read(reset=True)
    lfmm.lfmm_profile_enable(False)
    phase_ms = {k: v[0] / n_prof for k, v in phases.items()}
    phase_launch_ms = {k: v[0] / v[1] for k, v in phases.items() if v[1] > 0}

    h = step(s_d, t_d, f_d, u_d, opts)
    info = lfmm.lfmm_plan_get_info(h)
    torch.cuda.synchronize()
    lfmm.lfmm_plan_destroy(h)
    u_mixed = u_d.cpu().numpy()
    peaks, peak_src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))

    # roofline of the dominant kernel: the longest single kernel launch of the step
    P = 4 * (args.p - 1)
    tc_levels = [lvl for lvl in range(2, info["L"] + 1) if lvl >= TC_MIN_LEVEL]
    cands = {k: phase_launch_ms[k] for k in ("p2p", "m2l_tc", "p2m") if k in phase_launch_ms}
    dom = max(cands, key=cands.get)
    t_launch = cands[dom] * 1e-3
    if dom == "p2p":
        # one 4-byte table load + one multiply-add per pair: the binding pipe is the
        # shared-memory load path, 32 lanes per clock per SM
        pairs = near_pairs(prob.src, prob.tgt, info)
        achieved = pairs / t_launch / 1e9
        peak = SM_COUNT * 32 * sm_mhz * 1e6 / 1e9
        roof = {"kernel": "p2p_strip_kernel<float,32>", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Gpairs/s", "frac": achieved / peak, "traffic": traffic_for("p2p_strip_kernel"),
                "peak_basis": f"shared-memory loads: 152 SMs x 32 lanes/clk x {sm_mhz:.0f} MHz ({peak_src})",
                "units_per_launch": pairs, "ms_per_launch": cands[dom]}
    elif dom == "m2l_tc":
        roof = m2l_tc_roofline(info, P, tc_levels, phases, n_prof, peaks, peak_src)
    else:
        flops = 2 * P * ns
        achieved = flops / t_launch / 1e12
        peak = SM_COUNT * 128 * 2 * sm_mhz * 1e6 / 1e12
        roof = {"kernel": "p2m_kernel<float,32>", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic_for("p2m_kernel"),
                "peak_basis": f"FP32 FMA: 152 SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz ({peak_src})",
                "units_per_launch": flops, "ms_per_launch": cands[dom]}

    out = {"metric": METRIC, "value": value, "unit": "Mpoints/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "p": args.p, "P": info["P"], "leaf_size": 64, "leaf_side": info["leaf_side"],
                      "levels": info["L"], "precision": "mixed (fp32 near/far, fp64 final sum)",
                      "step": "lfmm_plan_create + lfmm_eval", "l2": "flushed between timed steps (256 MB write)",
                      "parallelism": f"replicas x{world}"},
           "e2e": {"value": value_e2e, "unit": "Mpoints/s", "ms_per_step": ms_e2e, "call": "lfmm_solve",
                   "h2d_bytes_per_step": int(s_h.numel() * 4 + t_h.numel() * 4 + f_h.numel() * 8),
                   "d2h_bytes_per_step": int(u_h.numel() * 8)},
           "gpu_launches": int(launches),
           "roofline": roof,
           "roofline_m2l_tc": (m2l_tc_roofline(info, P, tc_levels, phases, n_prof, peaks, peak_src)
                               if tc_levels and phases["m2l_tc"][1] > 0 else None),
           "phases_ms": phase_ms,
           "phases_note": "per-phase device time from CUDA events around each phase, over a pass of the same "
                          "step with LFMM_FLAG_SERIAL (every kernel alone on the device); the timed value runs "
                          "the near field beside the far field",
           "clocks": clocks}

    if not args.no_extras:
        import oracle
        idx = np.random.default_rng(123).choice(nt, 128, replace=False)
        ref = oracle.lattice_sum(prob.src, prob.f, prob.tgt[idx])
        scale = np.abs(ref).max()
        out["rel_err"] = float(np.abs(u_mixed[idx] - ref).max() / scale)
        # the plain all-binary64 path at the same accuracy bar (rel err <= 1e-6): the
        # smallest p that meets it on the sampled targets, at its best leaf size
        out["fp64_at_1e-6"] = fp64_equal_accuracy(lfmm, timed, s_d, t_d, f_d, u_d, idx, ref, ns, nt, value,
                                                  max(3, args.steps // 4))
        # the mixed path at the configuration's second order, p = 16 (P_pad = 64)
        o16 = lfmm.make_opts(lfmm.LFMM_MIXED, 16, 64, 32, 64)
        ms16, _ = timed(s_d, t_d, f_d, u_d, o16, max(3, args.steps // 4), 1, sync_ranks=False)
        u16 = u_d.cpu().numpy()
        out["mixed_p16"] = {"value": (ns + nt) / (ms16 * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms16,
                            "rel_err": float(np.abs(u16[idx] - ref).max() / scale), "leaf_size": 64,
                            "note": "plan create + eval, inputs resident, L2 flushed"}
        # plan creation with the operator cache cold (a proxies_per_edge not used before
        # gives a new cache key: skeletons, operators and their device images are built)
        out["cold_plan_create_ms"] = cold_plan_create(lfmm, s_d, t_d, ns, nt, stream, args.p)
        # the plain all-binary64 path at p = 16 on the same workload
        o64 = lfmm.make_opts(lfmm.LFMM_FP64, 16, 64, 32, 64)
        ms64, _ = timed(s_d, t_d, f_d, u_d, o64, max(2, args.steps // 5), 1, sync_ranks=False)
        u64 = u_d.cpu().numpy()
        out["fp64_plain_p16"] = {"value": (ns + nt) / (ms64 * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms64,
                                 "rel_err": float(np.abs(u64[idx] - ref).max() / scale), "leaf_size": 64}
        # the same at its best leaf size, and the float-float path (binary64-level accuracy)
        for key, prec, leaf in (("fp64_plain_p16_leaf128", lfmm.LFMM_FP64, 128), ("df_p16_leaf128", lfmm.LFMM_DF, 128)):
            o2 = lfmm.make_opts(prec, 16, leaf, 32, 64)
            ms2, _ = timed(s_d, t_d, f_d, u_d, o2, max(2, args.steps // 4), 1, sync_ranks=False)
            u2 = u_d.cpu().numpy()
            out[key] = {"value": (ns + nt) / (ms2 * 1e-3) / 1e6, "unit": "Mpoints/s", "ms_per_step": ms2,
                        "rel_err": float(np.abs(u2[idx] - ref).max() / scale), "leaf_size": leaf}
        out["cpu_baseline"] = cpu_baseline(prob)
        out["uniform_4k"] = uniform_4k_leg(lfmm)
        out["clustered_4m"] = clustered_leg(lfmm)
        out["forest"] = forest_leg(lfmm)
        out["eval_only"] = eval_leg(lfmm)
        out["multi_rhs"] = multi_leg(lfmm)
        out["solvers"] = solvers_leg(lfmm)
        if args.serve_requests > 0:
            out["serve"] = serve_leg(lfmm, args.serve_requests, args.serve_slots, args.serve_pool,
                                     args.serve_budget_ms)
    print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
