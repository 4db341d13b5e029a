#!/usr/bin/env python
"""Benchmark of the execution stage (Algorithm 2) on B300.

Workload (default, `--workload serving`): one compiled 16x100 grid CNF
(grid_cnf(16, 100, seed=1): 1600 variables, 2970 clauses, max-rank 17) and
a pool of 4096 weight-vector queries w(x) ~ U(0.05, 0.95), w(~x) = 1 - w(x)
(seed 1), evaluated in scaled FP32 with the queries batched along the query
index, Q = 256 per wave.  One step = one wave of Q queries through the whole
path: leaf materialisation, every pairwise contraction, the float64 root.

Reported (one JSON line on rank 0):
  value      queries/s with weights already resident in HBM (graph replay of
             wmc_execute_device), max over ranks, whole job;
  e2e        the same through wmc_execute with host buffers (H2D weights and
             D2H results inside the timed region);
  roofline   the streaming contraction kernel (the dominant one): its
             algorithmic bytes / its CUDA-event time, against the measured
             HBM copy bandwidth;
  plain_fp64 the plain one-query-at-a-time FP64 path on the same GPU;
  latency    p50/p99 of (result ready - scheduled arrival) for a Poisson
             stream through the continuous-batching server;
  cpu_baseline the CPU oracle (bucket elimination) on a bounded sample.

`--impl reference` times the CPU oracle itself on the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import wmcgen  # noqa: E402

METRIC = "WMC queries/s and p50/p99 latency vs plain FP64 path; % of HBM roofline"
GRID_H, GRID_W, GRID_SEED = 16, 100, 1
POOL = 4096
# DRAM traffic / algorithmic bytes of the dominant kernel (k2_chain) over a
# serving wave's mix of chains, from one ncu capture, and the SHA-256 of the
# chain kernel's source it was taken on (the shared helpers at the top of
# kernels.cuh, the TMA-staged and chain kernels' section, dev_common.cuh):
# when that source differs, the ratio no longer describes the kernel and
# `roofline.traffic` is null.
TRAFFIC_CAPTURE = {"ratio": 736.2e6 / 939.7e6,
                   "chain_source_sha256": "869b1e344008fb48e90f0cdc05e382ea3b2bf8220381d04400614e18e0fa7f07"}


def _kernel_source_sha256() -> str:
    import hashlib
    csrc = os.path.join(ROOT, "paper_2006_15512_b300", "csrc")
    with open(os.path.join(csrc, "kernels.cuh")) as f:
        k = f.read()
    with open(os.path.join(csrc, "dev_common.cuh")) as f:
        dc = f.read()
    pre = k[:k.index("// ------------------------------------------------------------ K1 generic")]
    tma = k[k.index("// ------------------------------------------------- K2 with TMA staging"):
            k.index("// ------------------------------------------- batched small contractions")]
    chain = k[k.index("// ---------------------------------------------- chain of frontier eliminations"):
              k.index("// ----------------------------------------- long chains, direct loads")]
    return hashlib.sha256((pre + tma + chain + dc).encode()).hexdigest()


def traffic_ratio():
    """(ratio or None, note)."""
    if TRAFFIC_CAPTURE["ratio"] is None:
        return None, "no ncu capture of the current kernel source"
    if TRAFFIC_CAPTURE["chain_source_sha256"] != _kernel_source_sha256():
        return None, "kernel source changed since the ncu capture"
    return TRAFFIC_CAPTURE["ratio"], "ncu capture of k2_chain on this kernel source (serving wave mix)"


def wave_offset(step: int, rank: int, world: int, n_waves: int, Q: int) -> int:
    """Query-pool offset of a rank's wave: ranks take disjoint waves of the
    pool (replicas with no data exchange; each rank's work is fixed as the
    world grows, i.e. weak scaling)."""
    return ((step * world + rank) % n_waves) * Q


def max_over_ranks(value: float, dist, device) -> float:
    """The job's time is the slowest rank's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def tf32_peak():
    """Dense TF32 tensor peak (TFLOP/s): the measured bf16 burst GEMM rate
    times the nominal TF32/bf16 ratio (1.1 / 2.25 PFLOP/s)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal TF32/bf16"
    except Exception:
        return 1800.0 * 1.1 / 2.25, "fallback bf16 x nominal TF32/bf16"


def workload():
    cnf = wmcgen.grid_cnf(GRID_H, GRID_W, GRID_SEED)
    wq, wnq = wmcgen.query_weights(cnf.n_vars, POOL, seed=1, lo=0.05, hi=0.95)
    return cnf, wq, wnq


def config(Q, slots=1):
    return {"workload": f"serving: {GRID_H}x{GRID_W} grid CNF (seed {GRID_SEED}), pool of {POOL} "
                        f"weight-vector queries w~U(0.05,0.95), waves of Q={Q}",
            "Q": Q, "precision": "scaled fp32 (fp64 root)", "waves_in_flight": slots,
            "l2": "inputs larger than L2: each wave streams 2^16-2^17 x Q float32 frontier tensors "
                  "(64-128 MiB at Q=256) through ~400 launches"}


class Clocks:
    """nvidia-smi sampler for the timed region."""

    def __init__(self, index=0):
        self.samples = []
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.samples)}


def cpu_baseline(cnf, wq, wnq, gpu_results, budget_s=15.0):
    """The CPU baseline leg: the oracle (bucket elimination, long double)
    per query on the host cores, for as many pool queries as fit in
    budget_s (at least one); the same oracle values give the accuracy of
    the GPU results for those queries (gpu_results: (mant, exp2) pairs of
    the first pool queries)."""
    import oracle
    from oracle import Big
    col = [i * GRID_W + j + 1 for j in range(GRID_W) for i in range(GRID_H)]
    vals = []
    t0 = time.perf_counter()
    i = 0
    while i == 0 or (time.perf_counter() - t0 < budget_s and i < min(64, len(gpu_results))):
        vals.append(oracle.bucket_elim(cnf, wq[i], wnq[i], order=col))
        i += 1
    dt = time.perf_counter() - t0
    cpu = {"value": i / dt, "unit": "queries/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{i} pool queries of the 16x100 grid, long-double bucket elimination, {dt:.1f} s"}
    err = max(Big(*gpu_results[j]).rel_diff(vals[j]) for j in range(i))
    return cpu, {"max_rel_err_vs_oracle": err, "n": i}


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle timed on the same workload."""
    if rank != 0:
        return
    cnf, wq, wnq = workload()
    import oracle
    col = [i * GRID_W + j + 1 for j in range(GRID_W) for i in range(GRID_H)]
    for s in range(args.warmup):
        oracle.bucket_elim(cnf, wq[s], wnq[s], order=col)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.bucket_elim(cnf, wq[(args.warmup + s) % POOL], wnq[(args.warmup + s) % POOL], order=col)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "queries/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f80 (long double)", "data": "synthetic",
            "config": {"workload": config(args.Q)["workload"], "step": "one query"},
            "cpu_baseline": {"value": v, "unit": "queries/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"{args.steps} pool queries, one per step"},
            "e2e": {"value": v, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def poisson_run(srv, wq, wnq, rate, n):
    """n queries arriving as a Poisson stream at `rate` per second (seed 2),
    open loop: every arrival that is due is submitted at once (one
    wmc_submit_many call for all of them), so the client keeps up at high
    rates.  Latency = server-stamped completion - scheduled arrival.  The
    client's garbage collector is paused during the loop: a full collection
    over the objects an earlier run left (tens of milliseconds) would submit
    a burst of arrivals late and charge the pause to the server."""
    import gc
    arr = wmcgen.poisson_arrivals(n, rate, seed=2)
    gc.collect()
    gc_was_on = gc.isenabled()
    gc.disable()
    try:
        return _poisson_loop(srv, wq, wnq, rate, n, arr)
    finally:
        if gc_was_on:
            gc.enable()


def _poisson_loop(srv, wq, wnq, rate, n, arr):
    pool = wq.shape[0]
    tickets = []
    st0 = srv.stats()
    t0 = time.monotonic()
    j = 0
    while j < n:
        now = time.monotonic() - t0
        if arr[j] > now:
            time.sleep(min(arr[j] - now, 0.001))
            continue
        k = j
        while k < n and arr[k] <= now:
            k += 1
        idx = np.arange(j, k) % pool
        tickets += srv.submit_many(wq[idx], wnq[idx])
        j = k
    done = srv.collect_done_ns(tickets, timeout_s=600)
    st = srv.stats()
    lat_ms = np.array([(done[i] / 1e9 - (t0 + arr[i])) * 1e3 for i in range(n)])
    span = max(done) / 1e9 - t0
    served = n / span
    waves = int(st.waves - st0.waves)
    return {"rate_qps": rate, "n_queries": n, "p50_ms": float(np.percentile(lat_ms, 50)),
            "p99_ms": float(np.percentile(lat_ms, 99)), "mean_ms": float(lat_ms.mean()),
            "served_qps": served, "waves": waves,
            "mean_wave_q": (st.completed - st0.completed) / max(waves, 1),
            "saturated": bool(served < 0.95 * rate)}


def run_ours(args, rank, world):
    import torch
    import paper_2006_15512_b300 as w
    w.wmc_set_fusion(args.fusion)

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    Q = args.Q
    cnf, wq, wnq = workload()
    net = w.Network.from_cnf(cnf)
    plan = w.Plan(net, precision=w.WMC_SCALED_FP32)
    # the walk's layout for this Q: the autotuner's pick (every layout gives
    # the same bits)
    tune = plan.autotune(Q, stream=torch.cuda.current_stream().cuda_stream) if not args.no_tune else None
    info = plan.info(Q)
    n = cnf.n_vars
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    # device-resident query pool and outputs
    d_wp = torch.from_numpy(wq).to(dev)
    d_wn = torch.from_numpy(wnq).to(dev)
    # wave slots: each wave in flight has its own stream, workspace and
    # outputs; consecutive waves alternate between the slots, so one wave's
    # launches overlap the other's (continuous batching)
    n_slots = max(1, args.slots)
    slot_streams = [torch.cuda.Stream(device=dev) for _ in range(n_slots)]
    slot_ws = [torch.empty(info.workspace_bytes, dtype=torch.uint8, device=dev) for _ in range(n_slots)]
    slot_out = [(torch.empty(Q, dtype=torch.float64, device=dev), torch.empty(Q, dtype=torch.int64, device=dev),
                 torch.empty(Q, dtype=torch.int32, device=dev)) for _ in range(n_slots)]
    ws, (mant, ex, fl) = slot_ws[0], slot_out[0]
    n_waves = POOL // Q

    def wave(i):
        off = wave_offset(i, rank, world, n_waves, Q)
        k = i % n_slots
        m, e, f = slot_out[k]
        plan.execute_device(Q, d_wp[off:off + Q], d_wn[off:off + Q], slot_ws[k], m, e, f,
                            stream=slot_streams[k].cuda_stream)

    for i in range(args.warmup):
        wave(i)
    torch.cuda.synchronize()
    # ---- timed region (device-resident inputs)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = w.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(dev.index) as clk:
        ev0.record(stream)
        for st_ in slot_streams:
            st_.wait_event(ev0)
        for i in range(args.steps):
            wave(args.warmup + i)
        for st_ in slot_streams:
            stream.wait_stream(st_)
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = w.launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    if args.only_waves:  # profiling driver: the timed waves only
        if rank == 0:
            print(json.dumps({"waves": args.warmup + args.steps, "Q": Q, "ms": ms}), flush=True)
        return
    t_max = max_over_ranks(ms, dist, dev)
    value = world * args.steps * Q / (t_max / 1e3)

    # ---- end to end through the public serving API with host buffers: the
    # queries of `steps` waves submitted at once (wmc_submit), results
    # collected (wmc_wait); the server copies each wave's weights in from
    # pinned staging and its results back, with n_slots waves in flight
    host_wp, host_wn = np.ascontiguousarray(wq), np.ascontiguousarray(wnq)
    srv = w.Server(plan, max_batch=Q, max_waves=n_slots)
    for t in [srv.submit(host_wp[j], host_wn[j]) for j in range(Q * n_slots)]:
        srv.wait(t)  # warm the server's graphs
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    tickets = []
    for i in range(args.steps):
        off = wave_offset(args.warmup + i, rank, world, n_waves, Q)
        tickets += srv.submit_many(host_wp[off:off + Q], host_wn[off:off + Q])
    e2e_res = [srv.wait(t) for t in tickets]
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    srv.close()
    e2e = {"value": world * args.steps * Q / e2e_s, "unit": "queries/s",
           "h2d_bytes_per_step": 2 * Q * n * 8, "d2h_bytes_per_step": Q * (8 + 8 + 4),
           "api": "wmc_submit_many (one call per wave of queries) / wmc_wait"}
    # the synchronous one-wave call (wmc_execute), for comparison
    plan.execute(host_wp[:Q], host_wn[:Q])
    t0 = time.perf_counter()
    for i in range(args.steps):
        off = wave_offset(args.warmup + i, rank, world, n_waves, Q)
        plan.execute(host_wp[off:off + Q], host_wn[off:off + Q])
    sync_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    e2e_sync = {"value": world * args.steps * Q / sync_s, "unit": "queries/s", "api": "wmc_execute, one wave per call"}

    if rank != 0:
        return

    # ---- roofline of the streaming contraction kernel (one eager walk)
    import ctypes
    nmax = 1 << 16
    node_ms = (ctypes.c_float * nmax)()
    kinds = (ctypes.c_int32 * nmax)()
    nbytes = (ctypes.c_double * nmax)()
    nl = ctypes.c_int64()
    w.check(w.wmc_profile_walk(plan.handle, Q, ctypes.c_void_p(d_wp.data_ptr()),
                               ctypes.c_void_p(d_wn.data_ptr()), ctypes.c_void_p(ws.data_ptr()),
                               info.workspace_bytes, ctypes.c_void_p(mant.data_ptr()),
                               ctypes.c_void_p(ex.data_ptr()), ctypes.c_void_p(fl.data_ptr()),
                               ctypes.c_void_p(sp), nmax, node_ms, kinds, nbytes, ctypes.byref(nl)),
            "wmc_profile_walk")
    L = min(nl.value, nmax)
    k_ms = np.array([node_ms[i] for i in range(L)])
    k_kind = np.array([kinds[i] for i in range(L)])
    k_bytes = np.array([nbytes[i] for i in range(L)])
    hbm, src = peaks()
    sel = (k_kind == 1) | (k_kind == 4) | (k_kind == 8) | (k_kind == 9)
    walk_ms = float(k_ms.sum())
    achieved = float(k_bytes[sel].sum() / (k_ms[sel].sum() / 1e3) / 1e9) if sel.any() else 0.0
    # DRAM bytes per launch: the traffic / algorithmic-bytes ratio of one ncu
    # capture of the chain kernel over a wave's mix of plain, growth and
    # shrink chains, scaled to this run's average streaming launch
    bpl = float(k_bytes[sel].mean()) if sel.any() else 0.0
    ratio, traffic_note = traffic_ratio()
    traffic = ratio * bpl if ratio else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "traffic_note": traffic_note,
                "peak_source": src, "timing": "each streaming launch of one eager walk, CUDA events, "
                                              "launches serialised (no overlap between waves)",
                "kernel": "k2_chain / k2_tma / k2_stream (streaming contractions)",
                "tma_launches": int((k_kind == 4).sum()),
                "chain_launches": int((k_kind == 8).sum()),
                "chain_share_of_streaming": float(k_ms[k_kind == 8].sum() / max(k_ms[sel].sum(), 1e-12)),
                "tma_share_of_streaming": float(k_ms[k_kind == 4].sum() / max(k_ms[sel].sum(), 1e-12)),
                "launches": int(sel.sum()), "share_of_walk": float(k_ms[sel].sum() / walk_ms),
                "avg_launch_us": float(k_ms[sel].mean() * 1e3) if sel.any() else None,
                "bytes_per_launch": float(k_bytes[sel].mean()) if sel.any() else None,
                "generic_k1_share": float(k_ms[k_kind == 0].sum() / walk_ms),
                "small_phase_share": float(k_ms[k_kind == 7].sum() / walk_ms),
                "walk_launches": int(L),
                "eager_walk_ms": walk_ms}

    # ---- plain one-query-at-a-time FP64 path on the same GPU
    plan64 = w.Plan(net, precision=w.WMC_FP64)
    info64 = plan64.info(1)
    ws64 = torch.empty(info64.workspace_bytes, dtype=torch.uint8, device=dev)
    for i in range(3):
        plan64.execute_device(1, d_wp[i:i + 1], d_wn[i:i + 1], ws64, mant, ex, fl, stream=sp)
    torch.cuda.synchronize()
    n_plain = args.plain_queries
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(n_plain):
        plan64.execute_device(1, d_wp[i:i + 1], d_wn[i:i + 1], ws64, mant, ex, fl, stream=sp)
    e1.record(stream)
    torch.cuda.synchronize()
    plain_qps = n_plain / (e0.elapsed_time(e1) / 1e3)

    # ---- Poisson serving runs (continuous batching), one per arrival rate
    latency_by_rate = []
    if args.rate > 0:
        srv = w.Server(plan, max_batch=Q, max_waves=args.waves)
        # warm every power-of-two wave size's graph
        for q in [1 << k for k in range(int(math.log2(Q)) + 1)]:
            for t in srv.submit_many(wq[:q], wnq[:q]):
                srv.wait(t)
        for rate in args.rates:
            latency_by_rate.append(poisson_run(srv, wq, wnq, rate, max(args.n_queries, int(rate * 0.5))))
        srv.close()
    latency = latency_by_rate[0] if latency_by_rate else None
    # ---- CPU baseline leg (and, from its oracle values, the accuracy of
    # the GPU results for the same pool queries)
    cpu, accuracy = None, {"max_rel_err_vs_oracle": None, "n": 0}
    if world == 1 and not args.no_cpu_baseline:
        res = plan.execute(host_wp[:Q], host_wn[:Q])
        cpu, accuracy = cpu_baseline(cnf, wq, wnq, [(r.mant, r.exp2) for r in res])
    accuracy["stated_bound"] = e2e_res[0].rel_err_bound if e2e_res else None
    line = {"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config(Q, n_slots), "e2e": e2e, "e2e_sync": e2e_sync,
            "gpu_launches": int(launches), "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "plain_fp64": {"value": plain_qps, "unit": "queries/s", "queries": n_plain,
                           "speedup_of_batched": value / world / plain_qps},
            "latency": latency, "latency_by_rate": latency_by_rate, "walk_autotune": tune,
            "accuracy": accuracy,
            "plan": {"max_rank": info.max_rank, "n_nodes": info.n_nodes,
                     "workspace_MiB": info.workspace_bytes / 2 ** 20,
                     "algorithmic_GB_per_wave": info.algorithmic_bytes / 1e9}}
    # the whole wave over the timed region: algorithmic bytes per wave / time
    # per wave (two waves in flight overlap, so this is the rate the step
    # achieves, not a single kernel's)
    wave_gbs = info.algorithmic_bytes / (t_max / args.steps / 1e3) / 1e9
    line["roofline"]["in_context"] = {
        "what": "the whole step in the timed region: algorithmic bytes per wave / ms_per_step "
                "(two waves in flight; the chain kernel is ~96% of a wave's device time)",
        "alg_GB_per_step": info.algorithmic_bytes / 1e9, "ms_per_step": t_max / args.steps,
        "achieved_GBs": wave_gbs, "frac": wave_gbs / hbm}
    print(json.dumps(line), flush=True)


def _timed(fn, reps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def _rel_diff(m1, e1, m2, e2):
    """|a - b| / |b| for a = m1 * 2^e1, b = m2 * 2^e2, without leaving the
    float64 range."""
    if m2 == 0:
        return 0.0 if m1 == 0 else float("inf")
    return abs(math.ldexp(m1, e1 - e2) - m2) / abs(m2)


def cpu_baseline_random3cnf(cases, gpu_results):
    """CPU baseline leg of the random 3-CNF config: the oracle's brute force
    (Def. 2.1 over 2^20 assignments) per formula on the host cores; its
    values also give the accuracy of the GPU results."""
    import oracle
    t0 = time.perf_counter()
    vals = [oracle.brute_force(cnf, wp, wn)[0] for (cnf, wp, wn) in cases]
    dt = time.perf_counter() - t0
    err = max(_rel_diff(m, e, v.mant, v.exp2) for (m, e), v in zip(gpu_results, vals))
    return {"value": len(cases) / dt, "unit": "formulas/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"{len(cases)} formulas, brute force over 2^20 assignments"}, err


def cpu_baseline_uneven(sample, gpu_results, budget_s=20.0):
    """CPU baseline leg of the uneven batch: the oracle (bucket elimination,
    long double, along the narrowest of its orders) on formulas of the batch
    until budget_s is spent; its values also give the accuracy of the GPU
    results for those formulas."""
    import oracle
    t0 = time.perf_counter()
    errs, n = [], 0
    for (kind, cnf, wp, wn), (m, e) in zip(sample, gpu_results):
        if n and time.perf_counter() - t0 > budget_s:
            break
        orders = [oracle.min_degree_order(cnf), list(range(1, cnf.n_vars + 1))]
        if kind.startswith("grid"):
            h_, w_ = (int(v) for v in kind[4:].split("x"))
            orders.append(wmcgen.grid_column_order(h_, w_))
        order = min(orders, key=lambda o: oracle.induced_width(cnf, o))
        v = oracle.bucket_elim(cnf, wp, wn, order=order, max_width=30)
        errs.append(_rel_diff(m, e, v.mant, v.exp2))
        n += 1
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "formulas/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{n} formulas of the batch (every 16th), long-double bucket elimination, {dt:.1f} s"}, errs


def plan_many(w, cands, precision, cap, count):
    """Plans of the first `count` candidates whose plans fit max-rank `cap`,
    planned on host threads (the planner releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    out, rejected = [], 0

    def one(c):
        try:
            return w.Plan(w.Network.from_cnf(c[1], c[2], c[3]), precision=precision, max_rank_cap=cap)
        except w._abi.WmcError:
            return None
    with ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        while len(out) < count:
            chunk = [next(cands) for _ in range(64)]
            for c, p in zip(chunk, ex.map(one, chunk)):
                if p is None:
                    rejected += 1
                elif len(out) < count:
                    out.append((p, c))
    return out, rejected


def run_other(args):
    """Measurements of the non-headline configs (one JSON line each)."""
    import torch
    import paper_2006_15512_b300 as w
    w.wmc_set_fusion(args.fusion)
    hbm, src = peaks()
    out = {"workload": args.workload}
    if args.workload == "random3cnf":
        # n=20, m=60 random 3-CNF, FP64, one query per call (latency)
        lat, res, cases = [], [], []
        for seed in range(10):
            cnf = wmcgen.random_kcnf(20, 60, seed=seed)
            wp, wn = wmcgen.weights_complementary(20, seed, 0.1, 0.9)
            plan = w.Plan(w.Network.from_cnf(cnf, wp, wn), precision=w.WMC_FP64)
            plan.execute()
            lat.append(_timed(lambda: plan.execute(), 20))
            r = plan.execute()[0]
            res.append((r.mant, r.exp2))
            cases.append((cnf, wp, wn))
        cpu, err = cpu_baseline_random3cnf(cases, res)
        out.update({"metric": "latency per query (host buffers, FP64)", "p50_us": float(np.median(lat) * 1e6),
                    "max_us": float(max(lat) * 1e6), "max_rel_err": err, "cpu_baseline": cpu})
    elif args.workload == "grid":
        # 24x200 grid, one query, scaled FP32 and FP64; the reference value
        # is the stored golden (written by the oracle's own script)
        with open(os.path.join(ROOT, "tests", "golden", "grid_24x200.json")) as f:
            g = json.load(f)["values"][0]
        cnf = wmcgen.grid_cnf(24, 200, g["seed"])
        wp, wn = wmcgen.weights_complementary(4800, g["seed"], 0.05, 0.95)
        net = w.Network.from_cnf(cnf, wp, wn)
        for name, prec in (("fp32", w.WMC_SCALED_FP32), ("fp64", w.WMC_FP64)):
            plan = w.Plan(net, precision=prec)
            info = plan.info(1)
            plan.execute()
            t = _timed(lambda: plan.execute(), 3)
            r = plan.execute()[0]
            out[name] = {"ms": t * 1e3, "alg_GB": info.algorithmic_bytes / 1e9,
                         "frac_hbm": info.algorithmic_bytes / t / 1e9 / hbm,
                         "rel_err": _rel_diff(r.mant, r.exp2, g["mant"], g["exp2"]),
                         "log10": r.log10, "max_rank": info.max_rank, "stated_bound": r.rel_err_bound}
    elif args.workload == "sweep":
        rows = []
        tf32 = tf32_peak()
        for (ra, rb, b, k) in args.sweep_rows:
            case = wmcgen.pair_case(ra, rb, b, k, seed=7 + ra + rb + k, shuffle=False)
            rc = len(case.labels_c)
            A = torch.from_numpy(case.a).cuda(); B = torch.from_numpy(case.b).cuda()
            C = torch.empty(1 << rc, dtype=torch.float64, device="cuda")
            f64 = lambda: w.contract_pair(0, case.labels_a, A, case.labels_b, B, case.labels_c, C)
            f64()
            t64 = _timed(f64, 3)
            # the autotuner's pick (same bits): the first call measures
            w.wmc_set_autotune(1)
            try:
                f64(); t64_tuned = _timed(f64, 3)
            finally:
                w.wmc_set_autotune(0)
            A32 = torch.empty(A.numel(), dtype=torch.float32, device="cuda")
            B32 = torch.empty(B.numel(), dtype=torch.float32, device="cuda")
            e = torch.zeros(3, dtype=torch.int64, device="cuda")
            w.to_scaled_fp32(A, A32, e[0:1]); w.to_scaled_fp32(B, B32, e[1:2])
            del C
            C32 = torch.empty(1 << rc, dtype=torch.float32, device="cuda")
            f32 = lambda: w.contract_pair(1, case.labels_a, A32, case.labels_b, B32, case.labels_c, C32,
                                          e[0:1], e[1:2], e[2:3])
            f32()
            t32 = _timed(f32, 3)
            w.wmc_set_autotune(1)
            try:
                f32(); t32_tuned = _timed(f32, 3)
            finally:
                w.wmc_set_autotune(0)
            picks = {}
            for name, prec in (("fp64", 0), ("fp32", 1)):
                v, ch = w.pair_variants(prec, case.labels_a, case.labels_b, case.labels_c)
                picks[name] = {"fixed": [w.PAIR_KINDS[v[0][0]], v[0][1]], "tuned": [w.PAIR_KINDS[v[ch][0]], v[ch][1]],
                               "variants": len(v)}
            n_el = (1 << ra) + (1 << rb) + (1 << rc)
            flops = 2.0 * (1 << (rc + k))
            row = {"rank_a": ra, "rank_b": rb, "batch": b, "summed": k,
                   "fp64_ms": t64 * 1e3, "fp64_GBs": 8 * n_el / t64 / 1e9, "fp64_GFLOPs": flops / t64 / 1e9,
                   "fp32_ms": t32 * 1e3, "fp32_GBs": 4 * n_el / t32 / 1e9, "fp32_GFLOPs": flops / t32 / 1e9,
                   "fp64_tuned_ms": t64_tuned * 1e3, "fp32_tuned_ms": t32_tuned * 1e3, "kernels": picks}
            n_free_a, n_free_b = ra - b - k, rb - b - k
            if n_free_a >= 7 and n_free_b >= 7 and 4 <= k <= 16:
                # tensor-core path: three TF32 products per float32 product
                row["fp32_kernel"] = "k4_tc (tcgen05, 3xTF32)"
                row["tensor_frac_of_tf32_peak_3x_products"] = 3 * flops / t32 / 1e12 / tf32[0]
                row["tensor_frac_of_tf32_peak_method_flops"] = flops / t32 / 1e12 / tf32[0]
                row["tf32_peak_tflops"] = tf32[0]
                row["tf32_peak_source"] = tf32[1]
            rows.append(row)
            del A, B, A32, B32, C32
            torch.cuda.empty_cache()
        out["rows"] = rows
        out["hbm_peak_GBs"] = hbm
    elif args.workload == "uneven":
        t0 = time.perf_counter()
        planned, rejected = plan_many(w, wmcgen.uneven_candidates(3), w.WMC_SCALED_FP32, args.rank_cap,
                                      args.n_formulas)
        plan_s = time.perf_counter() - t0
        kinds = {}
        for _, c in planned:
            kinds[c[0][:4]] = kinds.get(c[0][:4], 0) + 1
        t0 = time.perf_counter()
        w.wmc_set_batch_fusion(args.batch_fusion)
        batch = w.Batch([p for p, _ in planned])
        create_s = time.perf_counter() - t0
        info = batch.info()
        for _ in range(max(1, args.warmup)):
            batch.execute()
        reps = max(1, args.steps // 5)
        with Clocks(0) as clk:
            t = _timed(lambda: batch.execute(), reps)
        res = batch.execute()
        # per-formula graph loop on the same formulas
        for p, _ in planned:
            p.execute()
        t_loop = _timed(lambda: [p.execute() for p, _ in planned], 1)
        achieved = info.algorithmic_bytes / t / 1e9
        sample = [(c[0], c[1], c[2], c[3]) for _, c in planned][::16]
        gres = [(r.mant, r.exp2) for r in res][::16]
        cpu, errs = (None, [])
        if not args.no_cpu_baseline:
            cpu, errs = cpu_baseline_uneven(sample, gres)
        out.update({"metric": "formulas/s", "value": len(planned) / t, "unit": "formulas/s",
                    "persistent_ms": t * 1e3, "graph_loop_ms": t_loop * 1e3, "speedup_vs_graph_loop": t_loop / t,
                    "formulas": len(planned), "rejected": rejected, "mix": kinds,
                    "nodes": info.n_nodes, "tasks": info.n_tasks, "grid": info.grid,
                    "workspace_GiB": info.workspace_bytes / 2 ** 30,
                    "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                                 "frac": achieved / hbm, "traffic": None, "peak_source": src,
                                 "kernel": "k6_persistent (one launch; timed with the batch graph's "
                                           "clear, leaf and result kernels)",
                                 "alg_bytes": "one pass per node (|A| + |B| + |C|) or per chain of frontier "
                                              "steps (|A_1| + sum |S_i| + |C_D|)",
                                 "batch_fusion": args.batch_fusion,
                                 "alg_GB": info.algorithmic_bytes / 1e9},
                    "clocks": clk.summary(), "cpu_baseline": cpu,
                    "max_rel_err_sampled": max(errs) if errs else None, "sampled": len(errs),
                    "planning_s": plan_s, "batch_create_s": create_s})
    elif args.workload == "sliced":
        line = run_sliced(args, w)
        if not line:  # ranks other than 0 print nothing
            return
        out.update(line)
    print(json.dumps(out), flush=True)


SLICED_FORMULA = (56, 196, 4)   # random 3-CNF n, m, seed: no plan within rank 31 unsliced
SLICED_RANK = 24


def gather_shares(parts, dist, device):
    """All-gathers every rank's per-query partial results (mant, exp2) and
    returns them as [rank][query] pairs (one collective per array)."""
    import torch
    m = torch.tensor([r.mant for r in parts], dtype=torch.float64, device=device)
    e = torch.tensor([r.exp2 for r in parts], dtype=torch.int64, device=device)
    world = dist.get_world_size()
    ms = [torch.empty_like(m) for _ in range(world)]
    es = [torch.empty_like(e) for _ in range(world)]
    dist.all_gather(ms, m)
    dist.all_gather(es, e)
    return [[(float(a), int(b)) for a, b in zip(mm.tolist(), ee.tolist())] for mm, ee in zip(ms, es)]


def sliced_count(w, plan, wq, wnq, rank, world, dist, device):
    """Index slicing across processes (Alg. 3, Thm 4.2): this rank runs the
    walks of its contiguous share of the slice assignments
    (wmc_execute_slices), the ranks all-gather their per-query partial sums,
    and wmc_combine_results adds them.  Returns the per-query totals."""
    n_slices = 1 << plan.info(1).n_slice_vars
    lo, hi = w.slice_range(n_slices, rank, world)
    parts = plan.execute_slices(lo, hi, wq, wnq)
    if dist is None:
        return parts
    shares = gather_shares(parts, dist, device)
    Q = len(parts)
    return [w.combine_results([w.Result(m, e, 0.0, 0, 0.0) for (m, e) in (sh[q] for sh in shares)])
            for q in range(Q)]


def run_sliced(args, w):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
    n, m, seed = SLICED_FORMULA
    cnf = wmcgen.random_kcnf(n, m, seed=seed)
    Q = 1
    wq, wnq = wmcgen.query_weights(n, Q, seed=5, lo=0.05, hi=0.95)
    plan = w.Plan(w.Network.from_cnf(cnf), precision=w.WMC_SCALED_FP32, slice_to_rank=SLICED_RANK)
    info = plan.info(Q)
    n_slices = 1 << info.n_slice_vars
    for _ in range(max(1, args.warmup)):
        sliced_count(w, plan, wq, wnq, rank, world, dist, dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with Clocks(dev.index) as clk:
        for _ in range(args.steps):
            tot = sliced_count(w, plan, wq, wnq, rank, world, dist, dev)
    dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
    if rank != 0:
        return {}
    hbm, src = peaks()
    walks_per_s = args.steps * n_slices / dt
    alg = info.algorithmic_bytes * n_slices * args.steps / dt / 1e9
    return {"metric": "sliced counts/s (index slicing across processes, Alg. 3)",
            "value": args.steps / dt, "unit": "counts/s", "n_gpus": world,
            "slice_walks_per_s": walks_per_s, "slices": n_slices, "slice_vars": info.n_slice_vars,
            "max_rank": info.max_rank, "formula": f"random 3-CNF n={n} m={m} seed={seed}",
            "collective": "all_gather of per-query (mant, exp2) partial sums, then wmc_combine_results",
            "roofline": {"bound": "hbm", "achieved": alg, "peak": hbm, "unit": "GB/s", "frac": alg / hbm,
                         "peak_source": src, "alg_bytes": "per slice walk: sum over nodes of |A|+|B|+|C|"},
            "result": {"mant": tot[0].mant, "exp2": tot[0].exp2, "rel_err_bound": tot[0].rel_err_bound},
            "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--Q", type=int, default=256)
    ap.add_argument("--slots", type=int, default=2, help="waves in flight (streams + workspaces)")
    ap.add_argument("--rate", type=float, default=2000.0,
                    help="the arrival rate of the headline latency (first of --rates)")
    ap.add_argument("--rates", type=lambda x: [float(v) for v in x.split(",")], default=None,
                    help="arrival rates of the serving runs (queries/s, comma-separated)")
    ap.add_argument("--n-queries", type=int, default=4096)
    ap.add_argument("--waves", type=int, default=2)
    ap.add_argument("--plain-queries", type=int, default=32)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the fixed walk layout (no autotuning)")
    ap.add_argument("--fusion", type=int, default=-1,
                    help="longest chain of frontier eliminations per pass (-1: by the walk's lane count)")
    ap.add_argument("--workload", default="serving",
                    choices=["serving", "random3cnf", "grid", "sweep", "uneven", "sliced"])
    ap.add_argument("--n-formulas", type=int, default=512)
    ap.add_argument("--rank-cap", type=int, default=26, help="uneven batch: largest plan rank admitted")
    ap.add_argument("--batch-fusion", type=int, default=4,
                    help="uneven batch: longest chain of frontier steps in one pass (0: none)")
    ap.add_argument("--sweep-rows", type=lambda x: [tuple(int(v) for v in r.split(",")) for r in x.split(";")],
                    default=[(29, 5, 2, 1), (28, 12, 4, 4), (17, 17, 2, 1), (24, 22, 0, 8), (22, 22, 0, 16)],
                    help="sweep cases 'rank_a,rank_b,batch,summed;...'")
    ap.add_argument("--only-waves", action="store_true",
                    help="run the warm-up and timed waves only (profiling driver)")
    args = ap.parse_args()
    if args.rates is None:
        args.rates = [args.rate] + [r for r in (5000.0, 10000.0, 20000.0, 50000.0) if r != args.rate]
    if args.impl == "ours" and not args.only_waves:
        args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload != "serving":
        run_other(args)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
