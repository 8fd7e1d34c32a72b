#!/usr/bin/env python3
"""Benchmark of the HSS hot path on GB300.

Workload: N = 2^28 uint64 keys drawn uniform from [0, 2^64) (seed 1), p = 1024
virtual processors of 2^18 keys, eps = 0.02, s = 5 probes per processor per
round.  One step = one hss_sort call: local sort of every segment, splitter
rounds, exchange of runs to buckets and per-bucket merge, with the input
already resident in HBM.  The inputs (2 GiB) are larger than L2, so no flush
is needed between steps.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead (the reference arm).

Multi-GPU: the path does not shard across devices in this build; under
torchrun every rank runs an independent replica of the workload (weak
scaling) and `value` counts the keys of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "keys/s and % of HBM roofline (1 GB300) for HSS sort at eps; HSS rounds; batched jobs/s; p99"
LOG2N, P, EPS, SEED, OVERSAMPLE = 28, 1024, 0.02, 1, 5.0
WORKLOAD = ("HSS sort: N=2^28 uint64 keys, p=1024 segments of 2^18, eps=0.02, s=5; steps cycle over three seeded "
            "inputs: uniform [0,2^64) (seed 1), 32-Gaussian mixture sigma=2^40 (seed 2), Zipf s=1.2 over 2^12 values (seed 3); each input sampled with its own seed")
DISTS = (("uniform", 1), ("gauss_mix", 2), ("zipf", 3))
CPU_SAMPLE_LOG2N = 24      # cpu_baseline: first 2^24 keys, same p and eps
PATH_BYTES_PER_KEY = 98.3  # algorithmic bytes of one whole hss_sort step per key (keys only)
FLOOR_BYTES_PER_KEY = 67.5  # the method's floor: local sort R+W 16, gamma reads ~19.5, exchange 16, merge 16
REF_SAMPLE_LOG2N = 22      # reference arm: first 2^22 keys per step


def _max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's figure (the job's time): an all-reduce MAX over
    the ranks; x itself in a single process."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The sources the split pass's DRAM traffic depends on: its kernel and
# helpers in segsort.cu, the tile constants in segsort.cuh, and the shared
# device helpers.  The committed traffic record holds their hash.
_SPLIT_REGIONS = (("__device__ __forceinline__ uint32_t split_digit(", "// Exclusive scan of 256 shared values"),
                  ("__device__ __forceinline__ uint32_t warp_peers8(", "// On-chip sort of segments"),
                  ("__device__ __forceinline__ uint32_t splitter_digit(", "// Splitters of the first split"),
                  ("struct SplitArgs {", "__global__ void k_even_offsets("))


def split_source_hash(segsort_cu: str, segsort_cuh: str, internal_cuh: str):
    """sha256 (16 hex digits) of the split pass's sources, or None when a
    marker is missing."""
    parts = []
    for a, b in _SPLIT_REGIONS:
        i = segsort_cu.find(a)
        j = segsort_cu.find(b, i)
        if i < 0 or j < 0:
            return None
        parts.append(segsort_cu[i:j])
    i = segsort_cuh.find("constexpr int kRadixBits")
    j = segsort_cuh.find("\n", segsort_cuh.find("constexpr int kOsTile"))
    if i < 0 or j < 0:
        return None
    parts.append(segsort_cuh[i:j])
    parts.append(internal_cuh)
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def _traffic_record():
    """Per-launch DRAM bytes of the radix digit pass from the committed ncu
    summary, valid only while the split pass's sources are unchanged."""
    path = os.path.join(ROOT, "profiles", "k_split_traffic.txt")
    csrc = os.path.join(ROOT, "paper_1803_01237_gb300", "csrc")
    if not os.path.exists(path):
        return None
    texts = []
    for name in ("segsort.cu", "segsort.cuh", "hss_internal.cuh"):
        with open(os.path.join(csrc, name)) as f:
            texts.append(f.read())
    sha = split_source_hash(*texts)
    rec = {}
    for line in open(path):
        line = line.strip()
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            rec[k.strip()] = v.strip()
    if sha is None or rec.get("split_source_sha") != sha:
        return None
    try:
        return float(rec["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"hss_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            text = f.read()
        os.unlink(self.path)
        return self.summarize(text)

    @staticmethod
    def summarize(text: str):
        """Median SM clock, maximum clock and the throttle reasons seen
        active in nvidia-smi's CSV samples (None without a valid sample)."""
        rows = [ln.split(",") for ln in text.strip().splitlines() if ln.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(log2n: int):
    """The oracle as it stands on one host core (first 2^log2n keys of the
    workload), plus two references for context: the same method on all host
    cores (OpenMP, checked equal to the oracle in the CPU tests) on 4x the
    keys, and std::sort of the sample on one core."""
    import numpy as np
    import oracle
    from paper_1803_01237_gb300 import inputs
    full = inputs.uniform(1 << LOG2N, SEED)
    keys = np.ascontiguousarray(full[: 1 << log2n])
    t0 = time.perf_counter()
    res = oracle.hss(keys, P, EPS, SEED, oversample=OVERSAMPLE)
    dt = time.perf_counter() - t0
    assert res.status == 0
    line = {"value": (1 << log2n) / dt, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": f"first 2^{log2n} keys of the workload (same p={P}, eps={EPS}, seed), single-threaded C oracle, "
                      f"{dt:.1f} s"}
    n_omp = min(log2n + 2, LOG2N)
    big = np.ascontiguousarray(full[: 1 << n_omp])
    oracle.hss_omp(big[: 1 << 16], P, EPS, SEED, oversample=OVERSAMPLE)  # thread pool up
    t0 = time.perf_counter()
    r = oracle.hss_omp(big, P, EPS, SEED, oversample=OVERSAMPLE)
    dt_omp = time.perf_counter() - t0
    assert r[7] == 0
    line["all_cores"] = {"value": (1 << n_omp) / dt_omp, "unit": "keys/s", "cores": oracle.baseline_threads(),
                         "kind": "HSS with OpenMP on all host cores (same result as the oracle)",
                         "sample": f"first 2^{n_omp} keys, same p, eps, seed; {dt_omp:.2f} s"}
    t0 = time.perf_counter()
    oracle.std_sort(keys)
    dt_std = time.perf_counter() - t0
    line["std_sort"] = {"value": (1 << log2n) / dt_std, "unit": "keys/s", "cores": 1, "kind": "std::sort",
                        "sample": f"first 2^{log2n} keys; {dt_std:.2f} s"}
    return line


def run_reference(args):
    """Reference arm: the CPU oracle on a bounded sample per step."""
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1803_01237_gb300 import inputs
    oracle.build()
    keys = np.ascontiguousarray(inputs.uniform(1 << LOG2N, SEED)[: 1 << REF_SAMPLE_LOG2N])
    for _ in range(args.warmup):
        oracle.hss(keys, P, EPS, SEED, oversample=OVERSAMPLE)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.hss(keys, P, EPS, SEED, oversample=OVERSAMPLE)
        times.append(time.perf_counter() - t0)
        assert r.status == 0
    ms = 1000.0 * sum(times) / len(times)
    value = (1 << REF_SAMPLE_LOG2N) / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": 1 << LOG2N, "p": P, "eps": EPS, "distribution": "uniform",
                   "sample_per_step": f"first 2^{REF_SAMPLE_LOG2N} keys"},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": f"first 2^{REF_SAMPLE_LOG2N} keys of the workload per step, same p and eps"},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs

    rank, world, local = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()

    N = 1 << LOG2N
    keys_h = inputs.uniform(N, SEED)
    if args.dist:
        dists = tuple(d for d in DISTS if d[0] == args.dist)
    else:
        dists = DISTS if LOG2N == 28 and not args.uniform_only else (("uniform", SEED),)
    dev_inputs = []
    for name, sd in dists:
        kh = keys_h if name == "uniform" else inputs.SCALE_DISTRIBUTIONS[name](N, sd)
        dev_inputs.append((name, torch.from_numpy(kh.view(np.int64)).to(dev), sd))
    keys = dev_inputs[0][1]
    out = torch.empty_like(keys)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def step(k, flags=0):  # each input with its own seed, as in the oracle's records of this workload
        _, dk, sd = dev_inputs[k % len(dev_inputs)]
        return hss.sort(dk, P, EPS, sd, oversample=OVERSAMPLE, flags=flags, out=out)

    for w in range(max(args.warmup, len(dev_inputs))):
        step(w)
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = hss.launch_count()
    pass_ms, pass_launches, pass_keys, phase = 0.0, 0, 0, {}
    per_dist = {name: {"ms": 0.0, "steps": 0, "rounds": []} for name, _, _ in dev_inputs}
    rounds = None
    barrier()
    ev0.record(stream)
    for k in range(args.steps):
        r = step(k, flags=hss.FLAG_TIMING)
        pass_ms += r.ms_radix_pass_total
        pass_launches += r.radix_pass_launches
        pass_keys += r.radix_pass_keys
        for kk, v in r.ms_phase.items():
            phase[kk] = phase.get(kk, 0.0) + v
        pd = per_dist[dev_inputs[k % len(dev_inputs)][0]]
        pd["ms"] += sum(r.ms_phase.values())
        pd["steps"] += 1
        pd["rounds"].append(r.rounds)
        rounds = r
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = hss.launch_count() - launches0
    ms = _max_over_ranks(ev0.elapsed_time(ev1) / args.steps, dist, dev)
    value = world * N / (ms / 1000.0)
    dist_report = {name: {"device_ms_per_step": v["ms"] / max(v["steps"], 1),
                          "keys_per_s_device": N / (v["ms"] / max(v["steps"], 1) / 1000.0) if v["steps"] else None,
                          "rounds": sorted(set(v["rounds"]))} for name, v in per_dist.items()}

    # correctness spot check of the last output (sorted, offsets in range)
    o = out[:: max(1, N // (1 << 20))].cpu().numpy().view(np.uint64)
    sorted_ok = bool(np.all(o[:-1] <= o[1:]))

    # roofline of the dominant kernel: the one-sweep split pass reads and
    # writes every key of the segments it splits once (16 B per key)
    peak, peak_kind = _measured_peaks()
    avg_pass_ms = pass_ms / max(pass_launches, 1)
    bytes_per_pass = 16.0 * pass_keys / max(pass_launches, 1)
    achieved = bytes_per_pass / (avg_pass_ms / 1000.0) / 1e9 if pass_launches else 0.0
    traffic = _traffic_record()

    # end to end: pinned host keys -> hss_sort_host -> host sorted keys
    e2e = None
    if not args.no_e2e:
        hk = torch.empty(N, dtype=torch.int64, pin_memory=True)
        hk.copy_(torch.from_numpy(keys_h.view(np.int64)))
        ho = torch.empty(N, dtype=torch.int64, pin_memory=True)
        hkn, hon = hk.numpy(), ho.numpy()
        hss.sort_host(hkn, P, EPS, SEED, oversample=OVERSAMPLE, out=hon)
        n_e2e = max(2, min(args.steps, 5))
        barrier()
        t0 = time.perf_counter()
        calls_ms = []
        for _ in range(n_e2e):
            tc = time.perf_counter()
            hss.sort_host(hkn, P, EPS, SEED, oversample=OVERSAMPLE, out=hon)
            calls_ms.append(round(1000 * (time.perf_counter() - tc), 2))
        e2e_s = (time.perf_counter() - t0) / n_e2e
        e2e_s = _max_over_ranks(e2e_s, dist, dev)
        e2e = {"value": world * N / e2e_s, "unit": "keys/s", "h2d_bytes_per_step": 8 * N,
               "d2h_bytes_per_step": 8 * N + 16 * (P - 1) + 8 * (P + 1), "ms_per_step": 1000 * e2e_s,
               "api": "hss_sort_host (pinned host buffers, copies inside the call)", "input": "uniform",
               "calls_ms": calls_ms, "median_call_ms": sorted(calls_ms)[len(calls_ms) // 2],
               "note": "value and ms_per_step are the mean over the calls; on this shared host single calls "
                       "sometimes take 3-4 times the median while the device phases keep their times "
                       "(the host copies slow down)"}
        del hk, ho

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "p": P, "eps": EPS, "oversample": OVERSAMPLE,
                   "distributions": [n for n, _, _ in dev_inputs],
                   "l2": "inputs (2 GiB keys per distribution) larger than L2; no flush between steps",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "k_split (one-sweep MSD scatter, 16 B/key)",
                     "bytes_per_launch": bytes_per_pass,
                     "peak_source": f"{peak_kind} hbm_gbs", "avg_launch_ms": avg_pass_ms,
                     "launches": pass_launches},
        "path_roofline": {
            "model": "algorithmic HBM bytes of the whole step per key: local sort 8 (statistics) + 16 (split) + 16 "
                     "(on-chip sort), rounds ~2.3 (bitmap, probes), exchange 16, merge 8 + 16 + 16",
            "bytes_per_key": PATH_BYTES_PER_KEY, "achieved_GBs": PATH_BYTES_PER_KEY * world * N / (ms / 1000.0) / 1e9,
            "peak_GBs": peak, "frac": PATH_BYTES_PER_KEY * world * N / (ms / 1000.0) / 1e9 / peak,
            "floor_bytes_per_key": FLOOR_BYTES_PER_KEY,
            "frac_of_floor": FLOOR_BYTES_PER_KEY * world * N / (ms / 1000.0) / 1e9 / peak,
            "note": "headline fraction of the whole step; the 'roofline' object covers one kernel"},
        "per_distribution": dist_report,
        "hss": {"rounds": rounds.rounds, "sample_size": rounds.sample_size, "gamma": rounds.gamma,
                "tol": rounds.tol, "phase_ms": {k: v / args.steps for k, v in phase.items()},
                "kernels_per_step": rounds.kernel_launches, "output_sorted": sorted_ok},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(min(CPU_SAMPLE_LOG2N, LOG2N))
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch_workload(args):
    """Config 4: 4096 independent int64 sort jobs, sizes log-uniform in
    [2^10, 2^22], p = max(4, n / 2^14), eps = 0.05, each uniform or Zipf(1.1)
    over 2^16 values by a seeded coin.  A step is one hss_sort_batch call over
    all jobs, timed with the library's default choices and then (unless
    --no-tune) with the autotuner's choice of oversampling and sort tiling,
    which gives the line's value; the plain form (one hss_sort call per job,
    in order) is timed once on the same jobs for comparison."""
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()
    njobs = args.batch_jobs
    jobs, kinds = inputs.batch_jobs(njobs, 4, lo_log2=10, hi_log2=22, zipf_s=1.1, zipf_distinct=1 << 16)
    sizes = [len(x) for x in jobs]
    ps = [max(1, min(n, max(4, n >> 14))) for n in sizes]
    keys = torch.from_numpy(np.concatenate(jobs)).to(dev)
    del jobs
    out = torch.empty_like(keys)
    eps, seed = 0.05, 1
    for _ in range(args.warmup):
        hss.sort_batch(keys, sizes, ps, eps, seed, key_type="i64", out=out)
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = hss.launch_count()
    ev0.record()
    for _ in range(args.steps):
        r = hss.sort_batch(keys, sizes, ps, eps, seed, key_type="i64", out=out)
    ev1.record()
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = hss.launch_count() - l0
    ms = ev0.elapsed_time(ev1) / args.steps
    ok = all(s == 0 for s in r.job_status)
    rounds_b = float(np.mean(r.job_rounds))
    # plain form: one hss_sort per job (the single-call path), same jobs
    offs = np.concatenate([[0], np.cumsum(sizes)])
    tuned = None
    if not args.no_tune:
        # the project's autotuner picks oversampling and sort tiling on a
        # subset of the jobs (cached per GPU and batch shape), then the whole
        # batch is timed with its choice
        from paper_1803_01237_gb300 import autotune
        t_tune = time.perf_counter()
        choice = autotune.Tuner().tune_batch(keys, sizes, ps, eps, seed, key_type="i64")
        t_tune = time.perf_counter() - t_tune
        s_t, flags_t = choice.apply()
        try:
            hss.sort_batch(keys, sizes, ps, eps, seed, oversample=s_t, flags=flags_t, key_type="i64", out=out)
            torch.cuda.synchronize(dev)
            ev0.record()
            for _ in range(args.steps):
                rt = hss.sort_batch(keys, sizes, ps, eps, seed, oversample=s_t, flags=flags_t, key_type="i64", out=out)
            ev1.record()
            torch.cuda.synchronize(dev)
        finally:
            hss.reset_tuning()
        ms_t = ev0.elapsed_time(ev1) / args.steps
        tuned = {"choice": choice.__dict__, "jobs_per_s": njobs / (ms_t / 1000.0), "ms_per_step": ms_t,
                 "mean_rounds_per_job": float(np.mean(rt.job_rounds)), "all_jobs_ok": all(x == 0 for x in rt.job_status),
                 "tuning_seconds": t_tune,
                 "note": "oversampling s changes the sample, so the result is the oracle's for that s"}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rounds_p = []
    for j in range(njobs):
        kj = keys[int(offs[j]):int(offs[j + 1])]
        rr = hss.sort(kj, ps[j], eps, seed + j, key_type="i64", out=out[int(offs[j]):int(offs[j + 1])])
        rounds_p.append(rr.rounds)
    torch.cuda.synchronize(dev)
    plain_s = time.perf_counter() - t0
    line = {
        "metric": "batched jobs/s (HSS sort of independent int64 jobs)",
        "value": tuned["jobs_per_s"] if tuned else njobs / (ms / 1000.0),
        "unit": "jobs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tuned["ms_per_step"] if tuned else ms,
        "untuned": {"jobs_per_s": njobs / (ms / 1000.0), "ms_per_step": ms, "oversample": 5.0,
                    "tiling": "library defaults"},
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"batched HSS sort: {njobs} int64 jobs, sizes log-uniform [2^10, 2^22], "
                               "p = max(4, n/2^14), eps = 0.05, uniform or Zipf(1.1) over 2^16 values by a seeded coin",
                   "jobs": njobs, "keys": int(offs[-1]), "segments": int(sum(ps)),
                   "l2": "inputs larger than L2; no flush"},
        "keys_per_s": offs[-1] / (ms / 1000.0),
        "mean_rounds_per_job": rounds_b, "lockstep_rounds": r.lockstep_rounds, "all_jobs_ok": ok,
        "phase_ms": r.ms_phase, "gpu_launches": launches,
        "plain_form": {"jobs_per_s": njobs / plain_s, "keys_per_s": offs[-1] / plain_s, "seconds": plain_s,
                       "mean_rounds_per_job": float(np.mean(rounds_p)),
                       "api": "hss_sort per job, host loop, same stream"},
        "autotuned": tuned,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_morton_workload(args):
    """Config 3: N = 2^30 64-bit Morton keys of a seeded Plummer sphere (21
    bits per axis) with the particle index as a u32 payload, p = 16384,
    eps = 0.01.  A step is one hss_sort of keys and payload, both resident
    in HBM (12 GiB in, 12 GiB out: larger than L2, no flush).  The same
    line times the step as two-stage HSS with --groups groups
    (hss_sort_two_stage, key `two_stage`); --morton-form two times that form
    alone and makes it the line's value.  Unless --no-tune, the autotuner then
    picks the sort tiling, histogram form and round driver on this input at
    s = 5 (key `autotuned`: the same result, timed for both forms)."""
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()
    N, P, E, SEED = 1 << args.morton_log2n, 16384, 0.01, 7
    kh, ph = inputs.plummer_morton(N, SEED)
    keys = torch.from_numpy(kh.view(np.int64)).to(dev)
    pay = torch.from_numpy(ph.view(np.int32)).to(dev)
    del kh, ph
    out, out_p = torch.empty_like(keys), torch.empty_like(pay)
    single = args.morton_form in ("both", "single")
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r, phase, ms, launches, o = None, {}, None, 0, None
    if single:
        for _ in range(args.warmup):
            hss.sort(keys, P, E, SEED, payload=pay, out=out, out_payload=out_p)
        torch.cuda.synchronize(dev)
        l0 = hss.launch_count()
        ev0.record()
        for _ in range(args.steps):
            r = hss.sort(keys, P, E, SEED, payload=pay, out=out, out_payload=out_p, flags=hss.FLAG_TIMING)
            for k, v in r.ms_phase.items():
                phase[k] = phase.get(k, 0.0) + v / args.steps
        ev1.record()
        torch.cuda.synchronize(dev)
        launches = hss.launch_count() - l0
        ms = ev0.elapsed_time(ev1) / args.steps
        o = out[:: max(1, N // (1 << 20))].cpu().numpy().view(np.uint64)
    two = None
    if args.groups > 1 and args.morton_form in ("both", "two"):
        # The same step as two-stage HSS: the p processors split into
        # `groups` groups first, then every group sorted over p / groups
        # processors (Sec. 5.3; Sec. 7.3 takes r = sqrt(p) = 128 at p = 16384).
        R = args.groups
        for _ in range(max(1, args.warmup)):
            hss.sort_two_stage(keys, P, R, E, SEED, payload=pay, out=out, out_payload=out_p)
        torch.cuda.synchronize(dev)
        phase2 = {}
        l2 = hss.launch_count()
        ev0.record()
        for _ in range(args.steps):
            t = hss.sort_two_stage(keys, P, R, E, SEED, payload=pay, out=out, out_payload=out_p, flags=hss.FLAG_TIMING)
            for k, v in t.ms_phase.items():
                phase2[k] = phase2.get(k, 0.0) + v / args.steps
        ev1.record()
        torch.cuda.synchronize(dev)
        ms2 = ev0.elapsed_time(ev1) / args.steps
        o2 = out[:: max(1, N // (1 << 20))].cpu().numpy().view(np.uint64)
        two = {"groups": R, "ms_per_step": ms2, "keys_per_s": N / (ms2 / 1000.0),
               "stage1_rounds": t.stage1.rounds, "stage1_sample_size": t.stage1.sample_size,
               "stage2_lockstep_rounds": t.lockstep_rounds,
               "stage2_mean_rounds": float(np.mean(t.group_rounds)), "phase_ms": phase2,
               "gpu_launches": hss.launch_count() - l2, "output_sorted": bool(np.all(o2[:-1] <= o2[1:])),
               "same_output_as_single_stage": None if o is None else bool(np.array_equal(o, o2))}
    tuned = None
    if not args.no_tune:
        # The autotuner on this input at s = 5 (its tiling, histogram form and
        # round driver leave the result unchanged, so the tuned step is still
        # the oracle's), then both forms timed with its choice.
        import tempfile
        from dataclasses import asdict
        from paper_1803_01237_gb300 import autotune
        with tempfile.TemporaryDirectory() as td:
            tuner = autotune.Tuner(os.path.join(td, "tuning.json"))
            t0 = time.perf_counter()
            choice = tuner.tune(N, P, E, kind="morton", sample=keys, payload=pay, seed=SEED, trials=1,
                                space=([5.0], autotune.default_space(P)[1]), force=True)
            tuning_s = time.perf_counter() - t0
        s_, fl_ = choice.apply()
        try:
            forms = {}
            for form in (("single",) if not (args.groups > 1 and args.morton_form in ("both", "two")) else
                         ("single", "two")):
                call = (lambda: hss.sort(keys, P, E, SEED, payload=pay, out=out, out_payload=out_p, oversample=s_,
                                         flags=fl_)) if form == "single" else \
                       (lambda: hss.sort_two_stage(keys, P, args.groups, E, SEED, payload=pay, out=out,
                                                   out_payload=out_p, oversample=s_, flags=fl_))
                call()
                torch.cuda.synchronize(dev)
                ev0.record()
                for _ in range(args.steps):
                    call()
                ev1.record()
                torch.cuda.synchronize(dev)
                forms[form] = ev0.elapsed_time(ev1) / args.steps
        finally:
            hss.reset_tuning()
        tuned = {"choice": asdict(choice), "tuning_seconds": tuning_s,
                 "single_ms_per_step": forms.get("single"), "two_stage_ms_per_step": forms.get("two"),
                 "note": "autotuned at s = 5: same splitters, offsets and output as the library defaults"}
    clk = clocks.stop()
    if not single:
        if two is None:
            raise SystemExit("--morton-form two needs --groups > 1")
        # the two-stage form alone: it is the line's value
        ms, launches = two["ms_per_step"], two["gpu_launches"]
    line = {
        "metric": "keys/s (HSS sort with u32 payload)", "value": N / (ms / 1000.0), "unit": "keys/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"HSS sort of 2^{args.morton_log2n} Morton keys (Plummer sphere, 21 bits per axis) "
                               "+ u32 payload, p = 16384, eps = 0.01"
                               + ("" if single else f", two-stage with {args.groups} groups"),
                   "N": N, "p": P, "eps": E, "l2": "inputs larger than L2; no flush"},
        "hss": None if r is None else {"rounds": r.rounds, "sample_size": r.sample_size, "phase_ms": phase,
                                       "output_sorted": bool(np.all(o[:-1] <= o[1:]))},
        "gpu_launches": launches, "clocks": clk,
    }
    if two is not None:
        line["two_stage"] = two
    if tuned is not None:
        line["autotuned"] = tuned
    print(json.dumps(line), flush=True)
    return 0


def run_serve_workload(args):
    """Config 5: Poisson arrivals at 2000 partition requests/s, sizes
    log-uniform in [2^16, 2^26], p in {256, 1024, 4096}, eps = 0.02,
    lognormal(0, 2) keys on one 2^63 scale; the CDF network trains online on
    completed jobs and proposes the first cuts of later ones (plain HSS until
    it is ready).  Keys are device-resident slices of four lognormal pools."""
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs, serve

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()
    pool = [torch.from_numpy(inputs.lognormal_job(1 << 26, 500 + b).view(np.int64)).to(dev) for b in range(4)]
    reqs = serve.poisson_requests(pool, args.serve_requests, rate=args.serve_rate, seed=7, lo_log2=16, hi_log2=26,
                                  ps=(256, 1024, 4096), eps=0.02)
    results = {}
    low_rate = args.serve_low_rate
    low_reqs = serve.poisson_requests(pool, max(1, min(args.serve_requests, int(low_rate * 5))), rate=low_rate,
                                      seed=8, lo_log2=16, hi_log2=26, ps=(256, 1024, 4096), eps=0.02)
    for rate_name, rr in (("offered", reqs), ("sustainable", low_reqs)):
        for mode in ("plain", "learned"):
            model = hss.CDFModel(dev).init(3, "log", 1, (1 << 63) - 1) if mode == "learned" else None
            srv = serve.Server(slots=args.serve_slots, model=model, train=True, train_steps=50, train_interval=0.05,
                               hbm_budget="free")
            srv.warmup()
            torch.cuda.synchronize(dev)
            clocks = ClockSampler(local)
            clocks.start()
            st = srv.run(rr, realtime=True)
            clk = clocks.stop()
            heldout = ([e for e, _ in srv.trainer.heldout] if srv.trainer is not None else None)
            srv.close()
            summ = st.summary()
            summ["heldout_errors_last"] = heldout
            summ["rate_per_s"] = args.serve_rate if rate_name == "offered" else low_rate
            summ["clocks"] = clk
            results[f"{rate_name}_{mode}"] = summ
    s_l = results["offered_learned"]
    line = {
        "metric": "served partition requests: p99 latency", "value": s_l["p99_ms"], "unit": "ms", "n_gpus": 1,
        "steps": args.serve_requests, "warmup": 1, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"served HSS partitions: Poisson {args.serve_rate:g}/s, {args.serve_requests} requests, "
                               "sizes log-uniform [2^16, 2^26], p in {256, 1024, 4096}, eps = 0.02, lognormal(0,2) keys",
                   "slots": args.serve_slots, "sustainable_rate_per_s": low_rate,
                   "admission": "a free slot and free device memory (cudaMemGetInfo), 1 GiB kept free"},
        "runs": results,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_rounds_workload(args):
    """Round-count study (the rounds of Sec. 7.1, Fig. 1): histogram rounds
    of hss_partition against p for oversampling s = 1 and s = 5 at eps = 2%,
    N = 2^26 uniform keys, p = 2^4 .. 2^16 (at p = 2^16 the p x (p-1)
    per-segment cut positions and the p x (sample capacity) probe positions
    take about 195 GiB of the device), with the growth of Theorem 4.8,
    O(log(log p / eps)), printed beside as log2(log2(p) / eps), and for s = 5
    the bound ceil(ln(2 ln p / eps) / ln(s / 4)) + 2."""
    import math
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()
    N, eps = 1 << 26, 0.02
    keys = torch.from_numpy(inputs.uniform(N, 1).view(np.int64)).to(dev)
    table = []
    for lp in range(4, 17):
        p = 1 << lp
        row = {"p": p, "log2_log2p_over_eps": math.log2(math.log2(p) / eps),
               "bound_s5": math.ceil(math.log(2.0 * math.log(p) / eps) / math.log(5.0 / 4.0)) + 2}
        for s_ in (1.0, 5.0):
            rounds = []
            for seed in (1, 2, 3):
                res, _ = hss.partition(keys, p, eps, seed, oversample=s_)
                rounds.append(res.rounds)
            row[f"rounds_s{int(s_)}"] = rounds
            row[f"mean_rounds_s{int(s_)}"] = float(np.mean(rounds))
        table.append(row)
        torch.cuda.empty_cache()
    line = {"metric": "HSS rounds vs p (s = 1 and s = 5, eps = 0.02)", "value": table[-1]["mean_rounds_s5"],
            "unit": "rounds", "n_gpus": 1, "steps": len(table), "warmup": 0, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "round-count study: N = 2^26 uniform u64, eps = 0.02, p = 2^4 .. 2^16, "
                                   "s in {1, 5}, seeds 1-3"},
            "table": table}
    print(json.dumps(line), flush=True)
    return 0


def run_schedules_workload(args):
    """Sampling-schedule ablation (Sec. 4.2.2, Theorem 4.7): at the bench
    shape (N = 2^28, p = 1024, eps = 0.02) on the three inputs, the rounds,
    the probes drawn over all rounds and the partition time of the
    proportional schedule (s = 5, the default), the k-round schedule
    s_j = (2 ln p / eps)^(j/k) for k = 2, 3, 4, and equal sampling per
    interval (HykSort)."""
    import numpy as np
    import torch
    from paper_1803_01237_gb300 import hss, inputs

    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hss.load()
    N = 1 << LOG2N
    rows = []
    for name, sd in DISTS:
        keys = torch.from_numpy(inputs.SCALE_DISTRIBUTIONS[name](N, sd).view(np.int64)).to(dev)
        for sched, k in (("proportional", 0), ("theory", 2), ("theory", 3), ("theory", 4), ("equal", 0)):
            hss.partition(keys, P, EPS, SEED, schedule=sched, schedule_k=k)  # warm
            torch.cuda.synchronize(dev)
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            res, _ = hss.partition(keys, P, EPS, SEED, schedule=sched, schedule_k=k, flags=hss.FLAG_TIMING)
            ev1.record()
            torch.cuda.synchronize(dev)
            rows.append({"input": name, "schedule": sched, "k": k, "rounds": res.rounds,
                         "probes": int(sum(res.sample_size)), "sample_size": res.sample_size,
                         "partition_ms": ev0.elapsed_time(ev1), "rounds_ms": res.ms_phase["rounds"]})
        del keys
        torch.cuda.empty_cache()
    line = {"metric": "sampling-schedule ablation: rounds and probes per partition", "value": None,
            "unit": "rounds", "n_gpus": 1, "steps": len(rows), "warmup": 1, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": f"hss_partition N=2^{LOG2N}, p={P}, eps={EPS}, seed {SEED}, three inputs"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--uniform-only", action="store_true", help="time the uniform input only")
    ap.add_argument("--dist", default=None, choices=[d[0] for d in DISTS], help="time one input only")
    ap.add_argument("--log2n", type=int, default=None,
                    help="smaller case of the same kernels (keeps 2^18 keys per segment); for profiling only")
    ap.add_argument("--workload", default="sort", choices=["sort", "batch", "serve", "rounds", "schedules", "morton"],
                    help="sort: the N=2^28 bench line (default); batch: 4096 independent jobs; serve: Poisson requests")
    ap.add_argument("--batch-jobs", type=int, default=4096)
    ap.add_argument("--no-tune", action="store_true", help="batch and morton workloads: skip the autotuned timing")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-low-rate", type=float, default=300.0)
    ap.add_argument("--morton-log2n", type=int, default=30, help="config 3 size (morton workload)")
    ap.add_argument("--morton-form", default="both", choices=["both", "single", "two"],
                    help="morton workload: time single-stage HSS, two-stage HSS or both (the value is the single stage "
                         "unless only the two-stage form runs)")
    ap.add_argument("--groups", type=int, default=128,
                    help="morton workload: also time two-stage HSS with this many groups (0: skip)")
    args = ap.parse_args()
    if args.workload == "batch" and args.impl == "gb300":
        args.warmup = max(args.warmup, 1)
        return run_batch_workload(args)
    if args.workload == "serve" and args.impl == "gb300":
        return run_serve_workload(args)
    if args.workload == "morton" and args.impl == "gb300":
        return run_morton_workload(args)
    if args.workload == "rounds" and args.impl == "gb300":
        return run_rounds_workload(args)
    if args.workload == "schedules" and args.impl == "gb300":
        return run_schedules_workload(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.log2n is not None:
        global LOG2N, P, WORKLOAD
        LOG2N = args.log2n
        P = max(1, 1 << max(0, LOG2N - 18))
        WORKLOAD = f"HSS sort: N=2^{LOG2N} uint64 keys uniform (seed 1), p={P}, eps=0.02, s=5 (profiling case)"
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
