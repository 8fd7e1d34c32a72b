"""The benchmark's contract on the host (no GPU): the reference arm's JSON
line, its behaviour under a two-rank torchrun launch, and the max-over-ranks
timing of the multi-process path over gloo."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


@pytest.mark.timeout(600)
def test_reference_arm_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


@pytest.mark.timeout(600)
def test_reference_arm_two_ranks_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench._max_over_ranks(10.0 + rank, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_max_over_ranks_gloo():
    """Every rank reports the slowest rank's time (world size 2, gloo)."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == {0: 11.0, 1: 11.0}
    import bench  # noqa: E402  (single process: the value itself)
    assert bench._max_over_ranks(3.5, None, "cpu") == 3.5


def test_split_traffic_record_rule():
    """The roofline's DRAM traffic comes from a committed capture that is
    void once the split pass's sources change: the hash moves with an edit
    inside them, not with one elsewhere in segsort.cu, is None when a marker
    is gone, and the full-size bytes are the capture's scaled by the keys."""
    sys.path.insert(0, ROOT)
    import bench
    csrc = os.path.join(ROOT, "paper_1803_01237_gb300", "csrc")
    cu, cuh, internal = (open(os.path.join(csrc, n)).read() for n in ("segsort.cu", "segsort.cuh", "hss_internal.cuh"))
    h = bench.split_source_hash(cu, cuh, internal)
    assert h is not None and len(h) == 16
    start = cu.find("struct SplitArgs {")
    inside = cu[:start + 18] + " " + cu[start + 18:]
    assert bench.split_source_hash(inside, cuh, internal) != h
    assert bench.split_source_hash(cu + "\n// trailing note\n", cuh, internal) == h
    assert bench.split_source_hash(cu.replace("struct SplitArgs {", "struct Split {"), cuh, internal) is None
    assert bench.split_source_hash(cu, cuh, internal + " ") != h
    rec = {}
    for line in open(os.path.join(ROOT, "profiles", "k_split_traffic.txt")):
        if "=" in line and not line.startswith("#"):
            k, v = line.strip().split("=", 1)
            rec[k] = v
    full = int(rec["dram_bytes_per_launch_capture"]) * (1 << bench.LOG2N) // int(rec["keys_capture"])
    assert int(float(rec["dram_bytes_per_launch_full_size"])) == full
    got = bench._traffic_record()
    assert got is None if rec["split_source_sha"] != h else got == float(full)


def test_clock_summary_of_nvidia_smi_samples():
    """The bench's clock record: median SM clock over the samples, the
    maximum clock, and every throttle reason seen active; malformed or
    partial lines are skipped and no valid sample gives None."""
    sys.path.insert(0, ROOT)
    import bench
    text = "\n".join([
        "0, 1965, 2070, 900.1, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2070, 850.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 870.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 870.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1990, 2070",
        "",
    ])
    got = bench.ClockSampler.summarize(text)
    assert got == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = "0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active\n"
    assert bench.ClockSampler.summarize(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.ClockSampler.summarize("") is None
    assert bench.ClockSampler.summarize("0, [N/A], [N/A], 0, 0x0, a, b, c, d\n") is None
