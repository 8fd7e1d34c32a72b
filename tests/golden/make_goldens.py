"""Write the oracle's records of the full-size workloads (test data).

Calls only the CPU oracle (``oracle/``) and the seeded input generators
(``paper_1803_01237_gb300/inputs.py``, which draw keys and hold none of the
method's arithmetic).  Nothing here runs on a GPU or reads a GPU result.

Records (one JSON file per workload, plus compressed arrays where the whole
splitter list is kept for element-by-element comparison):

  scale     N = 2^28 u64 keys, p = 1024, eps = 0.02, s = 5; uniform (seed 1),
            32-Gaussian mixture (seed 2), Zipf s = 1.2 over 2^12 values
            (seed 3); payload = input index.
  morton    N = 2^30 Morton keys of a Plummer sphere with the particle index
            as payload, p = 16384, eps = 0.01, seed 7.
  batch     4096 int64 jobs, sizes log-uniform in [2^10, 2^22] (plan seed 4),
            p = max(4, n / 2^14), eps = 0.05, job j with seed 1 + j.
  two_stage the morton workload sorted by two-stage HSS with r = 128 groups
            (Sec. 5.3; Sec. 7.3's r = sqrt(p)): stage 1's record and group
            offsets, every group's stage-2 record, the final offsets.

For every case: the round count, per-round sample sizes Z_j, |gamma_j| and
unresolved splitters (Sec. 4.2.2), tol, status, the offsets chi(0..p), the
splitter tags (key, seg, spos), and SHA-256 digests of the input and of the
globally sorted keys and payload (little-endian bytes).

Usage:  python tests/golden/make_goldens.py {scale|morton|batch|two_stage} [--workers K]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SCALE = {"N": 1 << 28, "p": 1024, "eps": 0.02, "oversample": 5.0,
         "inputs": {"uniform": 1, "gauss_mix": 2, "zipf": 3}}
MORTON = {"log2n": 30, "p": 16384, "eps": 0.01, "seed": 7, "oversample": 5.0}
TWO_STAGE = dict(MORTON, groups=128)
BATCH = {"njobs": 4096, "plan_seed": 4, "lo_log2": 10, "hi_log2": 22, "zipf_s": 1.1, "zipf_distinct": 1 << 16,
         "eps": 0.05, "seed": 1, "oversample": 5.0}


def sha(a: np.ndarray, n: int = 64) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()[:n]


def batch_p(n: int) -> int:
    """Processors of a batch job of n keys: max(4, n / 2^14), at most n."""
    return max(1, min(n, max(4, n >> 14)))


def _record(res, keys, payload) -> dict:
    spl_key = np.ascontiguousarray(res.splitter_key).view(np.uint64)
    return {
        "rounds": int(res.rounds), "status": int(res.status), "tol": int(res.tol),
        "sample_size": [int(x) for x in res.sample_size], "gamma": [int(x) for x in res.gamma],
        "unresolved": [int(x) for x in res.unresolved],
        "input_sha256": sha(np.ascontiguousarray(keys).view(np.uint64)),
        "offsets_sha256": sha(res.offsets.astype(np.uint64)),
        "splitters_sha256": sha(np.concatenate([spl_key, res.splitter_seg.astype(np.int64).view(np.uint64),
                                                res.splitter_spos.astype(np.uint64)])),
        "out_keys_sha256": sha(np.ascontiguousarray(res.out_keys).view(np.uint64)),
        "out_payload_sha256": None if payload is None else sha(res.out_payload.astype(np.uint32)),
    }


def _scale_one(dist: str):
    import oracle
    from paper_1803_01237_gb300 import inputs
    seed = SCALE["inputs"][dist]
    keys = inputs.SCALE_DISTRIBUTIONS[dist](SCALE["N"], seed)
    pay = np.arange(SCALE["N"], dtype=np.uint32)
    t = time.time()
    res = oracle.hss(keys, SCALE["p"], SCALE["eps"], seed, oversample=SCALE["oversample"], payload=pay)
    rec = _record(res, keys, pay)
    rec["oracle_seconds"] = round(time.time() - t, 1)
    arrays = {"offsets": res.offsets.astype(np.uint64), "spl_key": np.ascontiguousarray(res.splitter_key).view(np.uint64),
              "spl_seg": res.splitter_seg.astype(np.int32), "spl_spos": res.splitter_spos.astype(np.uint32)}
    return dist, rec, arrays


def make_scale(workers: int):
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(workers, 3)) as pool:
        out = pool.map(_scale_one, list(SCALE["inputs"]))
    recs = {"config": {k: v for k, v in SCALE.items()}, "cases": {}}
    arrays = {}
    for dist, rec, arr in out:
        recs["cases"][dist] = rec
        for k, v in arr.items():
            arrays[f"{dist}_{k}"] = v
    _write("scale", recs, arrays)


def make_morton(workers: int):
    import oracle
    from paper_1803_01237_gb300 import inputs
    N = 1 << MORTON["log2n"]
    keys, pay = inputs.plummer_morton(N, MORTON["seed"])
    t = time.time()
    res = oracle.hss(keys, MORTON["p"], MORTON["eps"], MORTON["seed"], oversample=MORTON["oversample"], payload=pay)
    rec = _record(res, keys, pay)
    rec["oracle_seconds"] = round(time.time() - t, 1)
    arrays = {"offsets": res.offsets.astype(np.uint64), "spl_key": np.ascontiguousarray(res.splitter_key).view(np.uint64),
              "spl_seg": res.splitter_seg.astype(np.int32), "spl_spos": res.splitter_spos.astype(np.uint32)}
    _write("morton", {"config": dict(MORTON), "cases": {"plummer": rec}}, arrays)


def make_two_stage(workers: int):
    import oracle
    from paper_1803_01237_gb300 import inputs
    cfg = TWO_STAGE
    N = 1 << cfg["log2n"]
    keys, pay = inputs.plummer_morton(N, cfg["seed"])
    t = time.time()
    res = oracle.hss_two_stage(keys, cfg["p"], cfg["groups"], cfg["eps"], cfg["seed"], oversample=cfg["oversample"],
                               payload=pay)
    st1 = res.stage1
    rec1 = {
        "rounds": int(st1.rounds), "status": int(st1.status), "tol": int(st1.tol),
        "sample_size": [int(x) for x in st1.sample_size], "gamma": [int(x) for x in st1.gamma],
        "unresolved": [int(x) for x in st1.unresolved],
        "input_sha256": sha(np.ascontiguousarray(keys).view(np.uint64)),
    }
    groups = []
    for g, st in enumerate(res.stage2):
        spl_key = np.ascontiguousarray(st.splitter_key).view(np.uint64)
        groups.append({
            "rounds": int(st.rounds), "status": int(st.status), "tol": int(st.tol),
            "sample_size": [int(x) for x in st.sample_size], "gamma": [int(x) for x in st.gamma],
            "unresolved": [int(x) for x in st.unresolved],
            "splitters_sha256": sha(np.concatenate([spl_key, st.splitter_seg.astype(np.int64).view(np.uint64),
                                                    st.splitter_spos.astype(np.uint64)]), 16),
        })
    recs = {"config": dict(cfg), "stage1": rec1, "groups": groups,
            "offsets_sha256": sha(res.offsets.astype(np.uint64)),
            "out_keys_sha256": sha(np.ascontiguousarray(res.out_keys).view(np.uint64)),
            "out_payload_sha256": sha(res.out_payload.astype(np.uint32)),
            "oracle_seconds": round(time.time() - t, 1)}
    arrays = {"offsets": res.offsets.astype(np.uint64),
              "group_spl_key": np.ascontiguousarray(st1.splitter_key).view(np.uint64),
              "group_spl_seg": st1.splitter_seg.astype(np.int32), "group_spl_spos": st1.splitter_spos.astype(np.uint32)}
    _write("two_stage", recs, arrays)


def _batch_one(j: int):
    import oracle
    from paper_1803_01237_gb300 import inputs
    sizes, coin = inputs.batch_job_plan(BATCH["njobs"], BATCH["plan_seed"], BATCH["lo_log2"], BATCH["hi_log2"])
    n = int(sizes[j])
    keys = inputs.batch_job(j, BATCH["plan_seed"], n, bool(coin[j]), BATCH["zipf_s"], BATCH["zipf_distinct"])
    p = batch_p(n)
    res = oracle.hss(keys, p, BATCH["eps"], BATCH["seed"] + j, oversample=BATCH["oversample"])
    rec = _record(res, keys, None)
    del rec["out_payload_sha256"]
    for k in ("input_sha256", "offsets_sha256", "splitters_sha256", "out_keys_sha256"):
        rec[k] = rec[k][:16]
    rec.update({"n": n, "p": p, "kind": "uniform" if coin[j] else "zipf"})
    return j, rec


def make_batch(workers: int):
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        out = pool.map(_batch_one, range(BATCH["njobs"]), chunksize=8)
    out.sort()
    _write("batch", {"config": dict(BATCH), "jobs": [r for _, r in out]}, None)


def _write(name: str, recs: dict, arrays):
    if name == "batch":  # 4096 job records: compact and gzipped
        import gzip
        with gzip.open(os.path.join(HERE, f"fullsize_{name}.json.gz"), "wt") as f:
            json.dump(recs, f, separators=(",", ":"))
            f.write("\n")
    else:
        with open(os.path.join(HERE, f"fullsize_{name}.json"), "w") as f:
            json.dump(recs, f, indent=1)
            f.write("\n")
    if arrays:
        np.savez_compressed(os.path.join(HERE, f"fullsize_{name}.npz"), **arrays)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["scale", "morton", "batch", "two_stage"])
    ap.add_argument("--workers", type=int, default=max(1, (os.cpu_count() or 2) - 1))
    a = ap.parse_args()
    t = time.time()
    {"scale": make_scale, "morton": make_morton, "batch": make_batch, "two_stage": make_two_stage}[a.which](a.workers)
    print(f"{a.which}: {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    main()
