"""Serving loop for HSS partition requests with continuous batching.

Requests (keys resident on the device, p, eps, seed) arrive over time.  A
request is admitted as soon as a slot is free and its device memory fits in
the budget; every slot runs on its own CUDA stream from its own host thread
(the C calls release the GIL), so the kernels of admitted requests overlap
on the GPU while later requests keep arriving.  Once the CDF network has
been trained on the splitters of completed jobs (exact ranks of sampled
keys), a request starts from the network's proposed cuts
(hss_partition_with_proposal) when the plan (plan_proposal: the network's
held-out error against the request's p, eps and size) expects them to save
a round; otherwise, before training, or if proposing fails, it runs plain
HSS.  The histogram rounds decide balance either way, so every result
satisfies the same contract, and a request computes the same splitters and
offsets alone or in the mix given the same proposal (which each completion
records).

Latency runs from a request's arrival time to the host seeing its result.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field

import torch

from . import hss


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    keys: torch.Tensor       # device keys (int64 storage of u64/i64 bits)
    p: int
    eps: float
    seed: int
    key_type: str = "u64"


@dataclass
class Completion:
    rid: int
    arrival: float
    admitted: float
    done: float
    rounds: int
    status: int
    n: int
    p: int
    tol: int
    offsets: torch.Tensor
    splitters: torch.Tensor
    proposal: torch.Tensor | None
    slot: int
    error: str | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def rounds_from(width: float, p: int, eps: float, s: float = 5.0) -> int:
    """Expected sampling rounds until every splitter is resolved when each
    splitter's interval holds a fraction `width` of the N keys, r = width p /
    eps times the 2 tol = eps N / p window.  None when r <= 1.  One when
    r <= 2: the bracket alone resolves about 1 / r of the splitters, and the
    round's s p samples (Sec. 4.2.2) gather on the rest.  Else each round
    shrinks the intervals by about s, plus one round for the largest of the
    p - 1 random gaps."""
    r = width * p / eps
    if r <= 1.0:
        return 0
    if r <= 2.0:
        return 1
    return math.ceil(math.log(r) / math.log(s) - 1e-9) + 1


def plain_rounds(p: int, eps: float, s: float = 5.0) -> int:
    """Expected rounds of plain HSS: round 1 spreads s p samples over the
    whole key range, leaving intervals of about N / (s p) keys; at least three
    rounds, since round 1 resolves splitters only by chance."""
    return max(3, 2 + math.ceil(math.log(max(1.0 / (s * eps), 1.0)) / math.log(s) - 1e-9))


def plan_proposal(p: int, eps: float, delta: float, per_max: int, s: float = 5.0) -> tuple[int, int, int]:
    """(per, expected rounds with the proposal, expected plain rounds), per = 0
    when plain HSS is expected to be cheaper.  Rounds with a proposal count
    the proposal's own ranking pass as one.

    A proposal of per cuts per splitter spread over +-delta brackets each
    target within 2 delta N / (per - 1) keys, at the price of ranking
    (p - 1) per cuts over whole segments (plain round 1 ranks s p).  Taken:
    the smallest per that reaches the fewest rounds, if it saves a round and
    its cuts stay within s p x (1 + rounds saved)."""
    plain = plain_rounds(p, eps, s)
    best = (0, plain)
    for per in range(2, per_max + 1):
        r = 1 + rounds_from(2.0 * delta / (per - 1), p, eps, s)
        if r < best[1] and (p - 1) * per <= s * p * (1 + plain - r):
            best = (per, r)
    return best[0], best[1], plain


@dataclass
class ServeStats:
    completions: list = field(default_factory=list)
    makespan: float = 0.0
    max_in_flight: int = 0
    max_bytes_in_flight: int = 0

    def summary(self) -> dict:
        ok = [c for c in self.completions if c.error is None]
        lat = sorted(c.latency for c in ok)

        def pct(q):
            if not lat:
                return None
            return lat[min(len(lat) - 1, max(0, math.ceil(q * len(lat)) - 1))]

        keys = sum(c.n for c in ok)
        with_prop = [c.rounds for c in ok if c.proposal is not None]
        plain = [c.rounds for c in ok if c.proposal is None]
        return {
            "requests": len(self.completions), "completed": len(ok),
            "jobs_per_s": len(ok) / self.makespan if self.makespan > 0 else None,
            "keys_per_s": keys / self.makespan if self.makespan > 0 else None,
            "p50_ms": 1e3 * pct(0.50) if lat else None, "p99_ms": 1e3 * pct(0.99) if lat else None,
            "mean_rounds_with_proposal": sum(with_prop) / len(with_prop) if with_prop else None,
            "mean_rounds_plain": sum(plain) / len(plain) if plain else None,
            "served_with_proposal": len(with_prop),
            "mean_cuts_per_splitter": (sum(c.proposal.numel() / max(c.p - 1, 1) for c in ok if c.proposal is not None)
                                       / len(with_prop) if with_prop else None),
            "max_in_flight": self.max_in_flight, "max_bytes_in_flight": self.max_bytes_in_flight,
            "makespan_s": self.makespan,
            "by_p": {str(pp): self._by_p(ok, pp) for pp in sorted({c.p for c in ok})},
        }

    @staticmethod
    def _by_p(ok: list, p: int) -> dict:
        cs = [c for c in ok if c.p == p]
        lat = sorted(c.latency for c in cs)
        wp = [c for c in cs if c.proposal is not None]
        return {"requests": len(cs), "with_proposal": len(wp),
                "mean_rounds": sum(c.rounds for c in cs) / len(cs),
                "p50_ms": 1e3 * lat[(len(lat) - 1) // 2]}


class _Trainer:
    """Online training of the CDF network on the splitters of completed jobs
    (targets rank / N on a common 2^40 scale).  It trains a shadow copy on
    its own stream and publishes the parameters to the serving model with
    one device copy under the model lock, so proposals never wait for a
    training run; completions that queued up meanwhile share the next run."""

    SCALE = 1 << 40

    def __init__(self, model: hss.CDFModel, lock: threading.Lock, steps: int, lr: float, keep_jobs: int,
                 min_jobs: int, device, interval: float = 0.0):
        self.model, self.lock, self.steps, self.lr = model, lock, steps, lr
        self.interval = interval
        self.last_train = -1e9
        self.keep_jobs, self.min_jobs = keep_jobs, min_jobs
        self.stream = torch.cuda.Stream(device=device, priority=0)  # the lowest: requests come first
        self.shadow = hss.CDFModel(device)
        self.shadow.key_type = model.key_type
        with torch.cuda.stream(self.stream):
            self.stream.wait_stream(torch.cuda.current_stream(device))
            self.shadow.buf.copy_(model.buf)
        self.q: queue.Queue = queue.Queue()
        self.pairs: list = []
        self.jobs_seen = 0
        self.trainings = 0
        self.loss: float | None = None
        # held-out error: (max |y(key) - rank/N| of the published model over a
        # completed job's splitters, measured before it trains on that job, N)
        self.heldout: list[tuple[float, int]] = []
        self.keep_heldout = 4
        self.max_pairs_per_job = 256
        self.timeline: list[tuple[float, float, int]] = []  # (start, end, points) of each training run
        self.ready = False
        self.thread = threading.Thread(target=self._loop, daemon=True)
        self.thread.start()

    def _heldout_dev(self, model: hss.CDFModel, keys: torch.Tensor, ranks: torch.Tensor, N: int) -> torch.Tensor:
        """max |y(key) - rank / N| over one job's splitters, queued on the
        trainer's stream (a device scalar)."""
        y = model.eval(keys, stream=self.stream).to(torch.float64)
        return (y - ranks.to(torch.float64) / N).abs().max()

    def submit(self, res, N: int, event: torch.cuda.Event):
        """Queue a completed job's result (its splitters and offsets become
        training pairs once `event`, recorded after the job, has passed)."""
        self.q.put((res, N, event))

    def stop(self):
        self.q.put(None)
        self.thread.join()

    def _loop(self):
        stop = False
        while not stop:
            items = [self.q.get()]
            if items[0] is not None and self.ready:
                # at most one run per interval once the model is serving:
                # training shares the GPU with the requests
                wait = self.interval - (time.perf_counter() - self.last_train)
                if wait > 0:
                    time.sleep(wait)
            while True:  # every completion queued meanwhile joins this run
                try:
                    items.append(self.q.get_nowait())
                except queue.Empty:
                    break
            with torch.cuda.stream(self.stream):
                pending = []  # held-out errors on the device, read after the run
                t_start = time.perf_counter()
                for item in items:
                    if item is None:
                        stop = True
                        continue
                    res, N, ev = item
                    self.stream.wait_event(ev)
                    res.splitters.record_stream(self.stream)
                    res.offsets.record_stream(self.stream)
                    keys, ranks = hss.training_pairs(res)
                    if keys.numel() > self.max_pairs_per_job:  # evenly spaced quantiles suffice
                        stride = -(-keys.numel() // self.max_pairs_per_job)
                        keys, ranks = keys[::stride].contiguous(), ranks[::stride].contiguous()
                    if self.trainings > 0 and keys.numel() > 0:
                        pending.append((self._heldout_dev(self.shadow, keys, ranks, N), N))
                    scaled = (ranks.to(torch.float64) * (self.SCALE / N)).to(torch.int64)
                    self.pairs.append((keys, scaled))
                    self.jobs_seen += 1
                self.pairs = self.pairs[-self.keep_jobs:]
                train = not stop and self.jobs_seen >= self.min_jobs and bool(self.pairs)
                if train:
                    tk = torch.cat([k for k, _ in self.pairs])
                    tr = torch.cat([r for _, r in self.pairs])
                    loss = self.shadow.train(tk, tr, self.SCALE, self.steps, self.lr, stream=self.stream)
                self.stream.synchronize()
                for err, N in pending:
                    self.heldout = (self.heldout + [(float(err.item()), N)])[-self.keep_heldout:]
                if not train:
                    continue
                with self.lock:
                    self.model.buf.copy_(self.shadow.buf)
                    self.stream.synchronize()
                    self.loss = float(loss.item())
                    self.trainings += 1
                    self.ready = True
                self.last_train = time.perf_counter()
                self.timeline.append((t_start, self.last_train, int(tk.numel())))


class Server:
    """Continuous-batching server of partition requests.

    slots          concurrent requests on the device (one stream each)
    hbm_budget     bytes of workspace admitted at once (None: no limit), or
                   "free": admit by the device memory free at the time
                   (cudaMemGetInfo, plus what the caching allocator holds
                   unused), keeping hbm_reserve bytes free
    hbm_reserve    bytes left free under hbm_budget="free"
    model          CDF network to train online and propose from (None: plain)
    per_splitter   most proposed cuts per splitter (each request takes the
                   fewest that reach its fewest expected rounds, see plan)
    train          whether completed jobs train the model (False: frozen)
    train_interval seconds between training runs once the model serves
    delta          band half-width of a frozen model's cuts (a fraction of N;
                   at least 0.25 / p); a trained model derives it from its
                   held-out errors over the recent jobs (see _delta)
    """

    def __init__(self, slots: int = 4, hbm_budget: int | str | None = None, model: hss.CDFModel | None = None,
                 per_splitter: int = 16, train: bool = True, train_steps: int = 100, lr: float = 0.01,
                 keep_jobs: int = 16, min_jobs: int = 2, train_interval: float = 0.0, delta: float = 0.0,
                 device=None, hbm_reserve: int = 1 << 30):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.slots = slots
        if isinstance(hbm_budget, str) and hbm_budget != "free":
            raise ValueError('hbm_budget: bytes, None or "free"')
        self.hbm_budget = hbm_budget
        self.hbm_reserve = int(hbm_reserve)
        self.pending_bytes = 0  # admitted under "free", not yet allocated
        self.model = model
        self.per_splitter = per_splitter
        self.frozen_delta = delta
        self.model_lock = threading.Lock()
        self.trainer = None
        self.frozen_ready = model is not None and not train
        if model is not None and train:
            self.trainer = _Trainer(model, self.model_lock, train_steps, lr, keep_jobs, min_jobs, self.device,
                                    train_interval)
        # high-priority streams: the block scheduler serves a request's
        # kernels before the trainer's, which only fill idle SMs
        self.streams = [torch.cuda.Stream(device=self.device, priority=-1) for _ in range(slots)]
        self.slot_ws = [None] * slots
        self.cv = threading.Condition()
        self.free_slots = list(range(slots))
        self.bytes_in_flight = 0

    @staticmethod
    def request_bytes(n: int, p: int, key_type: str = "u64", oversample: float = 5.0, nprop: int = 0) -> int:
        ws = hss.workspace_bytes("partition", n, p, key_type, False, oversample=oversample)
        return ws + 16 * max(p - 1, 1) + 8 * (p + 1) + 8 * nprop

    # a job of n keys drawn from the modelled distribution has its own CDF
    # within sqrt(ln(2 / alpha) / (2 n)) of it with probability 1 - alpha
    # (the Dvoretzky-Kiefer-Wolfowitz inequality, Massart's constant)
    ALPHA = 0.01

    @classmethod
    def _dkw(cls, n: int) -> float:
        return math.sqrt(math.log(2.0 / cls.ALPHA) / (2.0 * max(n, 1)))

    def _delta(self, p: int, n: int) -> float:
        """Half-width of the band of proposed cuts around each target i/p for
        a job of n keys: 1.25 x (the model's error beyond sampling noise, the
        largest over the recent held-out jobs, + the job's own sampling noise).
        A frozen model uses the `delta` it was given; a trained one without
        held-out jobs yet, 3 x its RMS training error."""
        t = self.trainer
        if t is not None and t.heldout:
            model_err = max(max(0.0, e - self._dkw(m)) for e, m in t.heldout)
            base = 1.25 * (model_err + self._dkw(n))
        elif t is not None and t.loss is not None:
            base = 3.0 * math.sqrt(t.loss)
        else:
            base = self.frozen_delta
        return max(base, 0.25 / p)

    def _propose(self, req: Request, stream) -> torch.Tensor | None:
        ready = self.frozen_ready or (self.trainer is not None and self.trainer.ready)
        if self.model is None or not ready or req.key_type != self.model.key_type:
            return None
        delta = self._delta(req.p, req.keys.numel())
        # the proposed cuts may not exceed the round sample capacity
        cap = min(req.keys.numel(), math.ceil(10.0 * req.p) + 4096)
        per, _, _ = plan_proposal(req.p, req.eps, delta, min(self.per_splitter, cap // max(req.p - 1, 1)))
        if per == 0:
            return None
        try:
            with self.model_lock:
                prop = self.model.propose(req.p, per, delta, stream=stream)
                stream.synchronize()
            return prop
        except hss.HSSError:
            return None

    def _serve_one(self, req: Request, slot: int, t0: float, admitted: float, need: int, stats: ServeStats,
                   grow: int = 0):
        stream = self.streams[slot]
        err = None
        res = None
        prop = None
        try:
            with torch.cuda.stream(stream):
                prop = self._propose(req, stream)
                if grow:  # the workspace is taken now: no longer pending
                    nb = self.request_bytes(req.keys.numel(), req.p, req.key_type)
                    ws = self.slot_ws[slot]
                    if ws is None or ws.numel() < nb:
                        self.slot_ws[slot] = None
                        self.slot_ws[slot] = torch.empty(nb, dtype=torch.uint8, device=self.device)
                    with self.cv:
                        self.pending_bytes -= grow
                        grow = 0
                if prop is not None:
                    try:
                        res, _ = self._partition(req, prop, stream, slot)
                    except hss.HSSError:
                        prop = None
                if res is None:
                    res, _ = self._partition(req, None, stream, slot)
                stream.synchronize()
        except Exception as e:  # recorded per request; the server keeps going
            err = repr(e)
        if grow:
            with self.cv:
                self.pending_bytes -= grow
        done = time.perf_counter() - t0  # the result is ready
        if self.trainer is not None and res is not None and err is None:
            # the trainer extracts the pairs on its own stream
            ev = torch.cuda.Event()
            ev.record(stream)
            self.trainer.submit(res, req.keys.numel(), ev)
        c = Completion(rid=req.rid, arrival=req.arrival, admitted=admitted, done=done,
                       rounds=res.rounds if res else -1, status=res.status if res else -1, n=req.keys.numel(),
                       p=req.p, tol=res.tol if res else -1, offsets=res.offsets if res else None,
                       splitters=res.splitters if res else None, proposal=prop, slot=slot, error=err)
        with self.cv:
            stats.completions.append(c)
            self.free_slots.append(slot)
            self.bytes_in_flight -= need
            self.cv.notify_all()

    def _partition(self, req: Request, prop, stream, slot: int):
        # each slot keeps one workspace, grown on demand and reused after its
        # stream has finished with it (slots run concurrently)
        nb = self.request_bytes(req.keys.numel(), req.p, req.key_type)
        ws = self.slot_ws[slot]
        if ws is None or ws.numel() < nb:
            self.slot_ws[slot] = None
            ws = torch.empty(nb, dtype=torch.uint8, device=self.device)
            self.slot_ws[slot] = ws
        return _partition_into(req, prop, ws, stream)

    def _available_bytes(self) -> int:
        """Device memory a new allocation can take now: free memory plus what
        the caching allocator holds without using it."""
        free, _ = torch.cuda.mem_get_info(self.device)
        reclaim = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        return int(free) + int(reclaim)

    def _growth(self, slot: int, req: Request, need: int) -> int:
        """Bytes a request on this slot allocates: its workspace beyond the
        slot's cached one, plus its outputs."""
        nb = self.request_bytes(req.keys.numel(), req.p, req.key_type)
        ws = self.slot_ws[slot]
        cached = ws.numel() if ws is not None else 0
        return max(0, nb - cached) + max(0, need - nb)

    def _fits(self, slot: int, req: Request, need: int) -> bool:
        if self.hbm_budget is None:
            return True
        if self.hbm_budget == "free":
            return self._growth(slot, req, need) + self.pending_bytes <= self._available_bytes() - self.hbm_reserve
        return self.bytes_in_flight + need <= self.hbm_budget

    def run(self, requests: list[Request], realtime: bool = True) -> ServeStats:
        """Serve the requests (sorted by arrival).  With realtime, a request
        is not admitted before its arrival time; otherwise all are ready at
        once (a closed loop)."""
        stats = ServeStats()
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        # work the caller queued before this call (the keys, a model trained
        # on the current stream) comes first on every stream the server uses
        cur = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(cur)
        if self.trainer is not None:
            self.trainer.stream.wait_stream(cur)
        threads = []
        t0 = time.perf_counter()
        for req in reqs:
            if realtime:
                wait = req.arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
            need = self.request_bytes(req.keys.numel(), req.p, req.key_type, nprop=(req.p - 1) * self.per_splitter)
            reject = isinstance(self.hbm_budget, int) and need > self.hbm_budget
            slot = -1
            with self.cv:
                while not reject:
                    if self.free_slots:
                        cand = self.free_slots[-1]
                        if self._fits(cand, req, need):
                            slot = cand
                            break
                        if self.hbm_budget == "free" and self.bytes_in_flight == 0 and self.pending_bytes == 0:
                            # nothing in flight: release the idle slots'
                            # workspaces, then it fits now or never will
                            idle = [k for k in self.free_slots if k != cand and self.slot_ws[k] is not None]
                            for k in idle:
                                self.slot_ws[k] = None
                            if idle and self._fits(cand, req, need):
                                slot = cand
                                break
                            reject = True
                            break
                    # a completion frees a slot or memory; memory freed
                    # elsewhere on the device is seen at the next poll
                    self.cv.wait(timeout=0.05 if self.hbm_budget == "free" else None)
                if not reject:
                    self.free_slots.pop()
                    grow = self._growth(slot, req, need) if self.hbm_budget == "free" else 0
                    self.pending_bytes += grow
                    self.bytes_in_flight += need
            if reject:
                stats.completions.append(Completion(
                    rid=req.rid, arrival=req.arrival, admitted=-1.0, done=time.perf_counter() - t0, rounds=-1,
                    status=hss.ERR_WORKSPACE, n=req.keys.numel(), p=req.p, tol=-1, offsets=None, splitters=None,
                    proposal=None, slot=-1, error="request exceeds the memory budget"))
                continue
            with self.cv:
                stats.max_in_flight = max(stats.max_in_flight, self.slots - len(self.free_slots))
                stats.max_bytes_in_flight = max(stats.max_bytes_in_flight, self.bytes_in_flight)
            admitted = time.perf_counter() - t0
            th = threading.Thread(target=self._serve_one, args=(req, slot, t0, admitted, need, stats, grow),
                                  daemon=True)
            th.start()
            threads.append(th)
        for th in threads:
            th.join()
        stats.makespan = time.perf_counter() - t0
        stats.completions.sort(key=lambda c: c.rid)
        return stats

    def warmup(self, key_type: str = "u64"):
        """Run one small request through every path a served request takes
        (partition, proposal, training pairs, the trainer's arithmetic) on
        every slot, so the first timed request pays no one-time costs (module
        loading, kernel attributes, allocator growth).  The model is left as
        it was."""
        n = 1 << 14
        keys = torch.arange(n, dtype=torch.int64, device=self.device) * 7919
        cur = torch.cuda.current_stream(self.device)
        for st in self.streams:
            st.wait_stream(cur)
        req = Request(rid=-1, arrival=0.0, keys=keys, p=16, eps=0.05, seed=1, key_type=key_type)
        for slot in range(self.slots):
            stream = self.streams[slot]
            with torch.cuda.stream(stream):
                res, _ = self._partition(req, None, stream, slot)
                tk, tr = hss.training_pairs(res)
                scaled = (tr.to(torch.float64) * (_Trainer.SCALE / n)).to(torch.int64)
                torch.cat([tk, tk]), torch.cat([scaled, scaled])
                if self.model is not None:
                    prop = self.model.propose(16, 2, 0.01, stream=stream)
                    self._partition(req, prop, stream, slot)
                stream.synchronize()
        if self.trainer is not None:
            with torch.cuda.stream(self.trainer.stream):
                w = hss.CDFModel(self.device)
                w.buf.copy_(self.model.buf)
                w.train(tk, tr, n, 2, 0.01, stream=self.trainer.stream)
                self.trainer._heldout_dev(w, tk[::2].contiguous(), tr[::2].contiguous(), n)
                self.trainer.stream.synchronize()

    def close(self):
        if self.trainer is not None:
            self.trainer.stop()


def _partition_into(req: Request, prop, ws: torch.Tensor, stream):
    """hss_partition(_with_proposal) of one request into a given workspace."""
    import ctypes
    lib = hss.load()
    keys = req.keys
    N = keys.numel()
    prm = hss._params(req.p, req.eps, req.seed, 5.0, 0, 0)
    spl = torch.empty((max(req.p - 1, 1), 2), dtype=torch.int64, device=keys.device)
    off = torch.empty(req.p + 1, dtype=torch.int64, device=keys.device)
    st = hss.Stats()
    kt = hss.KEY_TYPES[req.key_type]
    if prop is None:
        rc = lib.hss_partition(hss._ptr(keys), kt, N, ctypes.byref(prm), hss._ptr(spl), hss._ptr(off), hss._ptr(ws),
                               ws.numel(), ctypes.byref(st), hss._stream(stream))
        hss._check(rc, "hss_partition")
    else:
        rc = lib.hss_partition_with_proposal(hss._ptr(keys), kt, N, ctypes.byref(prm), hss._ptr(prop), prop.numel(),
                                             hss._ptr(spl), hss._ptr(off), hss._ptr(ws), ws.numel(),
                                             ctypes.byref(st), hss._stream(stream))
        hss._check(rc, "hss_partition_with_proposal")
    return hss._result(None, None, spl[:req.p - 1], off, st), ws


def poisson_requests(pool: list, n_requests: int, rate: float, seed: int, lo_log2: int = 16, hi_log2: int = 26,
                     ps=(256, 1024, 4096), eps: float = 0.02, key_type: str = "u64") -> list:
    """Requests with Poisson arrivals (rate per second), sizes log-uniform in
    [2^lo, 2^hi], p drawn from ps (at most one segment per key), each a slice
    of one of the device key buffers in `pool` at a seeded offset."""
    import numpy as np
    from . import inputs
    g = inputs.rng(seed, 12)
    gaps = g.exponential(1.0 / rate, n_requests)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * g.random(n_requests))).astype(np.int64)
    pick_p = g.integers(0, len(ps), n_requests)
    pick_pool = g.integers(0, len(pool), n_requests)
    out = []
    for i in range(n_requests):
        buf = pool[int(pick_pool[i])]
        n = int(min(sizes[i], buf.numel()))
        off = int(g.integers(0, buf.numel() - n + 1))
        p = int(min(ps[int(pick_p[i])], n))
        out.append(Request(rid=i, arrival=float(arrivals[i]), keys=buf[off:off + n], p=p, eps=eps, seed=1000 + i,
                           key_type=key_type))
    return out
