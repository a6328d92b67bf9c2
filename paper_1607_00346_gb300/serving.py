"""Request loop that keeps factored operators resident and batches solves.

Requests arrive over time (Poisson arrivals in the benchmark).  A request
names an operator (grid size n and coefficient seed) and carries nrhs
right-hand sides.  The server

* admits a factorization only when its predicted device footprint
  (``hif_predict_bytes``) fits in the memory budget next to the factors and
  factorizations already on the device; the least recently used idle
  operators are released to make room;
* keeps factored operators resident, so later requests for the same operator
  skip the factorization; with a spill directory, an evicted operator is
  written to disk (hif_save) and brought back by hif_load when it is asked
  for again;
* batches all waiting requests for one operator into a single multi-column
  PCG solve (one apply launch sequence for all their right-hand sides);
* runs admitted jobs on several worker threads, each with its own CUDA stream,
  so that requests that arrive while others are on the GPU are taken up as
  slots and memory free up and their kernels overlap on the device;
* records per-request latency (arrival to solution) and reports p50/p99 and
  solves per second.

The backend is pluggable: ``HifBackend`` drives the CUDA library through its C
ABI; tests use a fake backend to check the scheduling on the CPU.
"""
from __future__ import annotations

import math
import threading
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np

from . import inputs


@dataclass
class Request:
    rid: int
    n: int
    seed: int
    nrhs: int
    arrival: float
    m: int = 4
    # filled by the server
    t_start: float = math.nan
    t_done: float = math.nan
    iters: list = field(default_factory=list)
    relres: list = field(default_factory=list)
    factored: bool = False
    u: np.ndarray | None = None

    @property
    def op_key(self):
        return (self.n, self.m, self.seed)

    @property
    def latency(self):
        return self.t_done - self.arrival


def leaf_size(n: int) -> int:
    """Leaf cell side m with n = m 2^L: 4 when possible, else 3."""
    for m in (4, 3, 5, 6, 7):
        q = n // m
        if n % m == 0 and q > 0 and (q & (q - 1)) == 0:
            return m
    raise ValueError(f"no leaf size for n={n}")


class HifBackend:
    """Real backend: hif_factor / hif_solve through the C ABI."""

    def __init__(self, eps=1e-6, precision=1, lo=-2.0, hi=2.0, b=0.0, keep_u=False):
        import torch

        from . import hif
        self.torch = torch
        self.hif = hif
        self.eps, self.precision, self.lo, self.hi, self.b = eps, precision, lo, hi, b
        self.keep_u = keep_u
        hif.load()

    def new_stream(self):
        return self.torch.cuda.Stream()

    def predict_bytes(self, n, m):
        return self.hif.predict_bytes(n, m, eps=self.eps, precision=self.precision)

    def factor(self, n, m, seed, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            a = torch.from_numpy(inputs.coeff_log_uniform(n, self.lo, self.hi, seed)).cuda()
            h = self.hif.factor(n, m, a, b_const=self.b, eps=self.eps,
                                precision=self.precision, stream=stream)
        return h, int(h.stats()["factor_bytes"])

    def solve(self, h, n, rhs: np.ndarray, stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            f = torch.from_numpy(rhs).cuda()
            u = torch.zeros_like(f)
            its, rel = h.solve(f, u, stream=stream)
            uh = u.cpu().numpy() if self.keep_u else None
        return its, rel, uh

    def release(self, h):
        h.close()

    def save(self, h, path: str):
        h.save(path)

    def load(self, path: str, stream):
        h = self.hif.load_factor(path)
        return h, int(h.stats()["factor_bytes"])


@dataclass
class _Resident:
    handle: object
    bytes: int
    busy: int = 0


class Server:
    def __init__(self, backend, mem_budget: int, workers: int = 4, spill_dir: str | None = None):
        self.be = backend
        self.budget = int(mem_budget)
        self.workers = workers
        # with spill_dir, an evicted operator is written to disk (hif_save)
        # and a later request for it loads the file instead of refactoring
        self.spill_dir = spill_dir
        self.spilled: dict = {}    # op_key -> (path, bytes)
        self.lock = threading.Condition()
        self.resident: OrderedDict = OrderedDict()   # op_key -> _Resident (LRU order)
        self.reserved = 0          # bytes of factorizations in progress
        self.pending: deque = deque()
        self.inflight_keys: set = set()
        self.done: list = []
        self.failed: list = []
        self.log: list = []        # (time, event, detail)

    # ---- memory ---------------------------------------------------------------
    def _in_use(self):
        return self.reserved + sum(r.bytes for r in self.resident.values())

    def _make_room(self, need: int) -> bool:
        """Evict idle residents (LRU) until `need` bytes fit; False if impossible."""
        while self._in_use() + need > self.budget:
            victim = next((k for k, r in self.resident.items() if r.busy == 0), None)
            if victim is None:
                return False
            r = self.resident.pop(victim)
            if self.spill_dir is not None:
                import os
                path = os.path.join(self.spill_dir, "op_%d_%d_%d.hiff" % victim)
                self.be.save(r.handle, path)
                self.spilled[victim] = (path, r.bytes)
            self.be.release(r.handle)
            self.log.append((time.perf_counter(), "evict", victim))
        return True

    # ---- scheduling -------------------------------------------------------------
    def _next_job(self):
        """Pick waiting requests of one operator that can start now (lock held)."""
        seen = set()
        for req in list(self.pending):
            key = req.op_key
            if key in seen or key in self.inflight_keys:
                continue
            seen.add(key)
            batch = [r for r in self.pending if r.op_key == key]
            if key in self.resident:
                self.resident.move_to_end(key)
                self.resident[key].busy += 1
                for r in batch:
                    self.pending.remove(r)
                self.inflight_keys.add(key)
                return key, batch, 0
            spilled = self.spilled.get(key)
            need = spilled[1] if spilled else self.be.predict_bytes(req.n, req.m)
            if need > self.budget:
                # can never be admitted: fail these requests and move on
                for r in batch:
                    self.pending.remove(r)
                    r.t_done = time.perf_counter()
                    r.iters, r.relres = [-1] * r.nrhs, [math.nan] * r.nrhs
                self.failed.extend(batch)
                self.log.append((time.perf_counter(), "refused", key))
                continue
            if self._make_room(need):
                self.reserved += need
                for r in batch:
                    self.pending.remove(r)
                self.inflight_keys.add(key)
                return key, batch, need
        return None

    def _worker(self, stream):
        while True:
            with self.lock:
                job = None
                while job is None:
                    if self._stop and not self.pending:
                        return
                    job = self._next_job()
                    if job is None:
                        self.lock.wait(0.01)
            key, batch, reserved = job
            n, m, seed = key
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                if reserved:
                    with self.lock:
                        spilled = self.spilled.pop(key, None)
                    if spilled:
                        h, fbytes = self.be.load(spilled[0], stream)
                        self.log.append((time.perf_counter(), "load", key))
                    else:
                        h, fbytes = self.be.factor(n, m, seed, stream)
                    with self.lock:
                        self.reserved -= reserved
                        reserved = 0
                        self.resident[key] = _Resident(h, fbytes, busy=1)
                        for r in batch:
                            r.factored = True
                else:
                    with self.lock:
                        h = self.resident[key].handle
                rhs = np.concatenate([inputs.normal_rhs(n, r.nrhs, 10_000 + r.rid)
                                      for r in batch])
                its, rel, u = self.be.solve(h, n, rhs, stream)
            except Exception as exc:     # the job fails; the server carries on
                with self.lock:
                    self.reserved -= reserved
                    if key in self.resident:
                        self.resident[key].busy -= 1
                    self.inflight_keys.discard(key)
                    for r in batch:
                        r.t_done = time.perf_counter()
                        r.iters, r.relres = [-1] * r.nrhs, [math.nan] * r.nrhs
                    self.failed.extend(batch)
                    self.log.append((time.perf_counter(), "error", repr(exc)))
                    self.lock.notify_all()
                continue
            t1 = time.perf_counter()
            c = 0
            for r in batch:
                r.iters = list(its[c:c + r.nrhs])
                r.relres = list(rel[c:c + r.nrhs])
                if u is not None:
                    r.u = u[c:c + r.nrhs]
                c += r.nrhs
                r.t_done = t1
            with self.lock:
                self.resident[key].busy -= 1
                self.inflight_keys.discard(key)
                self.done.extend(batch)
                self.log.append((t1, "done", [r.rid for r in batch]))
                self.lock.notify_all()

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start); returns stats."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self._stop = False
        threads = []
        t_base = time.perf_counter()
        for _ in range(self.workers):
            s = self.be.new_stream()
            th = threading.Thread(target=self._worker, args=(s,), daemon=True)
            th.start()
            threads.append(th)
        for r in reqs:
            if realtime:
                delay = t_base + r.arrival - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            with self.lock:
                r.arrival = (t_base + r.arrival) if realtime else time.perf_counter()
                self.pending.append(r)
                self.lock.notify_all()
        with self.lock:
            self._stop = True
            self.lock.notify_all()
        for th in threads:
            th.join()
        t_end = time.perf_counter()
        return self.stats(t_end - t_base)

    def stats(self, makespan: float) -> dict:
        lat = sorted(r.latency for r in self.done)
        if not lat:
            return {}

        def pct(q):
            return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]

        solves = sum(r.nrhs for r in self.done)
        return {"requests": len(self.done), "solves": solves, "makespan_s": makespan,
                "solves_per_s": solves / makespan, "requests_per_s": len(self.done) / makespan,
                "p50_ms": 1e3 * pct(0.50), "p99_ms": 1e3 * pct(0.99),
                "factorizations": sum(1 for r in self.done if r.factored),
                "failed": len(self.failed),
                "max_iters": max(max(r.iters) for r in self.done)}

    def release_all(self):
        for r in self.resident.values():
            self.be.release(r.handle)
        self.resident.clear()


def poisson_requests(count: int, rate: float, sizes, seed: int, nrhs_max: int = 16,
                     repeat_prob: float = 0.0):
    """Seeded Poisson stream: sizes drawn uniformly, 1..nrhs_max rhs each.

    With repeat_prob > 0 a request reuses the operator of an earlier one."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        if out and rng.random() < repeat_prob:
            prev = out[int(rng.integers(len(out)))]
            n, oseed = prev.n, prev.seed
        else:
            n = int(sizes[int(rng.integers(len(sizes)))])
            oseed = int(rng.integers(1 << 30))
        out.append(Request(rid=i, n=n, m=leaf_size(n), seed=oseed,
                           nrhs=int(rng.integers(1, nrhs_max + 1)), arrival=t))
    return out
