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
* batches waiting requests: those for one operator become one multi-column
  system, and the systems of every resident operator that has waiting
  requests (grids of different sizes included) are solved together by one
  hif_solve_batch, whose preconditioner applications share their launches;
  each request's result is bitwise the one it gets when served alone;
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
        return self.solve_batch([h], [n], [rhs], stream)[0]

    def solve_batch(self, handles, ns, rhs_list, stream):
        """One hif_solve_batch over several operators; [(its, rel, u)] per operator."""
        torch = self.torch
        with torch.cuda.stream(stream):
            fs = [torch.from_numpy(np.ascontiguousarray(r)).cuda() for r in rhs_list]
            us = [torch.zeros_like(f) for f in fs]
            res = self.hif.solve_batch(handles, fs, us, stream=stream)
            out = []
            for (its, rel), u in zip(res, us):
                out.append((its, rel, u.cpu().numpy() if self.keep_u else None))
            stream.synchronize()
        return out

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
    def __init__(self, backend, mem_budget: int, workers: int = 4, spill_dir: str | None = None,
                 max_ops: int = 8, max_cols: int = 64):
        self.be = backend
        self.budget = int(mem_budget)
        self.workers = workers
        # one solve job takes the waiting requests of at most max_ops resident
        # operators and max_cols right-hand sides
        self.max_ops = max_ops
        self.max_cols = max_cols
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
        self.batch_sizes: list = []   # operators per solve job

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
        """Pick work that can start now (lock held).

        A solve job takes the waiting requests of every resident operator not
        already in a job (up to max_ops operators and max_cols columns); only
        when there is none, the first waiting operator that is not resident
        is admitted (its predicted footprint must fit) and factored; its
        requests then wait for the next solve job with the others.  Returns
        (keys, batches, reserved bytes) with one request list per key, or
        None."""
        keys, batches, cols = [], [], 0
        for req in list(self.pending):
            key = req.op_key
            if key in keys or key in self.inflight_keys or key not in self.resident:
                continue
            batch = [r for r in self.pending if r.op_key == key]
            nc = sum(r.nrhs for r in batch)
            if keys and (len(keys) >= self.max_ops or cols + nc > self.max_cols):
                continue
            keys.append(key)
            batches.append(batch)
            cols += nc
        if keys:
            for key, batch in zip(keys, batches):
                self.resident.move_to_end(key)
                self.resident[key].busy += 1
                for r in batch:
                    self.pending.remove(r)
                self.inflight_keys.add(key)
            return keys, batches, 0
        seen = set()
        for req in list(self.pending):
            key = req.op_key
            if key in seen or key in self.inflight_keys:
                continue
            seen.add(key)
            batch = [r for r in self.pending if r.op_key == key]
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
                return [key], [batch], need
        return None

    def _finish(self, keys, batches, results=None, exc=None):
        """Record a job's outcome (lock not held)."""
        t1 = time.perf_counter()
        with self.lock:
            for k, (key, batch) in enumerate(zip(keys, batches)):
                if exc is None:
                    its, rel, u = results[k]
                    c = 0
                    for r in batch:
                        r.iters = list(its[c:c + r.nrhs])
                        r.relres = list(rel[c:c + r.nrhs])
                        if u is not None:
                            r.u = u[c:c + r.nrhs]
                        c += r.nrhs
                        r.t_done = t1
                    self.done.extend(batch)
                    self.log.append((t1, "done", [r.rid for r in batch]))
                else:
                    for r in batch:
                        r.t_done = t1
                        r.iters, r.relres = [-1] * r.nrhs, [math.nan] * r.nrhs
                    self.failed.extend(batch)
                if key in self.resident:
                    self.resident[key].busy -= 1
                self.inflight_keys.discard(key)
            if exc is not None:
                self.log.append((t1, "error", repr(exc)))
            self.lock.notify_all()

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
            keys, batches, reserved = job
            t0 = time.perf_counter()
            for batch in batches:
                for r in batch:
                    r.t_start = t0
            try:
                if reserved:
                    key = keys[0]
                    n, m, seed = key
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
                        self.resident[key] = _Resident(h, fbytes, busy=0)
                        self.inflight_keys.discard(key)
                        # back to the front of the queue: the next solve job
                        # takes them with every other resident operator's
                        # waiting requests
                        for r in reversed(batches[0]):
                            r.factored = True
                            self.pending.appendleft(r)
                        self.lock.notify_all()
                    continue
                with self.lock:
                    handles = [self.resident[k].handle for k in keys]
                rhs = [np.concatenate([inputs.normal_rhs(k[0], r.nrhs, 10_000 + r.rid)
                                       for r in batch]) for k, batch in zip(keys, batches)]
                if len(self.batch_sizes) < 100000:
                    self.batch_sizes.append(len(keys))
                results = self.be.solve_batch(handles, [k[0] for k in keys], rhs, stream)
            except Exception as exc:     # the job fails; the server carries on
                with self.lock:
                    self.reserved -= reserved
                self._finish(keys, batches, exc=exc)
                continue
            self._finish(keys, batches, results)

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times relative to the start); returns stats.

        realtime=False: every request is waiting when the workers start."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        self._stop = False
        threads = []
        t_base = time.perf_counter()
        if not realtime:
            with self.lock:
                for r in reqs:
                    r.arrival = t_base
                    self.pending.append(r)
            reqs = []
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
                "operators_per_solve_mean": (sum(self.batch_sizes) / len(self.batch_sizes)
                                             if self.batch_sizes else 0.0),
                "operators_per_solve_max": max(self.batch_sizes, default=0),
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
