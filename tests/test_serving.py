"""Serving loop: admission by predicted footprint, resident operators,
batching of right-hand sides (per operator, and across operators of
different grid sizes into one batched solve), concurrent workers.

CPU tests drive the scheduler with a fake backend whose 'solution' is a known
function of the operator and the right-hand side; the GPU tests check that a
result is bit for bit the same alone and in a concurrent mix.
"""
import threading
import time

import numpy as np
import pytest

from paper_1607_00346_gb300 import inputs
from paper_1607_00346_gb300.serving import Request, Server, leaf_size, poisson_requests


class FakeHandle:
    def __init__(self, n, seed):
        self.n, self.seed, self.released = n, seed, False


class FakeBackend:
    """Factor = sleep; solve returns u = f / (1 + seed % 7) for checking."""

    def __init__(self, per_dof=100, t_factor=0.01, t_solve=0.002):
        self.per_dof, self.t_factor, self.t_solve = per_dof, t_factor, t_solve
        self.mu = threading.Lock()
        self.live = 0
        self.peak = 0
        self.factorizations = []
        self.loads = []
        self.solve_batches = []
        self.op_batches = []

    def new_stream(self):
        return None

    def predict_bytes(self, n, m):
        return n ** 3 * self.per_dof

    def factor(self, n, m, seed, stream):
        with self.mu:
            self.live += n ** 3 * self.per_dof
            self.peak = max(self.peak, self.live)
            self.factorizations.append((n, seed))
        time.sleep(self.t_factor)
        return FakeHandle(n, seed), n ** 3 * self.per_dof

    def solve_batch(self, handles, ns, rhs_list, stream):
        time.sleep(self.t_solve)
        out = []
        with self.mu:
            self.op_batches.append(sorted((h.n, h.seed) for h in handles))
        for h, rhs in zip(handles, rhs_list):
            assert not h.released
            with self.mu:
                self.solve_batches.append(rhs.shape[0])
            out.append(([1] * rhs.shape[0], [1e-12] * rhs.shape[0], rhs / (1.0 + h.seed % 7)))
        return out

    def release(self, h):
        h.released = True
        with self.mu:
            self.live -= h.n ** 3 * self.per_dof

    def save(self, h, path):
        with open(path, "w") as fh:
            fh.write("%d %d" % (h.n, h.seed))

    def load(self, path, stream):
        with open(path) as fh:
            n, seed = map(int, fh.read().split())
        with self.mu:
            self.live += n ** 3 * self.per_dof
            self.peak = max(self.peak, self.live)
            self.loads.append((n, seed))
        return FakeHandle(n, seed), n ** 3 * self.per_dof


def _check_results(done):
    for r in done:
        f = inputs.normal_rhs(r.n, r.nrhs, 10_000 + r.rid)
        assert np.allclose(r.u, f / (1.0 + r.seed % 7))


def test_all_served_and_split_back_correctly():
    be = FakeBackend()
    srv = Server(be, mem_budget=10 * 32 ** 3 * 100, workers=3)
    reqs = poisson_requests(30, rate=400.0, sizes=[16, 24, 32], seed=1, nrhs_max=4,
                            repeat_prob=0.5)
    st = srv.run(reqs)
    assert st["requests"] == 30 and st["failed"] == 0
    _check_results(srv.done)
    assert st["p50_ms"] <= st["p99_ms"]
    assert st["solves"] == sum(r.nrhs for r in reqs)


def test_budget_respected_and_lru_eviction():
    be = FakeBackend()
    budget = 2 * 32 ** 3 * 100          # two 32^3 operators at a time
    srv = Server(be, mem_budget=budget, workers=4)
    reqs = [Request(rid=i, n=32, m=4, seed=100 + i, nrhs=1, arrival=0.001 * i) for i in range(8)]
    srv.run(reqs)
    assert be.peak <= budget
    assert len(be.factorizations) == 8
    assert sum(1 for _ in srv.resident) <= 2


def test_same_operator_batched_and_factored_once():
    be = FakeBackend(t_factor=0.05)
    srv = Server(be, mem_budget=10 ** 9, workers=2)
    # eight requests for one operator arrive while its factorization runs
    reqs = [Request(rid=i, n=16, m=4, seed=7, nrhs=2, arrival=0.0 + 0.002 * i) for i in range(8)]
    srv.run(reqs)
    assert len(be.factorizations) == 1
    assert max(be.solve_batches) > 2          # several requests shared one solve
    _check_results(srv.done)


def test_different_operators_share_one_batched_solve():
    # three operators of different grid sizes are resident when requests for
    # all of them arrive together: one job solves them all
    be = FakeBackend(t_factor=0.001, t_solve=0.05)
    srv = Server(be, mem_budget=10 ** 9, workers=1)
    warm = [Request(rid=i, n=n, m=4, seed=40 + i, nrhs=1, arrival=0.0)
            for i, n in enumerate((16, 24, 32))]
    warm[1].m = 3
    srv.run(warm, realtime=False)
    be.op_batches.clear()
    reqs = [Request(rid=10 + i, n=n, m=(3 if n == 24 else 4), seed=40 + i, nrhs=2, arrival=0.0)
            for i, n in enumerate((16, 24, 32))]
    st = srv.run(reqs, realtime=False)
    assert st["failed"] == 0 and st["requests"] == 6
    assert [(16, 40), (24, 41), (32, 42)] in be.op_batches
    assert st["operators_per_solve_max"] == 3
    _check_results(srv.done)


def test_batched_solve_respects_operator_and_column_caps():
    be = FakeBackend(t_factor=0.001, t_solve=0.02)
    srv = Server(be, mem_budget=10 ** 9, workers=1, max_ops=2, max_cols=5)
    warm = [Request(rid=i, n=16, m=4, seed=60 + i, nrhs=1, arrival=0.0) for i in range(4)]
    srv.run(warm, realtime=False)
    be.op_batches.clear()
    reqs = [Request(rid=10 + i, n=16, m=4, seed=60 + i, nrhs=2, arrival=0.0) for i in range(4)]
    srv.run(reqs, realtime=False)
    assert all(len(b) <= 2 for b in be.op_batches) and len(be.op_batches) >= 2
    _check_results(srv.done)


def test_oversized_request_is_refused_and_others_served():
    be = FakeBackend()
    srv = Server(be, mem_budget=16 ** 3 * 100, workers=2)
    reqs = [Request(rid=0, n=32, m=4, seed=1, nrhs=1, arrival=0.0),     # too large
            Request(rid=1, n=16, m=4, seed=2, nrhs=2, arrival=0.001)]
    st = srv.run(reqs)
    assert st["failed"] == 1 and st["requests"] == 1
    assert srv.failed[0].rid == 0
    _check_results(srv.done)


def test_evicted_operators_spill_to_disk_and_come_back(tmp_path):
    be = FakeBackend(per_dof=100)
    # room for one 16^3 operator at a time: A, B, A, B ... forces evictions
    srv = Server(be, mem_budget=16 ** 3 * 100 + 10, workers=1, spill_dir=str(tmp_path))
    reqs = []
    for i in range(6):
        seed = 1 if i % 2 == 0 else 2
        reqs.append(Request(rid=i, n=16, seed=seed, nrhs=1, arrival=0.05 * i))
    srv.run(reqs, realtime=True)
    srv.release_all()
    assert len(srv.done) == 6 and not srv.failed
    _check_results(srv.done)
    # each operator is factored once; later uses come back from disk
    assert sorted(be.factorizations) == [(16, 1), (16, 2)]
    assert len(be.loads) >= 1
    assert be.peak <= srv.budget


def test_leaf_sizes():
    assert [leaf_size(n) for n in (16, 32, 48, 64, 96, 128)] == [4, 4, 3, 4, 3, 4]


@pytest.mark.gpu
def test_gpu_result_same_alone_and_in_the_mix():
    # the serving workload's sizes (32^3 - 64^3 here, m = 3 for 48^3) with
    # 1-16 right-hand sides: a Poisson mix on four workers, then a burst of
    # requests for the resident operators that one batched solve serves
    # together (grids of different sizes in shared apply launches); each
    # result is bit for bit the one its request gets when served alone
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00346_gb300 import build
    from paper_1607_00346_gb300.serving import HifBackend
    build.build_library()
    be = HifBackend(eps=1e-6, precision=1, keep_u=True)
    mix = poisson_requests(12, rate=40.0, sizes=[32, 48, 64], seed=5, nrhs_max=16,
                           repeat_prob=0.3)
    srv = Server(be, mem_budget=40 << 30, workers=4)
    st = srv.run(mix)
    assert st["requests"] == 12 and st["failed"] == 0
    ops = sorted({r.op_key for r in mix})
    burst = [Request(rid=100 + i, n=n, m=m, seed=seed, nrhs=1 + (5 * i) % 16, arrival=0.0)
             for i, (n, m, seed) in enumerate(ops)]
    srv.batch_sizes.clear()
    srv.max_cols = 1000
    st2 = srv.run(burst, realtime=False)
    assert st2["failed"] == 0 and st2["operators_per_solve_max"] == min(len(ops), srv.max_ops)
    assert len({n for n, _, _ in ops}) >= 2
    srv.release_all()
    for r in srv.done:
        assert max(r.relres) <= 1e-10
        alone = Server(be, mem_budget=40 << 30, workers=1)
        alone.run([Request(rid=r.rid, n=r.n, m=r.m, seed=r.seed, nrhs=r.nrhs, arrival=0.0)])
        a = alone.done[0]
        alone.release_all()
        assert np.array_equal(a.u, r.u), r.rid
        assert a.iters == r.iters


@pytest.mark.gpu
def test_gpu_spilled_operator_gives_the_same_solution(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00346_gb300 import build
    from paper_1607_00346_gb300.serving import HifBackend
    build.build_library()
    be = HifBackend(eps=1e-6, precision=1, keep_u=True)
    one = be.predict_bytes(16, 4)
    # room for one new operator next to a resident one (admission uses the
    # predicted footprint): alternating requests evict, spill and reload
    srv = Server(be, mem_budget=int(1.05 * one), workers=1, spill_dir=str(tmp_path))
    reqs = [Request(rid=i, n=16, seed=11 + (i % 2), nrhs=2, arrival=0.3 * i) for i in range(4)]
    st = srv.run(reqs)
    srv.release_all()
    assert st["requests"] == 4 and st["failed"] == 0
    assert any(ev == "load" for _, ev, _ in srv.log)
    first = {}
    for r in sorted(srv.done, key=lambda r: r.rid):
        assert max(r.relres) <= 1e-10
        alone = Server(be, mem_budget=8 << 30, workers=1)
        alone.run([Request(rid=r.rid, n=r.n, m=r.m, seed=r.seed, nrhs=r.nrhs, arrival=0.0)])
        a = alone.done[0]
        alone.release_all()
        # a reloaded factor is bitwise the saved one: the same solution
        assert np.array_equal(a.u, r.u)
        first.setdefault(r.seed, r)
