"""Host logic of the continuous-batching loop, with a stand-in executor
(no GPU): slots and the memory budget bound what is in flight, admission is
in arrival order, a decompress waits for the record it reads, latency
accounting and quantiles."""
import pytest

from paper_2507_11165_gb300 import serve
from paper_2507_11165_gb300.serve import FakeExecutor, Request, Server


def _max_concurrency(log):
    cur = best = 0
    for e in log:
        if e[0] == "submit":
            cur += 1
            best = max(best, cur)
        else:
            cur -= 1
    return best


def test_slots_bound_concurrency_and_fifo():
    reqs = [Request(id=i, t=0.0, op="compress", side=16, eb=1e-3) for i in range(10)]
    ex = FakeExecutor(lambda r: 0.004)
    sv = Server(ex, slots=3, budget_bytes=10 ** 12)
    done = sv.run(reqs)
    assert sorted(d.id for d in done) == list(range(10))
    assert _max_concurrency(ex.log) == 3 and sv.peak_concurrency == 3
    submits = [e[1] for e in ex.log if e[0] == "submit"]
    assert submits == list(range(10))  # arrival order
    for d in done:
        assert d.latency >= 0.004 - 1e-9 and d.status == 0
    # ten requests of 4 ms through three slots: at least four rounds
    assert max(d.t_done for d in done) >= 4 * 0.004 - 1e-6


def test_budget_bounds_bytes_in_flight():
    big = serve.device_bytes("compress", 64)
    reqs = [Request(id=i, t=0.0, op="compress", side=64, eb=1e-3) for i in range(4)]
    ex = FakeExecutor(lambda r: 0.003)
    sv = Server(ex, slots=8, budget_bytes=int(1.5 * big), keep_records=0)
    sv.run(reqs)
    assert _max_concurrency(ex.log) == 1  # one big request at a time fits
    assert sv.peak_bytes <= 1.5 * big


def test_requests_arriving_later_join_while_others_run():
    reqs = [Request(id=0, t=0.0, op="compress", side=8, eb=1e-3),
            Request(id=1, t=0.002, op="compress", side=8, eb=1e-3)]
    ex = FakeExecutor(lambda r: 0.02)
    sv = Server(ex, slots=4, budget_bytes=10 ** 12)
    done = {d.id: d for d in sv.run(reqs)}
    # the second is admitted while the first still runs (continuous batching, not a queue)
    assert done[1].t_admit < done[0].t_done
    assert sv.peak_concurrency == 2


def test_decompress_waits_for_its_record_and_falls_back_when_dropped():
    reqs = [Request(id=0, t=0.0, op="compress", side=8, eb=1e-3),
            Request(id=1, t=0.001, op="decompress", side=8, eb=1e-3, source=0)]
    ex = FakeExecutor(lambda r: 0.01)
    sv = Server(ex, slots=4, budget_bytes=10 ** 12)
    done = {d.id: d for d in sv.run(reqs)}
    assert done[1].op == "decompress"
    assert done[1].t_admit >= done[0].t_done - 1e-9  # admitted only once the record exists
    # keep no records: the decompress becomes a compress of its snapshot
    ex = FakeExecutor(lambda r: 0.002)
    sv = Server(ex, slots=4, budget_bytes=10 ** 12, keep_records=0)
    reqs[1] = Request(id=1, t=0.02, op="decompress", side=8, eb=1e-3, source=0)
    done = {d.id: d for d in sv.run(reqs)}
    assert done[1].op == "compress"


def test_request_larger_than_budget_is_refused():
    ex = FakeExecutor(lambda r: 0.001)
    sv = Server(ex, slots=2, budget_bytes=1000)
    with pytest.raises(RuntimeError):
        sv.run([Request(id=0, t=0.0, op="compress", side=32, eb=1e-3)])


def test_summary_quantiles():
    done = [serve.Done(i, "compress", 0.0, 0.0, (i + 1) * 1e-3, 4000, 0) for i in range(100)]
    s = serve.summarize(done, wall_s=1.0)
    assert s["n"] == 100 and s["failed"] == 0
    assert abs(s["p50_ms"] - 50.0) < 1e-9 and abs(s["p99_ms"] - 99.0) < 1e-9 and abs(s["max_ms"] - 100.0) < 1e-9
    assert abs(s["gbs"] - 100 * 4000 / 1e9) < 1e-15


def test_request_stream_recipe():
    reqs = serve.make_requests(n=300, rate=200.0, seed=5)
    assert len(reqs) == 300
    ts = [r.t for r in reqs]
    assert ts == sorted(ts)
    assert 0.8 * 1.5 < ts[-1] < 1.25 * 1.5  # 300 arrivals at 200 / s
    assert all(64 <= r.side <= 512 for r in reqs)
    ids = {r.id: r for r in reqs}
    for r in reqs:
        if r.op == "decompress":
            src = ids[r.source]
            assert src.op == "compress" and src.t < r.t and src.side == r.side
    frac = sum(r.op == "decompress" for r in reqs) / len(reqs)
    assert 0.35 < frac < 0.6


class _GrowingExecutor(FakeExecutor):
    """A stand-in whose request 0 re-runs with larger outlier arrays after its first poll."""

    def __init__(self, extra):
        super().__init__(lambda r: 0.01)
        self.extra = extra
        self.polled = set()

    def poll(self, h):
        self.polled.add(h[0].id)
        return super().poll(h)

    def extra_bytes(self, h):
        return self.extra if (h[0].id == 0 and 0 in self.polled) else 0


def test_capacity_rerun_counts_in_the_budget():
    need = serve.device_bytes("compress", 16)
    extra = 5 * need
    reqs = [Request(id=0, t=0.0, op="compress", side=16, eb=1e-3)]
    ex = _GrowingExecutor(extra)
    sv = Server(ex, slots=2, budget_bytes=10 ** 12, keep_records=4)
    sv.run(reqs)
    assert sv.peak_bytes >= need + extra  # the grown request was counted while in flight
    assert sv.bytes_in_flight == 0
    assert sv.records[0] == ex.record_bytes(reqs[0]) + extra  # and its kept record holds the larger arrays
