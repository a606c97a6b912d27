"""Host scheduling of the serving loop on CPU, with the library's batch calls replaced by a fake
that finishes each admitted request after a fixed number of Newton rounds: the in-flight
footprint never exceeds the HBM budget, an environment never has two requests in flight, the
oldest waiting request that fits is admitted first (a larger one waiting does not block smaller
ones behind it), finished requests free their budget at once, and every request completes."""
import numpy as np
import pytest

from paper_2411_04776_gb300 import serving as S
from paper_2411_04776_gb300 import workloads as W


class FakeBatch:
    def __init__(self, rounds):
        self.rounds = rounds  # Newton rounds each environment's requests take
        self.left = {}
        self.submits = []
        self.resets = []

    def create(self, descs, stream=None):
        return "handle"

    def submit(self, h, ids, poses, dts):
        assert len(ids) == len(poses) == len(dts)
        for e in ids:
            assert e not in self.left
            self.left[int(e)] = self.rounds[int(e)]
        self.submits.append(list(map(int, ids)))

    def advance(self, h, n):
        done = []
        for e in list(self.left):
            self.left[e] -= 1
            if self.left[e] == 0:
                done.append(e)
                del self.left[e]
        return np.array(done, dtype=np.int64), np.zeros(len(done), dtype=np.int32)

    def reset(self, h, e):
        self.resets.append(int(e))


@pytest.fixture
def server(monkeypatch):
    wls = [W.small_gel_sphere(s, n_steps=4) for s in range(5)]
    sizes = {0: 40.0, 1: 40.0, 2: 70.0, 3: 20.0, 4: 20.0}
    fake = FakeBatch(rounds={0: 2, 1: 3, 2: 1, 3: 4, 4: 2})
    calls = iter(range(len(wls)))
    monkeypatch.setattr(S.B, "tx_gel_footprint_bytes", lambda d: sizes[next(calls)])
    monkeypatch.setattr(S.B, "tx_batch_create", fake.create)
    monkeypatch.setattr(S.B, "tx_batch_submit", fake.submit)
    monkeypatch.setattr(S.B, "tx_batch_advance", fake.advance)
    monkeypatch.setattr(S.B, "tx_batch_reset", fake.reset)
    monkeypatch.setattr(S.B, "tx_batch_destroy", lambda h: None)
    srv = S.GelServer(wls, budget_bytes=100.0)
    yield srv, fake
    srv.handle = None  # fake handle: nothing to destroy once the real binding is back


def test_admission_respects_budget_and_order(server, monkeypatch):
    srv, fake = server
    peak = []
    orig = fake.submit

    def submit(h, ids, poses, dts):
        orig(h, ids, poses, dts)
        peak.append(srv.inflight_bytes)

    monkeypatch.setattr(S.B, "tx_batch_submit", submit)
    # round 0: 0, 1, 2 ask (oldest first: 0 and 1 fit = 80, 2 (70) does not); 3 and 4 ask later
    sched = [[0, 1, 2], [3], [4], [0], [], [1, 2], [], [], [3]]
    done = srv.run_schedule(sched)
    assert fake.submits[0] == [0, 1]
    assert fake.submits[1] == [3]  # 2 (70) still does not fit beside 0 and 1; 3 (20) does
    assert max(peak) <= 100.0 and srv.max_inflight_bytes <= 100.0
    assert len(done) == sum(len(s) for s in sched)
    assert all(r.status == 0 for r in done)
    # one request per environment in flight: an environment's requests finish in order, each
    # admitted only after the previous one finished
    for e in range(5):
        mine = sorted((r for r in done if r.env == e), key=lambda r: r.step)
        for a, b in zip(mine, mine[1:]):
            assert b.admitted >= a.done
    assert srv.inflight_bytes == 0.0 and not srv.inflight


def test_environment_resets_after_its_trajectory(server):
    srv, fake = server
    done = srv.run_schedule([[3]] * 6)  # the trajectory has 4 steps: the fifth request resets it
    assert [r.step for r in done] == list(range(6))
    assert fake.resets == [3]


def test_budget_below_one_gel_is_rejected(monkeypatch):
    monkeypatch.setattr(S.B, "tx_gel_footprint_bytes", lambda d: 1e12)
    with pytest.raises(ValueError):
        S.GelServer([W.small_gel_sphere(0, n_steps=2)], budget_bytes=1e9)


def test_large_gel_is_not_starved_by_small_ones(monkeypatch):
    """A large gel that does not fit beside the small ones in flight may be passed by younger
    small requests only max_bypass times; then admission holds the budget for it."""
    wls = [W.small_gel_sphere(s, n_steps=50) for s in range(5)]
    sizes = {0: 70.0, 1: 20.0, 2: 20.0, 3: 20.0, 4: 20.0}
    fake = FakeBatch(rounds={0: 1, 1: 2, 2: 2, 3: 2, 4: 2})
    calls = iter(range(len(wls)))
    monkeypatch.setattr(S.B, "tx_gel_footprint_bytes", lambda d: sizes[next(calls)])
    monkeypatch.setattr(S.B, "tx_batch_create", fake.create)
    monkeypatch.setattr(S.B, "tx_batch_submit", fake.submit)
    monkeypatch.setattr(S.B, "tx_batch_advance", fake.advance)
    monkeypatch.setattr(S.B, "tx_batch_reset", fake.reset)
    monkeypatch.setattr(S.B, "tx_batch_destroy", lambda h: None)
    for max_bypass, admitted_by in ((3, 8), (10 ** 9, None)):
        calls = iter(range(len(wls)))
        fake.left.clear()
        fake.submits.clear()
        srv = S.GelServer(wls, budget_bytes=100.0, max_bypass=max_bypass)
        # two small environments are always busy; the large one asks at round 1
        sched = [[1, 2], [0, 3, 4]] + [[1, 2, 3, 4]] * 18
        for k, s in enumerate(sched):
            for e in s:
                if not srv.queues[e]:
                    srv.enqueue(e, float(k))
            srv._admit(float(k))
            assert srv.inflight_bytes <= 100.0
            if srv.inflight:
                srv.advance(lambda: float(k))
        first = next((k for k, ids in enumerate(fake.submits) if 0 in ids), None)
        if admitted_by is None:
            assert first is None  # without the bound the small stream keeps the large gel out
        else:
            assert first is not None and first <= admitted_by, fake.submits
        srv.handle = None
