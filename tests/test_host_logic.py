"""Host-side logic that needs no GPU: workload generators, request
generation and the serving admission policy."""
import numpy as np

from paper_2310_08439_gb300 import inputs as I
from paper_2310_08439_gb300 import serve


class _FakeBatch:
    """Stands in for tmd.Batch in the host-side serving logic."""

    def __init__(self, n):
        self.n = np.array(n)
        self.released, self.ticks = [], []

    def release(self, k):
        self.released.append(k)

    def step(self, model, ids, dt, nsteps):
        self.ticks.append(list(ids))
        return [{"e_pot": 0.0, "e_kin": 0.0, "rebuilds": 0} for _ in ids]


def test_admission_waits_for_memory_and_releases_idle_systems():
    """Budget 11 with needs (5, 4, 6): systems 0 and 1 fit; system 2 waits
    until system 1 is idle, whose table is then released (system 0, still
    busy, stays)."""
    fb = _FakeBatch([50, 40, 60])
    res = serve.Residency(fb, [5, 4, 6], 11)
    reqs = [serve.Request(0, 0, 4, 0.0), serve.Request(1, 1, 1, 0.0), serve.Request(2, 2, 2, 0.0)]
    done, st = serve.serve_batched(fb, None, reqs, realtime=False, residency=res)
    by = {r.rid: r for r in done}
    assert st["requests"] == 3 and st["waited_on_memory"] == 1 and fb.released == [1]
    assert fb.ticks[0] == [0, 1] and fb.ticks[1] == [0, 2]
    assert by[2].start >= by[1].done and res.used <= 11
    assert st["atom_steps"] == 4 * 50 + 1 * 40 + 2 * 60


def test_admission_refuses_a_system_larger_than_the_budget():
    fb = _FakeBatch([50, 40])
    try:
        serve.Residency(fb, [5, 12], 11)
    except ValueError as e:
        assert "[1]" in str(e)
    else:
        raise AssertionError("a system larger than the budget was accepted")


def test_poisson_requests_rate_and_ranges():
    reqs = serve.poisson_requests(50, rate=2000.0, duration=2.0, seed=7)
    assert 3600 < len(reqs) < 4400
    arr = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(arr) > 0) and arr[-1] <= 2.0
    assert set(r.steps for r in reqs) == set(range(1, 11))
    assert min(r.system for r in reqs) >= 0 and max(r.system for r in reqs) < 50


def test_workload_shapes():
    w = I.batch()
    n = np.array([s.n for s in w.systems])
    assert len(w.systems) == 512 and 32 <= n.min() and n.max() <= 8192 * 1.1
    assert 6e5 < n.sum() < 9e5
    for s in w.systems[:20]:
        assert np.all(s.pos >= 0) and np.all(s.pos < s.box)
        L = s.box
        assert L.max() <= 2.0 * L.min() + 1e-9
    w = I.serve()
    n = np.array([s.n for s in w.systems])
    assert len(w.systems) == 256 and n.min() >= 32 and n.max() <= 55000
    assert abs(np.log(n).mean() - 0.5 * (np.log(64) + np.log(50000))) < 0.5
    t = I.tiny().systems[0]
    assert t.n == 32 and abs(t.box[0] - 7.22) < 1e-12
