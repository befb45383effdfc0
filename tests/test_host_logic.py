"""Host-side logic that needs no GPU: workload generators, request
generation and the serving admission policy."""
import numpy as np

from paper_2310_08439_gb300 import inputs as I
from paper_2310_08439_gb300 import serve


def test_admission_by_memory_budget():
    w = I.serve(n_systems=10, seed=32, n_max=3000)
    per = serve.bytes_per_atom(w.model)
    total = sum(s.n for s in w.systems) * per
    ids, used = serve.admit(w.systems, w.model, total // 2)
    assert 0 < len(ids) < len(w.systems) and used <= total // 2
    ids, used = serve.admit(w.systems, w.model, total)
    assert len(ids) == len(w.systems)


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
