"""Continuous batching: every request's result is the same alone and in the
mix (its system's trajectory depends only on its own requests)."""
import numpy as np
import pytest

from paper_2310_08439_gb300 import inputs as I
from paper_2310_08439_gb300 import serve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_requests_same_alone_and_in_the_mix(tmdlib, precision):
    """In the BF16 form the network tiles mix atoms of different systems; each
    tile row is computed on its own, so the trajectories stay bitwise equal."""
    w = I.serve(n_systems=6, seed=31, n_max=2000)
    m = tmdlib.Model(w.model, precision=precision)
    reqs_a = serve.poisson_requests(len(w.systems), rate=400.0, duration=0.05, seed=3, max_steps=4)
    assert len(reqs_a) >= 8
    reqs_b = [serve.Request(r.rid, r.system, r.steps, r.arrival) for r in reqs_a]
    mix = tmdlib.Batch(w.systems)
    alone = tmdlib.Batch(w.systems)
    done_mix, st_mix = serve.serve_batched(mix, m, reqs_a, realtime=False)
    done_alone, st_alone = serve.serve_alone(alone, m, reqs_b, realtime=False)
    assert st_mix["requests"] == st_alone["requests"] == len(reqs_a)
    by_id = {r.rid: r for r in done_alone}
    for r in done_mix:
        q = by_id[r.rid]
        assert r.thermo["e_pot"] == q.thermo["e_pot"], r.rid
        assert r.thermo["e_kin"] == q.thermo["e_kin"], r.rid
    for k in range(len(w.systems)):
        pa, va, fa = mix.get_system(k)
        pb, vb, fb = alone.get_system(k)
        assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    assert st_mix["calls"] < st_alone["calls"] * max(r.steps for r in reqs_a)


def test_memory_admission_waits_and_matches_alone(tmdlib):
    """A device-memory budget that holds two of three systems: the third
    system's request waits, the system is admitted once an idle system's table
    is released, and its trajectory equals the one it has alone."""
    w = I.serve(n_systems=3, seed=33, n_max=1200)
    m = tmdlib.Model(w.model)
    per = serve.bytes_per_atom(w.model)
    need = [int(s.n) * per for s in w.systems]
    budget = max(need[0] + need[1], need[0] + need[2])   # never all three at once
    assert budget < sum(need)
    reqs = [serve.Request(0, 0, 4, 0.0), serve.Request(1, 1, 1, 0.0), serve.Request(2, 2, 2, 0.0)]
    b = tmdlib.Batch(w.systems, skin=1.0, rebuild_every=5)
    res = serve.Residency(b, need, budget)
    done, st = serve.serve_batched(b, m, reqs, realtime=False, residency=res)
    assert st["requests"] == 3 and st["waited_on_memory"] >= 1 and st["releases"] >= 1, st
    assert res.used <= budget
    by = {r.rid: r for r in done}
    assert by[2].start >= by[1].done      # system 2 started after system 1 finished and was released
    alone = tmdlib.Batch([w.systems[2]], skin=1.0, rebuild_every=5)
    alone.step(m, [0], 1.0, 2)
    pa, va, fa = alone.get_system(0)
    pb, vb, fb = b.get_system(2)
    assert np.array_equal(pa, pb) and np.array_equal(va, vb) and np.array_equal(fa, fb)
    with pytest.raises(ValueError):
        serve.Residency(b, need, min(need) - 1)
