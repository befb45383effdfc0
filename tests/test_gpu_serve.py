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
