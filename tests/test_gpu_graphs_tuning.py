"""Launch machinery around the kernels: tile shapes (set by hand or picked by
the autotuner) and the captured CUDA graphs of the MD and batch loops.  None
of it may change a result: forces accumulate in fixed point and are compared
bit for bit; energies differ only in the grouping of FP64 partial sums, and
virials in that and in which pairs share a lane's FP32 sum."""
import numpy as np
import pytest

from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _dev(s):
    torch = _torch()
    return (torch.as_tensor(s.pos, dtype=torch.float64, device="cuda"),
            torch.as_tensor(s.types, dtype=torch.int32, device="cuda"))


def _eval(tmd, m, nl, pos, types, box):
    torch = _torch()
    out = tmd.evaluate(m, nl, pos, types, box)
    torch.cuda.synchronize()
    return (float(out["energy"].item()), out["forces"].cpu().numpy().copy(), out["virial"].cpu().numpy().copy())


def test_tuning_roundtrip_and_rejection(tmdlib):
    w = I.tiny()
    m = tmdlib.Model(w.model)
    assert m.tuning == {"tile_rows": 0, "pair_blocks_per_sm": 0}
    m.tuning = {"tile_rows": 32, "pair_blocks_per_sm": 8}
    assert m.tuning == {"tile_rows": 32, "pair_blocks_per_sm": 8}
    for bad in ({"tile_rows": 48}, {"pair_blocks_per_sm": -1}, {"pair_blocks_per_sm": 65}):
        with pytest.raises(tmdlib.TmdError) as e:
            m.tuning = bad
        assert e.value.status == tmdlib.ERR_INVALID_ARG
    assert m.tuning == {"tile_rows": 32, "pair_blocks_per_sm": 8}


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_tile_shapes_do_not_change_results(tmdlib, precision):
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model, precision=precision)
    pos, types = _dev(s)
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, w.model.rc)
    e0, f0, v0 = _eval(tmdlib, m, nl, pos, types, s.box)
    for rows in (32, 64):
        for bps in (1, 4, 32):
            m.tuning = {"tile_rows": rows, "pair_blocks_per_sm": bps}
            e, f, v = _eval(tmdlib, m, nl, pos, types, s.box)
            assert np.array_equal(f, f0), (rows, bps)
            assert abs(e - e0) <= 1e-12 * abs(e0), (rows, bps)
            # the force pass sums each lane's virial terms in FP32 between
            # FP64 flushes, and the grid decides which pairs share a lane
            assert np.abs(v - v0).max() <= 1e-8 * np.abs(v0).max(), (rows, bps)


def test_autotune_keeps_a_candidate_and_the_results(tmdlib):
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    pos, types = _dev(s)
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, w.model.rc)
    e0, f0, _ = _eval(tmdlib, m, nl, pos, types, s.box)
    best = tmdlib.autotune(m, nl, pos, types, s.box)
    assert best["tile_rows"] in (32, 64)
    assert best["pair_blocks_per_sm"] in (4, 8, 16, 32)
    assert best["ms"] > 0.0
    assert m.tuning == {"tile_rows": best["tile_rows"], "pair_blocks_per_sm": best["pair_blocks_per_sm"]}
    e1, f1, _ = _eval(tmdlib, m, nl, pos, types, s.box)
    assert np.array_equal(f1, f0)
    assert abs(e1 - e0) <= 1e-12 * abs(e0)


def test_batch_autotune(tmdlib):
    w = I.batch(n_systems=6, seed=22)
    w.systems = [x for x in w.systems if x.n <= 3000][:4]
    m = tmdlib.Model(w.model)
    b = tmdlib.Batch(w.systems)
    ids = list(range(len(w.systems)))
    E0, _ = b.compute(m, ids)
    best = b.autotune(m, ids)
    assert best["tile_rows"] in (32, 64) and best["pair_blocks_per_sm"] in (4, 8, 16, 32)
    E1, _ = b.compute(m, ids)
    assert np.allclose(E1, E0, rtol=1e-12, atol=0.0)


def _md(tmd, w, graphs, stream, nsteps, rebuild_every):
    s = w.systems[0]
    m = tmd.Model(w.model)
    g = tmd.System(s.n, s.box, s.pbc, skin=1.0)
    g.set_state(s.pos, s.vel, s.types, s.masses, stream=stream)
    tmd.set_graphs(graphs)
    try:
        for _ in range(nsteps):   # one call per step: every call after the second replays
            g.step(m, 1.0, 1, rebuild_every=rebuild_every, stream=stream)
    finally:
        tmd.set_graphs(True)
    return g.get_state(stream=stream)


@pytest.mark.parametrize("rebuild_every", [1, 0])
def test_md_graph_replay_matches_eager(tmdlib, rebuild_every):
    torch = _torch()
    w = I.medium()
    w.systems[0].vel = I.maxwell_velocities(w.systems[0].masses, 300.0, np.random.default_rng(5))
    side = torch.cuda.Stream()
    r0 = tmdlib.graph_replays()
    pg, vg, fg = _md(tmdlib, w, True, side, 6, rebuild_every)
    assert tmdlib.graph_replays() - r0 >= 3           # steps 3..6 replay the captured graph
    pe, ve, fe = _md(tmdlib, w, False, side, 6, rebuild_every)
    assert np.array_equal(pg, pe) and np.array_equal(vg, ve) and np.array_equal(fg, fe)


def test_batch_graph_replay_matches_eager(tmdlib):
    torch = _torch()
    w = I.batch(n_systems=6, seed=23)
    w.systems = [x for x in w.systems if x.n <= 3000][:3]
    rng = np.random.default_rng(1)
    for x in w.systems:
        x.vel = I.maxwell_velocities(x.masses, 300.0, rng)
    m = tmdlib.Model(w.model)
    side = torch.cuda.Stream()
    ids = list(range(len(w.systems)))
    out = []
    for graphs in (True, False):
        tmdlib.set_graphs(graphs)
        try:
            b = tmdlib.Batch(w.systems)
            r0 = tmdlib.graph_replays()
            for _ in range(5):
                b.step(m, ids, 1.0, 1, stream=side)
            if graphs:
                assert tmdlib.graph_replays() - r0 >= 2
            out.append([b.get_system(k) for k in ids])
        finally:
            tmdlib.set_graphs(True)
    for a, c in zip(out[0], out[1]):
        for x, y in zip(a, c):
            assert np.array_equal(x, y)


def _md_call(tmd, w, graphs, stream, nsteps, rebuild_every, skin):
    s = w.systems[0]
    m = tmd.Model(w.model)
    g = tmd.System(s.n, s.box, s.pbc, skin=skin)
    g.set_state(s.pos, s.vel, s.types, s.masses, stream=stream)
    tmd.set_graphs(graphs)
    try:
        g.step(m, 1.0, 2, rebuild_every=rebuild_every, stream=stream)           # initial forces, off-cadence start
        th = g.step(m, 1.0, nsteps, rebuild_every=rebuild_every, stream=stream)
    finally:
        tmd.set_graphs(True)
    p, v, f = g.get_state(stream=stream)
    return p, v, f, th, g.counters()


@pytest.mark.parametrize("rebuild_every,skin,nsteps", [(5, 1.0, 33), (0, 1.0, 40), (0, 0.02, 40)])
def test_md_runs_match_step_by_step(tmdlib, rebuild_every, skin, nsteps):
    """Runs of steps decided on the device (cadence rebuild inside, skin flags
    read once per run) give the step-by-step trajectory bitwise.  The 0.02 A
    skin makes the skin criterion fire inside runs, which are then undone
    and stepped again one step at a time."""
    torch = _torch()
    w = I.medium()
    w.systems[0].vel = I.maxwell_velocities(w.systems[0].masses, 300.0, np.random.default_rng(5))
    side = torch.cuda.Stream()
    pr, vr, fr, thr, cr = _md_call(tmdlib, w, True, side, nsteps, rebuild_every, skin)
    pe, ve, fe, the, ce = _md_call(tmdlib, w, False, side, nsteps, rebuild_every, skin)
    assert np.array_equal(pr, pe) and np.array_equal(vr, ve) and np.array_equal(fr, fe)
    assert thr["rebuilds"] == the["rebuilds"] and cr["steps"] == ce["steps"] == nsteps + 2
    assert ce["runs"] == 0 and cr["runs"] + cr["reruns"] >= 2
    if skin >= 1.0:
        assert cr["reruns"] == 0 and cr["runs"] >= 2
    else:
        assert cr["reruns"] >= 1 and thr["rebuilds"] > 3
