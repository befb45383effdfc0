"""Tabulated radial basis (Sec. "The H_abck tensor and Batch Rational 1D
Interpolation") on the GPU, through the C ABI.

With a table the GPU path interpolates H and H' between grid points instead of
evaluating the Gaussians and the cutoff; the oracle interpolates the same grid
in FP64, so the parity bars are those of the direct path (|dE| <= 1e-6 |E|,
max |dF| <= 1e-5 RMS(F), max |dW| <= 1e-5 max |W|).  Against the direct
oracle the difference is the interpolation error, which shrinks as h^3 in the
forces; it is printed for the record and bounded loosely.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5


def _torch():
    import torch
    return torch


def _eval(tmd, m, s, r_list):
    torch = _torch()
    nl = tmd.NeighborList()
    pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
    types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
    nl.build(pos, types, s.box, s.pbc, r_list)
    out = tmd.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    return {"energy": float(out["energy"].item()), "forces": out["forces"].double().cpu().numpy(),
            "virial": out["virial"].cpu().numpy().reshape(3, 3)}


def _errs(g, o):
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    return (abs(g["energy"] - o["energy"]) / abs(o["energy"]),
            float(np.abs(g["forces"] - o["forces"]).max()) / rms,
            float(np.abs(g["virial"] - o["virial"]).max()) / float(np.abs(o["virial"]).max()))


@pytest.mark.parametrize("wname,ppa", [("tiny", 16), ("tiny", 256), ("medium", 32), ("medium", 128)])
def test_table_parity_with_tabulated_oracle(tmdlib, wname, ppa):
    w = getattr(I, wname)()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    m.set_radial_table(ppa)
    g = _eval(tmdlib, m, s, w.model.rc + (0.0 if wname == "tiny" else 1.0))
    o = O.evaluate(O.OracleModel(w.model, radial_table=ppa), s.pos, s.types, s.box, s.pbc)
    dE, dF, dW = _errs(g, o)
    d = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    iE, iF, iW = _errs(g, d)
    print(f"{wname} ppa {ppa}: vs tabulated oracle dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}; "
          f"vs direct oracle dE/E={iE:.2e} dF/rms={iF:.2e} dW/max={iW:.2e}")
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL
    if ppa >= 128:   # interpolation error below the FP32 bars
        assert iE <= E_TOL and iF <= F_TOL and iW <= W_TOL


@pytest.mark.parametrize("K,S,widths", [(8, 3, [12, 8]), (16, 4, [8, 8, 8]), (32, 2, [16]), (32, 3, [8, 12])])
def test_table_model_shapes(tmdlib, K, S, widths):
    """Every (K, S) kernel instance with a table, on a ragged multi-species cell."""
    rng = np.random.default_rng(K * 10 + S + 1)
    pos, box = I.lattice("bcc", (4, 4, 3), 3.1)
    s = I.System(I.jitter_and_wrap(pos, box, 0.12, rng), rng.integers(0, S, len(pos)).astype(np.int32),
                 box, np.ones(3, np.int32))
    p = I.random_model(S, K, 5.5, widths, seed=K + S)
    om = O.OracleModel(p)
    G = O.evaluate(om, s.pos, s.types, s.box, s.pbc, want_G=True)["G"]
    rms = np.sqrt((G ** 2).mean(axis=0)).reshape(1, -1)
    p = I.random_model(S, K, 5.5, widths, seed=K + S, feature_scale=np.repeat(np.maximum(rms, 1e-2), S, axis=0))
    m = tmdlib.Model(p)
    m.set_radial_table(64)
    g = _eval(tmdlib, m, s, p.rc)
    o = O.evaluate(O.OracleModel(p, radial_table=64), s.pos, s.types, s.box, s.pbc)
    dE, dF, dW = _errs(g, o)
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (dE, dF, dW)


def test_table_switch_and_rejection(tmdlib):
    """0 returns to direct evaluation bit for bit; a rejected size keeps the
    table in use."""
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    d0 = _eval(tmdlib, m, s, w.model.rc)
    m.set_radial_table(64)
    t0 = _eval(tmdlib, m, s, w.model.rc)
    assert not np.array_equal(t0["forces"], d0["forces"])
    for bad in (-1, 8, 48, 2048):
        with pytest.raises(tmdlib.TmdError) as e:
            m.set_radial_table(bad)
        assert e.value.status == tmdlib.ERR_INVALID_ARG
    t1 = _eval(tmdlib, m, s, w.model.rc)
    assert np.array_equal(t1["forces"], t0["forces"])
    m.set_radial_table(0)
    d1 = _eval(tmdlib, m, s, w.model.rc)
    assert np.array_equal(d1["forces"], d0["forces"]) and d1["energy"] == d0["energy"]


def test_table_in_batches(tmdlib):
    w = I.batch(n_systems=10, seed=24)
    w.systems = [x for x in w.systems if x.n <= 1200][:4]
    m = tmdlib.Model(w.model)
    m.set_radial_table(128)
    b = tmdlib.Batch(w.systems)
    ids = list(range(len(w.systems)))
    E, W = b.compute(m, ids)
    om = O.OracleModel(w.model, radial_table=128)
    for k, s in enumerate(w.systems):
        o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
        _, _, fb = b.get_system(k)
        rms = np.sqrt((o["forces"] ** 2).mean())
        assert abs(E[k] - o["energy"]) <= E_TOL * abs(o["energy"]), k
        assert np.abs(fb - o["forces"]).max() <= F_TOL * rms, k
        assert np.abs(W[k] - o["virial"]).max() <= W_TOL * np.abs(o["virial"]).max(), k


def test_table_noalloc_matches_compute(tmdlib):
    torch = _torch()
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    m.set_radial_table(128)
    nl = tmdlib.NeighborList()
    pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
    types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
    nl.build(pos, types, s.box, s.pbc, w.model.rc + 1.0)
    off, nbr, sh = nl.export()
    shift4 = np.zeros((len(nbr), 4), np.int8)
    shift4[:, :3] = sh
    shift4[:, 3] = s.types[nbr]
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")

    def outputs():
        return (torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(s.n, dtype=torch.float32, device="cuda"),
                torch.zeros((s.n, 3), dtype=torch.float32, device="cuda"),
                torch.zeros(9, dtype=torch.float64, device="cuda"))
    ref, out = outputs(), outputs()
    tmdlib.compute(m, nl, pos, types, s.box, *ref)
    tmdlib.compute_noalloc(m, dev(off, torch.int64), dev(nbr, torch.int32), dev(shift4, torch.int8), pos, types,
                           s.box, *out)
    torch.cuda.synchronize()
    rE, _, rF, rW = (t.double().cpu().numpy() for t in ref)
    E, _, F, W = (t.double().cpu().numpy() for t in out)
    rms = np.sqrt((rF ** 2).mean())
    assert abs(E[0] - rE[0]) <= E_TOL * abs(rE[0])
    assert np.abs(F - rF).max() <= F_TOL * rms
    assert np.abs(W - rW).max() <= W_TOL * np.abs(rW).max()


def test_table_md_graph_replay_matches_eager(tmdlib):
    """A captured MD step replays with the table, and switching the table on
    after capture takes a new graph (the table is part of the graph's key)."""
    torch = _torch()
    w = I.medium()
    s = w.systems[0]
    s.vel = I.maxwell_velocities(s.masses, 300.0, np.random.default_rng(6))
    side = torch.cuda.Stream()
    res = []
    for graphs in (True, False):
        m = tmdlib.Model(w.model)
        g = tmdlib.System(s.n, s.box, s.pbc, skin=1.0)
        g.set_state(s.pos, s.vel, s.types, s.masses, stream=side)
        tmdlib.set_graphs(graphs)
        try:
            for step in range(8):
                if step == 4:
                    m.set_radial_table(128)
                g.step(m, 1.0, 1, rebuild_every=1, stream=side)
        finally:
            tmdlib.set_graphs(True)
        res.append(g.get_state(stream=side))
    for a, b in zip(res[0], res[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("ppa", [64, 256])
def test_embedding_network_radial_table(tmdlib, ppa):
    """Radial functions from an embedding network (given as a table of H, H')
    on the GPU against the oracle built from the same table.  The network's
    first layer is normalised by the descriptor RMS of this radial basis (as
    every workload's model is), so that the comparison is well conditioned."""
    rng = np.random.default_rng(ppa)
    pos, box = I.lattice("fcc", (5, 5, 4), 3.61)
    s = I.System(I.jitter_and_wrap(pos, box, 0.1, rng), rng.integers(0, 2, len(pos)).astype(np.int32), box,
                 np.ones(3, np.int32))
    S, K, rc, widths = 2, 16, 6.0, [32, 32]
    H, dH = I.embedding_radial_table(S, K, rc, ppa, seed=11)
    p0 = I.random_model(S, K, rc, widths, seed=12)
    G = O.evaluate(O.OracleModel(p0, radial_table=ppa, table_values=(H, dH)), s.pos, s.types, s.box, s.pbc,
                   want_G=True)["G"]
    rms = np.sqrt((G ** 2).mean(axis=0)).reshape(1, -1)
    p = I.random_model(S, K, rc, widths, seed=12, feature_scale=np.repeat(rms, S, axis=0))
    m = tmdlib.Model(p)
    m.set_radial_table_values(ppa, H, dH)
    g = _eval(tmdlib, m, s, rc)
    o = O.evaluate(O.OracleModel(p, radial_table=ppa, table_values=(H, dH)), s.pos, s.types, s.box, s.pbc)
    dE, dF, dW = _errs(g, o)
    print(f"embedding-net table ppa {ppa}: dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}")
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL
    # back to the model's Gaussians: a different potential
    m.set_radial_table(0)
    d = _eval(tmdlib, m, s, rc)
    assert not np.allclose(d["forces"], g["forces"])


def test_table_values_rejected(tmdlib):
    w = I.tiny()
    p = w.model
    H, dH = I.embedding_radial_table(p.n_species, p.n_radial, p.rc, 64, seed=1)
    m = tmdlib.Model(p)
    bad = [(48, H, dH), (64, H[:, :, :-1], dH[:, :, :-1]), (64, np.where(H == H, np.nan, H), dH)]
    for ppa, h, d in bad:
        with pytest.raises(tmdlib.TmdError) as e:
            m.set_radial_table_values(ppa, h, d)
        assert e.value.status == tmdlib.ERR_INVALID_ARG
