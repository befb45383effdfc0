"""Batches (many resident systems evaluated by one set of launches) against
single-system evaluations and the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _single(tmd, model, s):
    import torch
    m = tmd.Model(model)
    nl = tmd.NeighborList()
    pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
    types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
    nl.build(pos, types, s.box, s.pbc, model.rc)
    out = tmd.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    return (float(out["energy"].item()), out["forces"].double().cpu().numpy(),
            out["virial"].cpu().numpy().reshape(3, 3))


@pytest.fixture(scope="module")
def small_batch():
    w = I.batch(n_systems=10, seed=21)
    # keep the test quick: drop the largest systems
    w.systems = [s for s in w.systems if s.n <= 3000][:8]
    return w


def test_batch_equals_single_and_oracle(tmdlib, small_batch):
    w = small_batch
    m = tmdlib.Model(w.model)
    b = tmdlib.Batch(w.systems)
    ids = list(range(len(w.systems)))
    E, W = b.compute(m, ids)
    om = O.OracleModel(w.model)
    for k, s in enumerate(w.systems):
        e1, f1, w1 = _single(tmdlib, w.model, s)
        _, _, fb = b.get_system(k)
        assert abs(E[k] - e1) <= 1e-12 * abs(e1) + 1e-9, k
        assert np.abs(fb - f1).max() <= 1e-6 * max(np.abs(f1).max(), 1e-6), k
        assert np.abs(W[k] - w1).max() <= 1e-6 * max(np.abs(w1).max(), 1e-6), k
        if s.n <= 1200:
            o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
            rms = np.sqrt((o["forces"] ** 2).mean())
            assert abs(E[k] - o["energy"]) <= 1e-6 * abs(o["energy"]), k
            assert np.abs(fb - o["forces"]).max() <= 1e-5 * rms, k
            assert np.abs(W[k] - o["virial"]).max() <= 1e-5 * np.abs(o["virial"]).max(), k


@pytest.mark.parametrize("kind", ["tcgen05", "mma_sync"])
def test_bf16_batch_equals_single(tmdlib, small_batch, kind):
    """BF16 network form: the batch's network tiles hold atoms of several
    systems, and each tile row is computed on its own, so every system's
    result equals its single evaluation (up to the FP32 rounding of the
    descriptors, which the BF16 rounding of the network input can amplify to
    BF16 size on single elements)."""
    import torch
    w = small_batch
    try:
        tmdlib.set_network_kernel(kind)
        m = tmdlib.Model(w.model, precision="bf16")
        b = tmdlib.Batch(w.systems)
        E, _ = b.compute(m, list(range(len(w.systems))))
        for k, s in enumerate(w.systems):
            nl = tmdlib.NeighborList()
            pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
            types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
            nl.build(pos, types, s.box, s.pbc, w.model.rc)
            out = tmdlib.evaluate(m, nl, pos, types, s.box)
            torch.cuda.synchronize()
            _, _, fb = b.get_system(k)
            f1 = out["forces"].double().cpu().numpy()
            rms = np.sqrt((f1 ** 2).mean())
            assert np.sqrt(((fb - f1) ** 2).mean()) <= 1e-3 * rms, k
            assert abs(E[k] - float(out["energy"].item())) <= 1e-6 * abs(E[k]), k
    finally:
        tmdlib.set_network_kernel("auto")
    assert tmdlib.device_status() == 0


def test_batch_subset_leaves_others_untouched(tmdlib, small_batch):
    w = small_batch
    m = tmdlib.Model(w.model)
    b = tmdlib.Batch(w.systems)
    E_all, _ = b.compute(m, list(range(len(w.systems))))
    before = [b.get_system(k)[2].copy() for k in range(len(w.systems))]
    sub = [5, 1, 3]
    E_sub, _ = b.compute(m, sub)
    for j, k in enumerate(sub):
        assert E_sub[j] == E_all[k]
    for k in range(len(w.systems)):
        assert np.array_equal(b.get_system(k)[2], before[k])


def test_batch_step_matches_system_step(tmdlib, small_batch):
    w = small_batch
    m = tmdlib.Model(w.model)
    systems = [s for s in w.systems[:3]]
    rng = np.random.default_rng(0)
    for s in systems:
        s.vel = I.maxwell_velocities(s.masses, 300.0, rng)
    b = tmdlib.Batch(systems)
    th = b.step(m, [0, 1, 2], 1.0, 5)
    for k, s in enumerate(systems):
        g = tmdlib.System(s.n, s.box, s.pbc, skin=0.0)
        g.set_state(s.pos, s.vel, s.types, s.masses)
        ths = g.step(m, 1.0, 5, rebuild_every=1)
        p1, v1, f1 = g.get_state()
        p2, v2, f2 = b.get_system(k)
        d = p2 - p1
        d -= np.rint(d / s.box) * s.box
        assert np.abs(d).max() < 1e-10, k
        assert np.abs(v2 - v1).max() < 1e-10, k
        assert abs(th[k]["e_pot"] - ths["e_pot"]) <= 1e-9 * abs(ths["e_pot"]), k
        assert abs(th[k]["e_kin"] - ths["e_kin"]) <= 1e-9 * abs(ths["e_kin"]) + 1e-12, k


@pytest.mark.parametrize("k", [285, 68])
def test_fp32_batch_network_small_force_systems(tmdlib, k):
    """Two systems of the 512-system workload whose net forces are small
    against the pair terms (RMS ~0.004 eV/A): the FP32 path must still be
    within 1e-5 of the force RMS (the 192-128-128 network's input gradient
    is the largest error source there)."""
    w = I.batch()
    s = w.systems[k]
    e, f, v = _single(tmdlib, w.model, s)
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    rms = np.sqrt((o["forces"] ** 2).mean())
    assert abs(e - o["energy"]) <= 1e-6 * abs(o["energy"])
    assert np.abs(f - o["forces"]).max() <= 1e-5 * rms
    assert np.abs(v - o["virial"]).max() <= 1e-5 * np.abs(o["virial"]).max()


@pytest.mark.parametrize("skin,every", [(1.0, 5), (0.03, 0)])
def test_resident_tables_follow_tmd_step(tmdlib, skin, every):
    """Resident neighbour tables (rc + skin, rebuilt per system on the cadence
    or by the skin criterion, Sec. "Evaluation"): every system of a batch of
    uneven systems follows, bitwise, its own tmd_step trajectory with the same
    table policy, and the batch counts the same table builds.  The 0.03 A skin
    makes the skin criterion fire at different steps in different systems."""
    w = I.serve(n_systems=6, seed=31, n_max=2000)
    m = tmdlib.Model(w.model)
    b = tmdlib.Batch(w.systems, skin=skin, rebuild_every=every)
    ids = list(range(len(w.systems)))
    nsteps = 12
    th_b = b.step(m, ids, 1.0, nsteps)
    rebuilds = []
    for k, s in enumerate(w.systems):
        sy = tmdlib.System(s.n, s.box, s.pbc, skin)
        sy.set_state(s.pos, s.vel, s.types, s.masses)
        th = sy.step(m, 1.0, nsteps, rebuild_every=every)
        p, v, f = sy.get_state()
        pb, vb, fb = b.get_system(k)
        assert np.array_equal(p, pb) and np.array_equal(v, vb) and np.array_equal(f, fb), k
        assert th_b[k]["rebuilds"] == th["rebuilds"], (k, th_b[k]["rebuilds"], th["rebuilds"])
        assert abs(th_b[k]["e_pot"] - th["e_pot"]) <= 1e-9 * abs(th["e_pot"]), k
        rebuilds.append(th["rebuilds"])
    if every:
        assert all(r == 1 + nsteps // every for r in rebuilds), rebuilds
    else:
        assert len(set(rebuilds)) > 1 and max(rebuilds) > 1, rebuilds


def test_released_table_is_rebuilt_with_the_same_forces(tmdlib):
    """A released system keeps its state; its next evaluation builds a new
    table in a (reused) pool region and gives the same forces."""
    w = I.serve(n_systems=4, seed=32, n_max=1500)
    m = tmdlib.Model(w.model)
    b = tmdlib.Batch(w.systems, skin=1.0, rebuild_every=0)
    ids = list(range(len(w.systems)))
    b.compute(m, ids)
    f0 = [b.get_system(k)[2] for k in ids]
    reg0, pool0, builds0 = b.table_info(1)
    assert reg0 > 0 and pool0 >= reg0 and builds0 == 1
    b.release(1)
    assert b.table_info(1)[0] == 0
    b.compute(m, [1, 3])
    reg1, pool1, builds1 = b.table_info(1)
    assert reg1 > 0 and builds1 == 2 and pool1 == pool0    # the released region was reused
    for k in ids:
        assert np.array_equal(b.get_system(k)[2], f0[k]), k


def test_resident_table_and_owned_call_argument_errors(tmdlib):
    """The batch's table calls and the owned-centre evaluation reject bad
    arguments with TMD_ERR_INVALID_ARG before touching the GPU."""
    import torch
    w = I.medium()
    s = w.systems[0]
    b = tmdlib.Batch([s], skin=1.0)
    for bad in (lambda: b.set_skin(-1.0), lambda: b.set_skin(float("nan")), lambda: b.set_skin(1.0, -1),
                lambda: b.release(1), lambda: b.release(-1), lambda: b.table_info(1)):
        with pytest.raises(tmdlib.TmdError) as e:
            bad()
        assert e.value.status == tmdlib.ERR_INVALID_ARG
    m = tmdlib.Model(w.model)
    pos = torch.as_tensor(s.pos, device="cuda")
    types = torch.as_tensor(s.types, device="cuda")
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, w.model.rc)
    for n_owned in (-1, s.n + 1):
        with pytest.raises(tmdlib.TmdError) as e:
            tmdlib.compute_owned(m, nl, pos, types, n_owned, s.box,
                                 energy=torch.zeros(1, dtype=torch.float64, device="cuda"))
        assert e.value.status == tmdlib.ERR_INVALID_ARG
