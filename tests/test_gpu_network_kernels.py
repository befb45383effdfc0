"""The two kernels of the BF16 network form: tcgen05 (tensor memory, 128-atom
tiles) and mma.sync (64-atom tiles).  Both take BF16 operands with FP32
accumulation, so each is held to the BF16 bounds against the FP64 oracle and
the two agree to well within those bounds; the tcgen05 kernel's bounded waits
must not have run out."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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
    return {"energy": float(out["energy"].item()), "e_atom": out["e_atom"].double().cpu().numpy(),
            "forces": out["forces"].double().cpu().numpy(), "virial": out["virial"].cpu().numpy().reshape(3, 3)}


def _cases():
    tiny, medium, batch = I.tiny(), I.medium(), I.batch(n_systems=12, seed=31)
    bs = [x for x in batch.systems if 600 <= x.n <= 2500][0]
    return {"tiny": (tiny.model, tiny.systems[0], tiny.model.rc),
            "medium": (medium.model, medium.systems[0], medium.model.rc + 1.0),
            "batch_model": (batch.model, bs, batch.model.rc)}


@pytest.mark.parametrize("case", ["tiny", "medium", "batch_model"])
def test_tcgen05_and_mma_sync_agree(tmdlib, case, capsys):
    p, s, r_list = _cases()[case]
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    res = {}
    try:
        for kind in ("tcgen05", "mma_sync"):
            tmdlib.set_network_kernel(kind)
            res[kind] = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, r_list)
    finally:
        tmdlib.set_network_kernel("auto")
    assert tmdlib.device_status() == 0
    lines = []
    for kind, g in res.items():
        dE = abs(g["energy"] - o["energy"]) / abs(o["energy"])
        dF = np.abs(g["forces"] - o["forces"]).max() / rms
        dFr = np.sqrt(((g["forces"] - o["forces"]) ** 2).mean()) / rms
        lines.append(f"{kind}: dE/E={dE:.2e} max|dF|/rms={dF:.2e} rms(dF)/rms={dFr:.2e}")
        assert dE < 1e-3 and dFr < 5e-2 and dF < 0.5, (kind, dE, dFr, dF)
    a, b = res["tcgen05"], res["mma_sync"]
    cross = np.sqrt(((a["forces"] - b["forces"]) ** 2).mean()) / rms
    ea = np.abs(a["e_atom"] - b["e_atom"]).max()
    with capsys.disabled():
        print(f"\n[{case}] " + "; ".join(lines) + f"; tcgen05 vs mma.sync rms(dF)/rms={cross:.2e} max|dEa|={ea:.2e}")
    assert cross < 2e-2
    assert ea < 5e-3 * max(1.0, np.abs(b["e_atom"]).max())


def test_tcgen05_ragged_tiles_and_species_boundaries(tmdlib):
    """Atom counts that leave a partial last tile, and tiles holding two
    species (perm order groups atoms by species)."""
    rng = np.random.default_rng(9)
    pos, box = I.lattice("fcc", (5, 4, 3), 3.6)    # 240 atoms: one full and one partial 128-atom tile
    s = I.System(I.jitter_and_wrap(pos, box, 0.1, rng), rng.integers(0, 3, len(pos)).astype(np.int32), box,
                 np.ones(3, np.int32))
    p = I.random_model(3, 16, 5.0, [48, 32], seed=4)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    res = {}
    try:
        for kind in ("tcgen05", "mma_sync"):
            tmdlib.set_network_kernel(kind)
            res[kind] = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, p.rc)
    finally:
        tmdlib.set_network_kernel("auto")
    assert tmdlib.device_status() == 0
    g = res["tcgen05"]
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) < 1e-3
    assert np.sqrt(((g["forces"] - o["forces"]) ** 2).mean()) / rms < 5e-2
    assert np.sqrt(((g["forces"] - res["mma_sync"]["forces"]) ** 2).mean()) / rms < 2e-2


def test_network_kernel_selection(tmdlib):
    # accumulators plus stored derivatives beyond 512 TMEM columns: mma.sync only
    p = I.random_model(1, 16, 5.0, [256, 256, 256], seed=2)
    s = I.tiny().systems[0]
    try:
        tmdlib.set_network_kernel("tcgen05")
        with pytest.raises(tmdlib.TmdError) as e:
            _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, p.rc)
        assert e.value.status == tmdlib.ERR_UNIMPLEMENTED
        tmdlib.set_network_kernel("auto")   # falls back to mma.sync
        g = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, p.rc)
        assert np.isfinite(g["energy"])
        with pytest.raises(tmdlib.TmdError) as e:
            tmdlib.check(tmdlib.lib().tmd_set_network_kernel(7))
        assert e.value.status == tmdlib.ERR_INVALID_ARG
    finally:
        tmdlib.set_network_kernel("auto")


def test_bounded_wait_gives_up_and_the_context_survives(tmdlib):
    """Failure detection without a fault: the self-test kernel waits on an
    mbarrier that nothing signals; the bounded wait gives up, the status word
    reports the timeout once, and the next tensor-core evaluation is normal."""
    assert tmdlib.device_status() == 0
    assert tmdlib.selftest_bounded_wait()
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.device_status()
    assert e.value.status == tmdlib.ERR_TIMEOUT
    assert tmdlib.device_status() == 0          # read and cleared
    p, s, r_list = _cases()["medium"]
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    g = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, r_list)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    assert abs(g["energy"] - o["energy"]) / abs(o["energy"]) < 1e-3
    assert np.sqrt(((g["forces"] - o["forces"]) ** 2).mean()) / rms < 5e-2
    assert tmdlib.device_status() == 0


def test_tile_energies_over_many_tiles_per_block(tmdlib):
    """131,072 atoms (1,024 tcgen05 tiles, several per block): the energy the
    kernels reduce per tile equals the sum of the per-atom energies they write
    (to FP64 rounding), for both kernels of the BF16 form, and the two kernels'
    forces agree as on the small cells."""
    w = I.large(reps=32)
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    m.set_precision("bf16")
    res = {}
    try:
        for kind in ("tcgen05", "mma_sync"):
            tmdlib.set_network_kernel(kind)
            g = _eval(tmdlib, m, s, w.model.rc + 1.0)
            assert abs(g["energy"] - g["e_atom"].sum()) <= 1e-12 * abs(g["energy"]), kind
            res[kind] = g
    finally:
        tmdlib.set_network_kernel("auto")
    assert tmdlib.device_status() == 0
    a, b = res["tcgen05"], res["mma_sync"]
    rms = np.sqrt((b["forces"] ** 2).mean())
    assert np.sqrt(((a["forces"] - b["forces"]) ** 2).mean()) <= 2e-2 * rms
    assert abs(a["energy"] - b["energy"]) <= 1e-4 * abs(b["energy"])
