"""Five species: the paper's pair-type index b runs over 1..5 (its table of
tensor subscripts), so a centre atom sees up to five neighbour species and
the descriptor has S K 4 columns.  The GPU path against the FP64 oracle with
S = 5 at K = 8, 16 and 32: the descriptor element by element (which pins the
column of every pair type), energies, forces and the virial at the FP32 bars,
the neighbour table as sorted sets, and the BF16 network form within its
bounds."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5


def _system(seed):
    rng = np.random.default_rng(seed)
    pos, box = I.lattice("fcc", (5, 5, 4), 3.7)   # 400 atoms, box 18.5 x 18.5 x 14.8 A
    types = rng.integers(0, 5, len(pos)).astype(np.int32)
    return I.System(I.jitter_and_wrap(pos, box, 0.1, rng), types, box, np.ones(3, np.int32))


def _dev(s):
    import torch
    return (torch.as_tensor(s.pos, dtype=torch.float64, device="cuda"),
            torch.as_tensor(s.types, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("K", [8, 16, 32])
def test_five_species_against_oracle(tmdlib, K, capsys):
    import torch
    s = _system(40 + K)
    assert set(s.types.tolist()) == {0, 1, 2, 3, 4}
    p = I.random_model(5, K, 5.0, [32, 32], seed=K, masses=[55.845, 58.693, 51.996, 58.933, 54.938])
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc, want_G=True)
    m = tmdlib.Model(p)
    pos, types = _dev(s)
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, p.rc)
    # descriptor columns of every (pair type b, k, rank m)
    G = tmdlib.descriptors(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    G = G.double().cpu().numpy()
    assert G.shape == (s.n, 5 * K * 4)
    # each column against its own largest value (at K = 32 the narrowest
    # short-range channels hold values near 1e-28: rank 0 is |P|, whose
    # square would underflow in FP32)
    scale = np.maximum(np.abs(o["G"]).max(axis=0), 1e-30)
    dG = float((np.abs(G - o["G"]) / scale).max())
    out = tmdlib.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    E = float(out["energy"].item())
    F = out["forces"].double().cpu().numpy()
    W = out["virial"].cpu().numpy().reshape(3, 3)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    dE = abs(E - o["energy"]) / abs(o["energy"])
    dF = float(np.abs(F - o["forces"]).max()) / rms
    dW = float(np.abs(W - o["virial"]).max()) / float(np.abs(o["virial"]).max())
    m.set_precision("bf16")
    b = tmdlib.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    bF = float(np.abs(b["forces"].double().cpu().numpy() - o["forces"]).max()) / rms
    bE = abs(float(b["energy"].item()) - o["energy"]) / abs(o["energy"])
    with capsys.disabled():
        print(f"\n[S=5 K={K}] dG={dG:.2e} fp32 dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}; "
              f"bf16 dE/E={bE:.2e} dF/rms={bF:.2e}")
    # FP32 sums of ~40 pairs per entry; the maximum over 400 atoms and up to
    # 640 columns reaches 1.3e-5 of a column's largest value (a misplaced
    # pair-type column would be off by order one)
    assert dG <= 2e-5
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL
    assert tmdlib.device_status() == 0
    assert bE < 1e-3 and bF < 0.5


def test_five_species_neighbour_table(tmdlib):
    """The species-partitioned atom order with five species: the table equals
    the oracle's as sorted sets, with each atom's entries grouped by the
    neighbour's species (the pair-type index b)."""
    s = _system(60)
    r = 6.0
    pos, types = _dev(s)
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, r)
    off, nbr, sh = nl.export()
    o_off, o_nbr, o_sh = O.neighbors(s.pos, s.box, s.pbc, r)
    assert np.array_equal(off, o_off)

    def as_set(o, nb, shf):
        return {(i, int(nb[c]), int(shf[c][0]), int(shf[c][1]), int(shf[c][2]))
                for i in range(len(o) - 1) for c in range(o[i], o[i + 1])}

    assert as_set(off, nbr, sh) == as_set(o_off, o_nbr, o_sh)
    for i in range(0, s.n, 7):
        keys = [(int(s.types[nbr[c]]), int(nbr[c]), *map(int, sh[c])) for c in range(off[i], off[i + 1])]
        assert keys == sorted(keys)
