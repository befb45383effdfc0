"""Radial parameters that differ per species pair.  Gaussian centre and width
of channel k belong to the pair (centre species, neighbour species), the
subscripts a and b of H_abck; with the same parameters for every pair (as in
the other workloads) a layout that swapped the two would go unnoticed.  Here
each of the nine pairs of three species has its own centres and widths, and
the GPU path is held to the FP64 oracle: descriptors element by element,
energy, forces and virial at the FP32 bars, with H evaluated directly and
read from the table built from the same parameters.  The parameters are
asymmetric enough that the swapped layout moves the descriptor by order one
(0.8 and 8 of a column's largest value at K = 8 and 16)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5


def _model(K):
    p = I.random_model(3, K, 5.0, [32, 32], seed=70 + K)
    ti, tj = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    p.mu = p.mu + (0.07 * (3 * ti + tj))[:, :, None]           # centres shifted by up to 0.56 A
    p.eta = p.eta * (1.0 + 0.1 * (2 * ti + tj))[:, :, None]    # widths scaled by up to 1.6
    return p


def _system(seed):
    rng = np.random.default_rng(seed)
    pos, box = I.lattice("fcc", (5, 5, 4), 3.7)   # 400 atoms
    types = rng.integers(0, 3, len(pos)).astype(np.int32)
    return I.System(I.jitter_and_wrap(pos, box, 0.1, rng), types, box, np.ones(3, np.int32))


@pytest.mark.parametrize("K,ppa", [(8, 0), (16, 0), (16, 64)])
def test_pair_dependent_radial_parameters(tmdlib, K, ppa, capsys):
    import torch
    p, s = _model(K), _system(80 + K)
    assert not np.allclose(p.mu, p.mu.transpose(1, 0, 2))
    o = O.evaluate(O.OracleModel(p, radial_table=ppa) if ppa else O.OracleModel(p),
                   s.pos, s.types, s.box, s.pbc, want_G=True)
    m = tmdlib.Model(p)
    if ppa:
        m.set_radial_table(ppa)
    pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
    types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, p.rc)
    G = tmdlib.descriptors(m, nl, pos, types, s.box)
    out = tmdlib.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    G = G.double().cpu().numpy()
    scale = np.maximum(np.abs(o["G"]).max(axis=0), 1e-30)
    dG = float((np.abs(G - o["G"]) / scale).max())
    F = out["forces"].double().cpu().numpy()
    W = out["virial"].cpu().numpy().reshape(3, 3)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    dE = abs(float(out["energy"].item()) - o["energy"]) / abs(o["energy"])
    dF = float(np.abs(F - o["forces"]).max()) / rms
    dW = float(np.abs(W - o["virial"]).max()) / float(np.abs(o["virial"]).max())
    with capsys.disabled():
        print(f"\n[pair radial K={K} ppa={ppa}] dG={dG:.2e} dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}")
    assert dG <= 2e-5
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL
    assert tmdlib.device_status() == 0
