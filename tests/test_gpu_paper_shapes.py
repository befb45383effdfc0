"""The paper's potential geometries (Sec. "The Potential", Table pot_mae): the
k = 32 model (32 radial channels, network 128-128-128-1) and the k = 128 model
(128 channels, network 128-128-128-128-1), both with SquarePlus activations,
on random weights, on bcc W lattices at the two lattice constants of the
paper's weak-scaling runs (3.1887 A, about 0 GPa, and 2.8 A, about 270 GPa).
K = 64 and K = 128 run the descriptor pass in chunks of 32 channels.

FP32 bars as everywhere (|dE| <= 1e-6 |E|, max |dF| <= 1e-5 RMS(F),
max |dW| <= 1e-5 max |W|); the BF16 network form reports its errors and is
bounded loosely.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5
W_MASS = 183.84


def _torch():
    import torch
    return torch


def _bcc_w(a, reps, seed):
    rng = np.random.default_rng(seed)
    pos, box = I.lattice("bcc", reps, a)
    return I.System(I.jitter_and_wrap(pos, box, 0.1, rng), np.zeros(len(pos), np.int32), box,
                    np.ones(3, np.int32))


def _scaled_model(K, S, widths, system, seed, rc=6.0):
    """Random model whose first layer is normalised by the descriptor RMS of
    this configuration (the way the workloads' models are built)."""
    p = I.random_model(S, K, rc, widths, seed=seed, activation="squareplus", masses=[W_MASS] * S)
    G = O.evaluate(O.OracleModel(p), system.pos, system.types, system.box, system.pbc, want_G=True)["G"]
    rms = np.sqrt((G ** 2).mean(axis=0)).reshape(1, -1)
    return I.random_model(S, K, rc, widths, seed=seed, activation="squareplus", masses=[W_MASS] * S,
                          feature_scale=np.repeat(rms, S, axis=0))


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


@pytest.mark.parametrize("k,widths", [(32, [128, 128, 128]), (128, [128, 128, 128, 128])])
@pytest.mark.parametrize("a", [3.1887, 2.8])
def test_paper_potential_shapes(tmdlib, k, widths, a, capsys):
    s = _bcc_w(a, (4, 4, 4), seed=int(a * 1000) + k)
    p = _scaled_model(k, 1, widths, s, seed=k)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    m = tmdlib.Model(p)
    g = _eval(tmdlib, m, s, p.rc + 1.0)
    dE, dF, dW = _errs(g, o)
    m.set_precision("bf16")
    b = _eval(tmdlib, m, s, p.rc + 1.0)
    bE, bF, bW = _errs(b, o)
    with capsys.disabled():
        print(f"\n[k={k} a={a}] fp32 dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}; "
              f"bf16 dE/E={bE:.2e} dF/rms={bF:.2e} dW/max={bW:.2e}")
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL
    assert bE < 1e-3 and bF < 0.5


def test_k128_bf16_both_network_kernels(tmdlib):
    """The k = 128 network (Dd 512) in the BF16 form on both kernels: tcgen05
    (N passes of 256 for G') and mma.sync (narrow weight chunks, gradient
    buffers sharing the G tile)."""
    s = _bcc_w(3.1887, (3, 3, 3), seed=9)
    p = _scaled_model(128, 1, [128, 128, 128, 128], s, seed=128)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    res = {}
    try:
        for kind in ("tcgen05", "mma_sync"):
            tmdlib.set_network_kernel(kind)
            res[kind] = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, p.rc)
    finally:
        tmdlib.set_network_kernel("auto")
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    for kind, g in res.items():
        bE, bF, _ = _errs(g, o)
        assert bE < 1e-3 and bF < 0.5, (kind, bE, bF)
    cross = np.sqrt(((res["tcgen05"]["forces"] - res["mma_sync"]["forces"]) ** 2).mean()) / rms
    assert cross < 2e-2
    assert tmdlib.device_status() == 0


def test_k64_two_species(tmdlib):
    rng = np.random.default_rng(64)
    pos, box = I.lattice("bcc", (4, 4, 3), 3.1)
    s = I.System(I.jitter_and_wrap(pos, box, 0.12, rng), rng.integers(0, 2, len(pos)).astype(np.int32), box,
                 np.ones(3, np.int32))
    p = _scaled_model(64, 2, [32, 16], s, seed=65, rc=5.5)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    g = _eval(tmdlib, tmdlib.Model(p), s, p.rc)
    dE, dF, dW = _errs(g, o)
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (dE, dF, dW)
    # BF16 form: Dd 512 with two species (G' in two N passes, tiles spanning species)
    b = _eval(tmdlib, tmdlib.Model(p, precision="bf16"), s, p.rc)
    bE, bF, _ = _errs(b, o)
    rms = float(np.sqrt((o["forces"] ** 2).mean()))
    assert bE < 1e-3 and np.sqrt(((b["forces"] - o["forces"]) ** 2).mean()) / rms < 5e-2, (bE, bF)
    assert tmdlib.device_status() == 0


def test_k128_with_radial_table_and_batch(tmdlib):
    """The chunked descriptor pass with a tabulated radial basis, and the
    batched path, on the k = 128 geometry."""
    s = _bcc_w(3.1887, (3, 3, 3), seed=7)
    p = _scaled_model(128, 1, [128, 128, 128, 128], s, seed=128)
    m = tmdlib.Model(p)
    m.set_radial_table(256)
    g = _eval(tmdlib, m, s, p.rc)
    o = O.evaluate(O.OracleModel(p, radial_table=256), s.pos, s.types, s.box, s.pbc)
    dE, dF, dW = _errs(g, o)
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (dE, dF, dW)
    m.set_radial_table(0)
    s2 = _bcc_w(2.8, (3, 3, 4), seed=8)
    b = tmdlib.Batch([s, s2])
    E, W = b.compute(m, [0, 1])
    for k, x in enumerate((s, s2)):
        o = O.evaluate(O.OracleModel(p), x.pos, x.types, x.box, x.pbc)
        _, _, f = b.get_system(k)
        rms = np.sqrt((o["forces"] ** 2).mean())
        assert abs(E[k] - o["energy"]) <= E_TOL * abs(o["energy"]), k
        assert np.abs(f - o["forces"]).max() <= F_TOL * rms, k
        assert np.abs(W[k] - o["virial"]).max() <= W_TOL * np.abs(o["virial"]).max(), k


def test_unsupported_shapes_are_rejected(tmdlib):
    for S, K, widths in [(2, 128, [16]), (3, 64, [16]), (1, 256, [16]), (1, 24, [16])]:
        with pytest.raises(tmdlib.TmdError) as e:
            tmdlib.Model(I.random_model(S, K, 5.0, widths, seed=1))
        assert e.value.status == tmdlib.ERR_UNIMPLEMENTED, (S, K)
    # activations of a 32-atom tile beyond the shared memory of an SM (two
    # species: every activation buffer of its own)
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.Model(I.random_model(2, 64, 5.0, [256, 256, 256, 256], seed=1))
    assert e.value.status == tmdlib.ERR_UNIMPLEMENTED


def test_wide_network_with_shared_input_buffer(tmdlib):
    """A one-species k = 128 model with four 256-wide layers: its FP32
    network tile fits on chip only because the second hidden layer reuses the
    input activations' buffer."""
    s = _bcc_w(3.1887, (3, 3, 3), seed=256)
    p = _scaled_model(128, 1, [256, 256, 256, 256], s, seed=256)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    g = _eval(tmdlib, tmdlib.Model(p), s, p.rc)
    dE, dF, dW = _errs(g, o)
    assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (dE, dF, dW)


def test_wide_network_bf16_is_supported_or_rejected_cleanly(tmdlib):
    """Switching the wide k = 128 model to the BF16 network either works on
    one of the two kernels (loose BF16 bars) or is refused with
    UNIMPLEMENTED; a refusal leaves the FP32 model usable."""
    s = _bcc_w(3.1887, (3, 3, 3), seed=257)
    p = _scaled_model(128, 1, [256, 256, 256, 256], s, seed=257)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    m = tmdlib.Model(p)
    try:
        m.set_precision("bf16")
    except tmdlib.TmdError as e:
        assert e.status == tmdlib.ERR_UNIMPLEMENTED
        g = _eval(tmdlib, m, s, p.rc)
        dE, dF, dW = _errs(g, o)
        assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (dE, dF, dW)
        return
    b = _eval(tmdlib, m, s, p.rc)
    bE, bF, _ = _errs(b, o)
    assert bE < 1e-3 and bF < 0.5, (bE, bF)
    assert tmdlib.device_status() == 0
