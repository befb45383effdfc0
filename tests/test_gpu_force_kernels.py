"""The two force passes of the unbatched evaluation: per-pair FP32 FMAs
(SIMT) and the per-atom product [H; H'] P' on TF32 tensor cores with split
operands (Eqs. U_abck, F1_abcx, F2_abcx).  Both are held to the FP32 bars
against the FP64 oracle (|dE| <= 1e-6 |E|, max |dF| <= 1e-5 RMS(F),
max |dW| <= 1e-5 max |W|) on one-species fcc cells with ragged neighbour
counts, and the tensor pass is refused with UNIMPLEMENTED where it does not
apply."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5


def _torch():
    import torch
    return torch


def _fcc(reps, a, sigma, seed):
    rng = np.random.default_rng(seed)
    pos, box = I.lattice("fcc", reps, a)
    return I.System(I.jitter_and_wrap(pos, box, sigma, rng), np.zeros(len(pos), np.int32), box,
                    np.ones(3, np.int32))


def _model(K, widths, s, seed, rc=6.0):
    p = I.random_model(1, K, rc, widths, seed=seed)
    G = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc, want_G=True)["G"]
    rms = np.sqrt((G ** 2).mean(axis=0)).reshape(1, -1)
    return I.random_model(1, K, rc, widths, seed=seed, feature_scale=rms)


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


@pytest.mark.parametrize("K,widths,a,sigma", [(16, [64, 64], 4.05, 0.1), (8, [32, 16], 3.61, 0.15),
                                              (32, [128, 128, 128], 3.61, 0.1), (16, [32], 2.9, 0.2)])
def test_tensor_and_simt_force_passes_match_the_oracle(tmdlib, K, widths, a, sigma, capsys):
    s = _fcc((5, 5, 4), a, sigma, seed=K + int(10 * a))
    p = _model(K, widths, s, seed=K)
    o = O.evaluate(O.OracleModel(p), s.pos, s.types, s.box, s.pbc)
    m = tmdlib.Model(p)
    res = {}
    try:
        for kind in ("simt", "tensor"):
            tmdlib.set_force_kernel(kind)
            res[kind] = _eval(tmdlib, m, s, p.rc + 1.0)
    finally:
        tmdlib.set_force_kernel("auto")
    for kind, g in res.items():
        dE, dF, dW = _errs(g, o)
        with capsys.disabled():
            print(f"\n[K={K} a={a}] {kind}: dE/E={dE:.2e} dF/rms={dF:.2e} dW/max={dW:.2e}")
        assert dE <= E_TOL and dF <= F_TOL and dW <= W_TOL, (kind, dE, dF, dW)


def test_tensor_force_pass_in_the_md_loop(tmdlib):
    """Captured MD steps with the tensor pass follow the SIMT trajectory
    within FP32 rounding over 10 steps (the pair sums differ in rounding
    order only)."""
    s = _fcc((5, 5, 5), 4.05, 0.1, seed=3)
    p = _model(16, [64, 64], s, seed=5)
    vel = I.maxwell_velocities(np.full(s.n, 26.982), 300.0, np.random.default_rng(4))
    out = {}
    try:
        for kind in ("simt", "tensor"):
            tmdlib.set_force_kernel(kind)
            m = tmdlib.Model(p)
            g = tmdlib.System(s.n, s.box, s.pbc, skin=1.0)
            g.set_state(s.pos, vel, s.types, np.full(s.n, 26.982))
            th = g.step(m, 1.0, 10, rebuild_every=5)
            out[kind] = (g.get_state(), th)
    finally:
        tmdlib.set_force_kernel("auto")
    (ps, vs, fs), ths = out["simt"]
    (pt, vt, ft), tht = out["tensor"]
    rms = np.sqrt((fs ** 2).mean())
    assert np.abs(ft - fs).max() <= 1e-4 * rms
    assert np.abs(pt - ps).max() < 1e-7
    assert abs(tht["e_pot"] - ths["e_pot"]) <= 1e-6 * abs(ths["e_pot"])


def test_tensor_force_pass_is_refused_where_it_does_not_apply(tmdlib):
    rng = np.random.default_rng(9)
    pos, box = I.lattice("fcc", (3, 3, 3), 3.61)
    s2 = I.System(I.jitter_and_wrap(pos, box, 0.1, rng), rng.integers(0, 2, len(pos)).astype(np.int32), box,
                  np.ones(3, np.int32))
    s1 = I.System(s2.pos, np.zeros(len(pos), np.int32), box, np.ones(3, np.int32))
    try:
        tmdlib.set_force_kernel("tensor")
        for s, p, table in ((s2, I.random_model(2, 16, 5.0, [16], seed=1), 0),
                            (s1, I.random_model(1, 64, 5.0, [16], seed=2), 0),
                            (s1, I.random_model(1, 16, 5.0, [16], seed=3), 64)):
            m = tmdlib.Model(p)
            if table:
                m.set_radial_table(table)
            with pytest.raises(tmdlib.TmdError) as e:
                _eval(tmdlib, m, s, p.rc)
            assert e.value.status == tmdlib.ERR_UNIMPLEMENTED
        assert tmdlib.lib().tmd_set_force_kernel(3) == tmdlib.ERR_INVALID_ARG
    finally:
        tmdlib.set_force_kernel("auto")
