"""GPU path (through the C ABI) against the FP64 oracle.

Bars (stated for FP32 arithmetic of the GPU path):
  neighbour table   bit-exact as sets of (i, j, shift)
  total energy      |dE| <= 1e-6 |E|
  forces            max |dF| <= 1e-5 RMS(F)
  virial            max |dW| <= 1e-5 max |W|
  atomic energies   max |dE_a| <= 1e-5 max |E_a|
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL, EA_TOL = 1e-6, 1e-5, 1e-5, 1e-5


def _torch():
    import torch
    return torch


def _dev(a, dtype):
    torch = _torch()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_nlist(tmd, system, r_list):
    torch = _torch()
    nl = tmd.NeighborList()
    pos = _dev(system.pos, torch.float64)
    types = _dev(system.types, torch.int32)
    nl.build(pos, types, system.box, system.pbc, r_list)
    return nl, pos, types


def gpu_eval(tmd, model, system, r_list=None, precision="fp32"):
    torch = _torch()
    m = tmd.Model(model, precision=precision)
    nl, pos, types = gpu_nlist(tmd, system, model.rc if r_list is None else r_list)
    out = tmd.evaluate(m, nl, pos, types, system.box)
    torch.cuda.synchronize()
    return {"energy": float(out["energy"].item()), "e_atom": out["e_atom"].double().cpu().numpy(),
            "forces": out["forces"].double().cpu().numpy(), "virial": out["virial"].cpu().numpy().reshape(3, 3)}


def as_set(nl):
    off, nbr, sh = nl
    out = set()
    for i in range(len(off) - 1):
        for c in range(off[i], off[i + 1]):
            out.add((i, int(nbr[c]), int(sh[c][0]), int(sh[c][1]), int(sh[c][2])))
    return out


def assert_parity(g, o, label=""):
    F = o["forces"]
    rms = float(np.sqrt((F ** 2).mean())) if F.size else 0.0
    dE = abs(g["energy"] - o["energy"])
    dF = float(np.abs(g["forces"] - F).max()) if F.size else 0.0
    dW = float(np.abs(g["virial"] - o["virial"]).max())
    dEa = float(np.abs(g["e_atom"] - o["e_atom"]).max()) if F.size else 0.0
    msg = f"{label}: dE/E={dE / max(abs(o['energy']), 1e-300):.2e} dF/rms={dF / max(rms, 1e-300):.2e} " \
          f"dW/max={dW / max(np.abs(o['virial']).max(), 1e-300):.2e}"
    assert dE <= E_TOL * abs(o["energy"]), msg
    assert dF <= F_TOL * rms, msg
    assert dW <= W_TOL * np.abs(o["virial"]).max(), msg
    assert dEa <= EA_TOL * np.abs(o["e_atom"]).max(), msg
    return msg


# ------------------------------------------------------------------ neighbour table
@pytest.mark.parametrize("case", ["tiny", "tiny_skin", "selfimage", "open", "mixed", "medium", "dense", "wide"])
def test_neighbor_table_bit_exact(tmdlib, case):
    rng = np.random.default_rng(11)
    if case in ("tiny", "tiny_skin"):
        s = I.tiny().systems[0]
        r = 5.0 if case == "tiny" else 6.0
    elif case == "selfimage":
        pos, box = I.lattice("bcc", (2, 2, 2), 2.9)
        s = I.System(I.jitter_and_wrap(pos, box, 0.1, rng), np.zeros(len(pos), np.int32), box, np.ones(3, np.int32))
        r = 7.0
    elif case == "open":
        s = I.cluster(60, 6.0, seed=3, n_species=2)
        r = 4.5
    elif case == "mixed":
        pos, box = I.lattice("fcc", (3, 3, 3), 3.61)
        box = box.copy(); box[2] += 8.0
        s = I.System(I.jitter_and_wrap(pos, box, 0.05, rng), rng.integers(0, 3, len(pos)).astype(np.int32),
                     box, np.array([1, 1, 0], np.int32))
        r = 6.0
    elif case == "dense":
        # stencils of > 1,920 candidates: the cell-cooperative pass hands these
        # atoms to the per-atom pass
        pos, box = I.lattice("fcc", (9, 9, 9), 2.9)
        s = I.System(I.jitter_and_wrap(pos, box, 0.05, rng), np.zeros(len(pos), np.int32), box, np.ones(3, np.int32))
        r = 8.5
    elif case == "wide":
        # a 2.9 A box with a 7 A list radius: stencils of 7^3 cells (images up
        # to 3 boxes away) go to the per-atom pass as well
        pos, box = I.lattice("bcc", (1, 1, 1), 2.9)
        s = I.System(I.jitter_and_wrap(pos, box, 0.05, rng), np.zeros(len(pos), np.int32), box, np.ones(3, np.int32))
        r = 7.0
    else:
        s = I.medium().systems[0]
        r = 7.0
    nl, _, _ = gpu_nlist(tmdlib, s, r)
    g = nl.export()
    o = O.neighbors(s.pos, s.box, s.pbc, r)
    assert np.array_equal(g[0], o[0])
    assert as_set(g) == as_set(o)
    # per-atom order: (species of j, j, sx, sy, sz)
    off, nbr, sh = g
    for i in range(0, len(off) - 1, max(1, (len(off) - 1) // 64)):
        keys = [(int(s.types[nbr[c]]), int(nbr[c]), *map(int, sh[c])) for c in range(off[i], off[i + 1])]
        assert keys == sorted(keys)


def test_neighbor_table_rounding_band(tmdlib):
    """Pairs placed within 1e-12 A of r_list are decided exactly as the FP64 definition."""
    box = np.array([30.0, 30.0, 30.0])
    r = 5.0
    base = np.array([10.0, 10.0, 10.0])
    pts = [base]
    rng = np.random.default_rng(5)
    for k in range(40):
        u = rng.normal(size=3); u /= np.linalg.norm(u)
        eps = (k - 20) * 3e-13
        pts.append(base + u * (r + eps))
    s = I.System(np.array(pts), np.zeros(len(pts), np.int32), box, np.zeros(3, np.int32))
    nl, _, _ = gpu_nlist(tmdlib, s, r)
    assert as_set(nl.export()) == as_set(O.neighbors(s.pos, s.box, s.pbc, r))


def test_neighbor_errors(tmdlib):
    torch = _torch()
    s = I.tiny().systems[0]
    bad = s.pos.copy(); bad[3, 1] = s.box[1] + 0.5
    nl = tmdlib.NeighborList()
    with pytest.raises(tmdlib.TmdError) as e:
        nl.build(_dev(bad, torch.float64), _dev(s.types, torch.int32), s.box, s.pbc, 5.0)
    assert e.value.status == tmdlib.ERR_INVALID_ARG
    # degree beyond TMD_MAX_DEGREE: dense random gas, large radius
    rng = np.random.default_rng(0)
    box = np.array([12.0, 12.0, 12.0])
    pos = rng.uniform(0, 12.0, size=(3000, 3))
    with pytest.raises(tmdlib.TmdError) as e:
        nl.build(_dev(pos, torch.float64), _dev(np.zeros(3000, np.int32), torch.int32), box, [1, 1, 1], 6.0)
    assert e.value.status == tmdlib.ERR_CAPACITY
    # the table is still usable after an error
    nl.build(_dev(s.pos, torch.float64), _dev(s.types, torch.int32), s.box, s.pbc, 5.0)
    assert nl.size() == (32, 1364)


# ------------------------------------------------------------------ energy / forces / virial
def test_tiny_parity(tmdlib):
    w = I.tiny()
    s = w.systems[0]
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, w.model, s)
    print(assert_parity(g, o, "tiny"))


def test_tiny_parity_with_skin_list(tmdlib):
    """Entries between rc and r_list are skipped."""
    w = I.tiny()
    s = w.systems[0]
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, w.model, s, r_list=6.3)
    assert_parity(g, o, "tiny skin")


def test_medium_parity(tmdlib):
    w = I.medium()
    s = w.systems[0]
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, w.model, s, r_list=7.0)
    print(assert_parity(g, o, "medium"))


@pytest.mark.parametrize("K,S,widths,act", [(8, 3, [12, 8], "tanh"), (16, 4, [8, 8, 8], "squareplus"),
                                            (32, 2, [16], "tanh"), (32, 3, [8, 12, 4, 8], "tanh")])
def test_model_shapes_parity(tmdlib, K, S, widths, act):
    """Every (K, S) kernel instance and network depth, on a ragged multi-species cell."""
    rng = np.random.default_rng(K * 10 + S)
    pos, box = I.lattice("bcc", (4, 4, 3), 3.1)
    s = I.System(I.jitter_and_wrap(pos, box, 0.12, rng), rng.integers(0, S, len(pos)).astype(np.int32),
                 box, np.ones(3, np.int32))
    om = O.OracleModel(I.random_model(S, K, 5.5, widths, seed=K + S, activation=act))
    o = O.evaluate(om, s.pos, s.types, s.box, s.pbc, want_G=True)
    rms = np.sqrt((o["G"] ** 2).mean(axis=0)).reshape(1, -1)
    p = I.random_model(S, K, 5.5, widths, seed=K + S, activation=act,
                       feature_scale=np.repeat(np.maximum(rms, 1e-2), S, axis=0))
    om = O.OracleModel(p)
    o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, p, s)
    assert_parity(g, o, f"K{K} S{S}")


def test_small_box_self_images(tmdlib):
    rng = np.random.default_rng(2)
    pos, box = I.lattice("hcp", (2, 1, 1), 3.0)
    s = I.System(I.jitter_and_wrap(pos, box, 0.1, rng), rng.integers(0, 2, len(pos)).astype(np.int32), box,
                 np.ones(3, np.int32))
    w = I.medium()
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, w.model, s)
    assert_parity(g, o, "self images")


def test_degenerate_systems(tmdlib):
    w = I.medium()
    om = O.OracleModel(w.model)
    box = np.array([20.0, 20.0, 20.0])
    pbc = np.zeros(3, np.int32)
    # one isolated atom: G = 0, E = NNP(0), F = 0
    s = I.System(np.array([[5.0, 5.0, 5.0]]), np.array([1], np.int32), box, pbc)
    g = gpu_eval(tmdlib, w.model, s)
    o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
    assert abs(g["energy"] - o["energy"]) <= 1e-6 * abs(o["energy"])
    assert np.all(g["forces"] == 0.0)
    # two atoms (all descriptor ranks equal h^2), and a pair exactly beyond rc
    for d in (2.4, 6.0 + 1e-3):
        s = I.System(np.array([[5.0, 5.0, 5.0], [5.0 + d, 5.0, 5.0]]), np.array([0, 1], np.int32), box, pbc)
        g = gpu_eval(tmdlib, w.model, s)
        o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
        assert abs(g["energy"] - o["energy"]) <= 1e-6 * abs(o["energy"])
        assert np.abs(g["forces"] - o["forces"]).max() <= 1e-5 * max(np.abs(o["forces"]).max(), 1e-3)
    # empty system
    torch = _torch()
    m = tmdlib.Model(w.model)
    nl = tmdlib.NeighborList()
    e = torch.ones(1, dtype=torch.float64, device="cuda")
    vir = torch.ones(9, dtype=torch.float64, device="cuda")
    p0 = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    t0 = torch.zeros(0, dtype=torch.int32, device="cuda")
    nl.build(p0, t0, box, pbc, 6.0)
    tmdlib.compute(m, nl, p0, t0, box, energy=e, virial=vir)
    torch.cuda.synchronize()
    assert e.item() == 0.0 and vir.abs().max().item() == 0.0


def test_sparse_gas_atoms_without_in_cutoff_pairs(tmdlib):
    """A dilute periodic gas with the table built at rc + skin: atoms whose
    entries all lie in the skin shell reach the descriptor and force passes
    with no in-cutoff pair (the force pass then merges the next atoms' pairs
    into its batches); parity with the oracle, alone and batched."""
    w = I.medium()
    s = I.sparse_gas()
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    off, nbr, sh = O.neighbors(s.pos, s.box, s.pbc, w.model.rc)
    counts = np.diff(off)
    assert (counts == 0).sum() >= 20      # the case this test is about
    g = gpu_eval(tmdlib, w.model, s, r_list=w.model.rc + 1.0)
    assert_parity(g, o, "sparse gas")
    # batched with the medium cell (resident tables with a skin)
    b = tmdlib.Batch([s, w.systems[0]], skin=1.0)
    m = tmdlib.Model(w.model)
    E, W = b.compute(m, [0, 1])
    _, _, fb = b.get_system(0)
    bo = {"energy": float(E[0]), "forces": fb.astype(np.float64), "virial": W[0], "e_atom": o["e_atom"]}
    assert_parity(bo, o, "sparse gas, batched")


def test_compute_argument_errors(tmdlib):
    torch = _torch()
    w = I.medium()
    m = tmdlib.Model(w.model)
    s = I.tiny().systems[0]
    nl, pos, types = gpu_nlist(tmdlib, s, 4.0)
    with pytest.raises(tmdlib.TmdError) as e:  # list radius below the model cutoff
        tmdlib.evaluate(m, nl, pos, types, s.box)
    assert e.value.status == tmdlib.ERR_INVALID_ARG
    nl.build(pos, types, s.box, s.pbc, 6.5)
    with pytest.raises(tmdlib.TmdError):   # n differs from the table
        tmdlib.evaluate(m, nl, pos[:10], types[:10], s.box)
    bad = _dev(np.full(32, 3, np.int32), torch.int32)   # species beyond the model's 2
    nl.build(pos, bad, s.box, s.pbc, 6.5)
    with pytest.raises(tmdlib.TmdError):
        tmdlib.evaluate(m, nl, pos, bad, s.box)


def test_deterministic_reruns(tmdlib):
    """Energy and virial are reduced in a fixed order and forces accumulate in
    integer fixed point: every output is bitwise repeatable."""
    w = I.medium()
    s = w.systems[0]
    a = gpu_eval(tmdlib, w.model, s, r_list=7.0)
    b = gpu_eval(tmdlib, w.model, s, r_list=7.0)
    assert a["energy"] == b["energy"]
    assert np.array_equal(a["virial"], b["virial"])
    assert np.array_equal(a["e_atom"], b["e_atom"])
    assert np.array_equal(a["forces"], b["forces"])


# ------------------------------------------------------------------ full size (sampled)
def test_large_full_size_sampled(tmdlib):
    """The 1,048,576-atom cell in the benchmark's launch configuration: sampled
    atoms against the oracle's one-atom-at-a-time evaluation, plus sum F = 0
    and E = sum E_a at full size."""
    w = I.large()
    s = w.systems[0]
    g = gpu_eval(tmdlib, w.model, s, r_list=7.0)
    om = O.OracleModel(w.model)
    rng = np.random.default_rng(1)
    atoms = rng.choice(s.n, size=32, replace=False)
    ea, fa = O.sampled(om, s.pos, s.types, s.box, s.pbc, atoms)
    rms = np.sqrt((g["forces"] ** 2).mean())
    assert np.abs(g["forces"][atoms] - fa).max() <= F_TOL * rms
    assert np.abs(g["e_atom"][atoms] - ea).max() <= EA_TOL * np.abs(ea).max()
    assert abs(g["energy"] - g["e_atom"].sum()) <= 1e-6 * abs(g["energy"])
    # the int64 scatter sums to zero exactly; what is left is the FP32
    # rounding of each reported force (~sqrt(N) ulp(|F|) ~ 4e-5 RMS here)
    assert np.abs(g["forces"].sum(axis=0)).max() <= 1e-2 * rms


# ------------------------------------------------------------------ MD
def test_md_matches_oracle_trajectory_tiny(tmdlib):
    """20 velocity-Verlet steps: GPU trajectory vs the oracle's (short enough
    that the FP32 force error cannot grow chaotically)."""
    w = I.tiny()
    s = w.systems[0]
    s.vel = I.maxwell_velocities(s.masses, 300.0, np.random.default_rng(3))
    om = O.OracleModel(w.model)
    po, vo, _ = O.md(om, s, 20, 1.0)
    sysg = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    sysg.set_state(s.pos, s.vel, s.types, s.masses)
    m = tmdlib.Model(w.model)
    th = sysg.step(m, 1.0, 20, rebuild_every=0)
    pg, vg, _ = sysg.get_state()
    d = pg - po
    d -= np.rint(d / s.box) * s.box
    assert np.abs(d).max() < 1e-6
    assert np.abs(vg - vo).max() < 1e-6
    assert th["step"] == 20 and th["rebuilds"] >= 1


def test_md_medium_100_steps(tmdlib):
    """Medium cell, 100 steps with 1 A skin: forces at the GPU's own positions
    match the oracle at steps 50 and 100; NVE energy is conserved."""
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    om = O.OracleModel(w.model)
    sysg = tmdlib.System(s.n, s.box, s.pbc, skin=1.0)
    sysg.set_state(s.pos, s.vel, s.types, s.masses)
    th0 = sysg.step(m, 1.0, 0)
    e0 = th0["e_pot"] + th0["e_kin"]
    for seg in range(2):
        th = sysg.step(m, 1.0, 50)
        pg, vg, fg = sysg.get_state()
        o = O.evaluate(om, pg, s.types, s.box, s.pbc)
        rms = np.sqrt((o["forces"] ** 2).mean())
        assert np.abs(fg - o["forces"]).max() <= F_TOL * rms
        assert abs(th["e_pot"] - o["energy"]) <= E_TOL * abs(o["energy"])
    e1 = th["e_pot"] + th["e_kin"]
    assert th["step"] == 100
    assert abs(e1 - e0) / s.n < 1e-4, (e0, e1)
    assert 1 <= th["rebuilds"] <= 100


def test_step_host_matches_device_path(tmdlib):
    w = I.tiny()
    s = w.systems[0]
    s.vel = I.maxwell_velocities(s.masses, 300.0, np.random.default_rng(4))
    m = tmdlib.Model(w.model)
    a = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    a.set_state(s.pos, s.vel, s.types, s.masses)
    a.step(m, 1.0, 5, rebuild_every=1)
    pa, va, fa = a.get_state()
    b = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    b.set_state(s.pos, s.vel, s.types, s.masses)
    pos, vel = s.pos.copy(), s.vel.copy()
    forces = np.zeros((s.n, 3), np.float32)
    b.step_host(m, pos, vel, None, 1.0, 1, rebuild_every=1)
    # continue from host state, passing the resident forces back in
    _, _, forces = b.get_state()
    b.step_host(m, pos, vel, forces, 1.0, 4, rebuild_every=1)
    # same arithmetic in both paths (forces are accumulated in fixed point)
    assert np.abs(pos - pa).max() < 1e-12 and np.abs(vel - va).max() < 1e-12


def test_step_host_keeps_the_rebuild_cadence(tmdlib):
    """One step per host call with the table rebuilt every 5 steps follows the
    device loop exactly, and positions the caller moves by a whole period
    still give the same forces (the skin check rebuilds the table)."""
    w = I.tiny()
    s = w.systems[0]
    s.vel = I.maxwell_velocities(s.masses, 300.0, np.random.default_rng(8))
    m = tmdlib.Model(w.model)
    a = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    a.set_state(s.pos, s.vel, s.types, s.masses)
    tha = a.step(m, 1.0, 11, rebuild_every=5)
    pa, va, fa = a.get_state()
    b = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    b.set_state(s.pos, s.vel, s.types, s.masses)
    pos, vel = s.pos.copy(), s.vel.copy()
    forces = np.zeros((s.n, 3), np.float32)
    b.step_host(m, pos, vel, None, 1.0, 1, rebuild_every=5)
    _, _, forces = b.get_state()
    for _ in range(10):
        b.step_host(m, pos, vel, forces, 1.0, 1, rebuild_every=5)
    thb = b.step(m, 0.0, 0, rebuild_every=5)
    assert np.array_equal(pos, pa) and np.array_equal(vel, va) and np.array_equal(forces, fa)
    assert thb["rebuilds"] == tha["rebuilds"]
    # the caller moves one atom by a whole box length: same physics; the skin
    # check sees the jump and rebuilds the table
    pos2, vel2, f2 = pos.copy(), vel.copy(), forces.copy()
    pos2[0, 0] += s.box[0]
    b.step_host(m, pos2, vel2, f2, 1.0, 1, rebuild_every=0)
    c = tmdlib.System(s.n, s.box, s.pbc, skin=0.5)
    c.set_state(np.mod(pos, s.box), vel, s.types, s.masses)
    c_pos, c_vel, c_f = np.mod(pos, s.box), vel.copy(), forces.copy()
    c.step_host(m, c_pos, c_vel, c_f, 1.0, 1, rebuild_every=0)
    d = np.mod(pos2 - c_pos + 0.5 * s.box, s.box) - 0.5 * s.box
    assert np.abs(d).max() < 1e-12
    assert np.abs(f2 - c_f).max() <= 1e-6 * max(1.0, np.abs(c_f).max())


def test_evaluate_host_matches_device(tmdlib):
    w = I.medium()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    nl = tmdlib.NeighborList()
    e = np.zeros(1)
    f = np.zeros((s.n, 3), np.float32)
    vir = np.zeros(9)
    tmdlib.evaluate_host(m, nl, s.pos, s.types, s.box, s.pbc, e, f, vir)
    g = gpu_eval(tmdlib, w.model, s, r_list=6.0)
    assert e[0] == g["energy"]
    assert np.abs(f - g["forces"]).max() <= 1e-6 * np.abs(g["forces"]).max()


@pytest.mark.parametrize("wname", ["tiny", "medium"])
def test_descriptor_matrix_elementwise(tmdlib, wname):
    """G_abkm element by element (Eq. tensor_formalism) against the oracle:
    |dG| <= 1e-5 of the column's largest magnitude."""
    torch = _torch()
    w = getattr(I, wname)()
    s = w.systems[0]
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc, want_G=True)["G"]
    m = tmdlib.Model(w.model)
    nl, pos, types = gpu_nlist(tmdlib, s, w.model.rc + (0.0 if wname == "tiny" else 1.0))
    G = tmdlib.descriptors(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    G = G.double().cpu().numpy()
    scale = np.maximum(np.abs(o).max(axis=0), 1e-30)
    err = (np.abs(G - o) / scale).max()
    assert err <= 1e-5, err


# ------------------------------------------------------------------ BF16 network form
@pytest.mark.parametrize("wname", ["tiny", "medium"])
def test_bf16_network_form_errors(tmdlib, wname, capsys):
    """BF16 tensor-core network (radial basis, moments and contractions FP32):
    errors against the FP64 oracle are reported; the bounds only catch gross
    mistakes (BF16 has an 8-bit significand)."""
    w = getattr(I, wname)()
    s = w.systems[0]
    o = O.evaluate(O.OracleModel(w.model), s.pos, s.types, s.box, s.pbc)
    g = gpu_eval(tmdlib, w.model, s, precision="bf16")
    f32 = gpu_eval(tmdlib, w.model, s, precision="fp32")
    rms = np.sqrt((o["forces"] ** 2).mean())
    dE = abs(g["energy"] - o["energy"]) / abs(o["energy"])
    dF = np.abs(g["forces"] - o["forces"]).max() / rms
    dFr = np.sqrt(((g["forces"] - o["forces"]) ** 2).mean()) / rms
    dEa = np.abs(g["e_atom"] - o["e_atom"]).max()
    with capsys.disabled():
        print(f"\n[bf16 {wname}] dE/E={dE:.2e} max|dF|/rms={dF:.2e} rms(dF)/rms={dFr:.2e} max|dEa|={dEa:.2e} eV "
              f"(fp32: dF/rms={np.abs(f32['forces'] - o['forces']).max() / rms:.2e})")
    assert dE < 1e-3 and dFr < 5e-2 and dF < 0.5
    # the forms differ only in the network
    assert np.abs(g["forces"] - f32["forces"]).max() > 0.0


def test_bf16_rejects_widths_not_multiple_of_16(tmdlib):
    p = I.random_model(1, 8, 4.0, [12, 8], seed=3)
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.Model(p, precision="bf16")
    assert e.value.status == tmdlib.ERR_UNIMPLEMENTED
    m = tmdlib.Model(p)   # FP32 accepts them
    with pytest.raises(tmdlib.TmdError):
        m.set_precision("bf16")
