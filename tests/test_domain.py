"""Spatial domain decomposition of one system (the paper's MPI scheme,
Sec. "Evaluation"): slabs, ghost halo, owner-computes evaluation, reverse
exchange of ghost forces, FP64 all-reduce of energy and virial.

On the CPU the per-rank force call is the FP64 oracle restricted to the owned
centres (ghosts keep empty table rows), so the decomposed totals must equal
the single-box oracle to rounding; the exchanges run in one process and over
2 and 4 gloo ranks.  On the GPU the per-rank call is tmd_compute_owned and
the decomposed forces must equal tmd_compute on the whole box within the
FP32 bars."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2310_08439_gb300 import domain as D
from paper_2310_08439_gb300 import inputs as I

RC = 4.5


def _system():
    pos, box = I.lattice("fcc", (8, 3, 3), 3.61)
    rng = np.random.default_rng(41)
    pos = I.jitter_and_wrap(pos, box, 0.08, rng)
    types = rng.integers(0, 2, size=pos.shape[0]).astype(np.int32)
    vel = rng.normal(0.0, 0.01, size=pos.shape)
    mass = np.where(types == 0, 55.845, 63.546)
    p = I.random_model(2, 6, RC, [10, 8], seed=9)
    return pos, box, np.ones(3, dtype=np.int32), types, vel, mass, p


def oracle_engine(om, rc):
    def engine(pos, types, n_owned, box, pbc):
        off, nbr, sh = O.neighbors(pos, box, pbc, rc)
        cut = int(off[n_owned])
        off2 = off.copy()
        off2[n_owned + 1:] = cut            # ghosts are neighbours only
        out = O.compute(om, pos, types, box, (off2, nbr[:cut], sh[:cut]))
        return float(out["e_atom"][:n_owned].sum()), out["forces"], out["virial"]
    return engine


def _gather(slabs, domains, forces, n):
    F = np.zeros((n, 3))
    seen = np.zeros(n, dtype=int)
    for d, f in zip(domains, forces):
        F[d.gid] = f
        seen[d.gid] += 1
    assert np.all(seen == 1)
    return F


@pytest.mark.parametrize("R", [1, 2, 4])
def test_serial_decomposition_equals_single_box(R):
    pos, box, pbc, types, vel, mass, p = _system()
    om = O.OracleModel(p)
    ref = O.evaluate(om, pos, types, box, pbc)
    slabs = D.Slabs(box, pbc, R, RC)
    doms = D.split(slabs, pos, vel, types, mass)
    assert sum(d.n for d in doms) == pos.shape[0]
    E, forces, W = D.evaluate_serial(slabs, doms, oracle_engine(om, RC))
    F = _gather(slabs, doms, forces, pos.shape[0])
    scale = np.abs(ref["forces"]).max()
    assert abs(E - ref["energy"]) <= 1e-11 * abs(ref["energy"])
    assert np.abs(F - ref["forces"]).max() <= 1e-10 * scale
    assert np.abs(W - ref["virial"]).max() <= 1e-10 * np.abs(ref["virial"]).max()


def test_slabs_reject_a_halo_wider_than_a_slab():
    with pytest.raises(ValueError):
        D.Slabs([20.0, 20.0, 20.0], [1, 1, 1], 5, RC)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out, nsteps):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pos, box, pbc, types, vel, mass, p = _system()
        om = O.OracleModel(p)
        slabs = D.Slabs(box, pbc, world, RC)
        d = D.split(slabs, pos, vel, types, mass)[rank]
        comm = D.TorchComm(dist)
        eng = oracle_engine(om, RC)
        f, E, W = D.evaluate(comm, d, eng)
        res = {"E": E, "W": W, "gid": d.gid.copy(), "F": f}
        # velocity-Verlet with migration between slabs after every drift
        dt, conv = 1.0, 1.0 / 103.6427
        for _ in range(nsteps):
            d.vel += 0.5 * dt * f / d.mass[:, None] * conv
            d.pos += dt * d.vel
            D.migrate(comm, d)
            f, E2, _ = D.evaluate(comm, d, eng)
            d.vel += 0.5 * dt * f / d.mass[:, None] * conv
        res.update(md_gid=d.gid.copy(), md_pos=d.pos.copy(), md_vel=d.vel.copy(), md_E=E2)
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_equal_single_box(world):
    """Forward and reverse exchanges over gloo: the gathered forces, energy
    and virial equal the single-box oracle; 6 MD steps with migration between
    slabs follow the single-box oracle trajectory."""
    nsteps = 6
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out, nsteps)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(300)
            assert pr.exitcode == 0
        res = dict(out)
    pos, box, pbc, types, vel, mass, p = _system()
    om = O.OracleModel(p)
    ref = O.evaluate(om, pos, types, box, pbc)
    n = pos.shape[0]
    F = np.zeros((n, 3))
    for r in range(world):
        F[res[r]["gid"]] = res[r]["F"]
        assert res[r]["E"] == res[0]["E"] and np.array_equal(res[r]["W"], res[0]["W"])
    assert abs(res[0]["E"] - ref["energy"]) <= 1e-11 * abs(ref["energy"])
    assert np.abs(F - ref["forces"]).max() <= 1e-10 * np.abs(ref["forces"]).max()
    assert np.abs(res[0]["W"] - ref["virial"]).max() <= 1e-10 * np.abs(ref["virial"]).max()
    # the same MD in one box (the oracle's velocity-Verlet and wrap)
    sys1 = I.System(pos.copy(), types, box, pbc, vel=vel.copy(), masses=mass)
    traj = O.md(om, sys1, nsteps, 1.0)
    p_ref, v_ref = traj[0], traj[1]
    P = np.zeros((n, 3))
    V = np.zeros((n, 3))
    for r in range(world):
        P[res[r]["md_gid"]] = res[r]["md_pos"]
        V[res[r]["md_gid"]] = res[r]["md_vel"]
    dp = P - p_ref
    dp -= np.round(dp / box) * box           # the decomposed run wraps x at every migration
    assert np.abs(dp).max() <= 1e-9
    assert np.abs(V - v_ref).max() <= 1e-9 * np.abs(v_ref).max()


@pytest.mark.gpu
@pytest.mark.parametrize("R", [1, 3])
def test_gpu_domains_equal_whole_box(tmdlib, R):
    """tmd_compute_owned per domain, ghosts handed back: the gathered forces
    equal tmd_compute on the whole box within the FP32 bars."""
    import torch
    w = I.large(reps=16)                  # 16,384 atoms, L = 64.8 A
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    pos = torch.as_tensor(s.pos, device="cuda")
    types = torch.as_tensor(s.types, device="cuda")
    nl = tmdlib.NeighborList()
    nl.build(pos, types, s.box, s.pbc, w.model.rc)
    ref = tmdlib.evaluate(m, nl, pos, types, s.box)
    torch.cuda.synchronize()
    E0 = float(ref["energy"].item())
    F0 = ref["forces"].double().cpu().numpy()
    W0 = ref["virial"].cpu().numpy().reshape(3, 3)
    slabs = D.Slabs(s.box, s.pbc, R, w.model.rc)
    doms = D.split(slabs, s.pos, np.zeros_like(s.pos), s.types, s.masses)
    E, forces, W = D.evaluate_serial(slabs, doms, D.gpu_engine(tmdlib, m, torch, w.model.rc))
    F = _gather(slabs, doms, forces, s.n)
    rms = np.sqrt((F0 ** 2).mean())
    assert abs(E - E0) <= 1e-6 * abs(E0)
    assert np.abs(F - F0).max() <= 1e-5 * rms
    assert np.abs(W - W0).max() <= 1e-5 * np.abs(W0).max()
