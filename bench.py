#!/usr/bin/env python
"""Benchmark: TensorMD molecular-dynamics steps on one GB300 (or N replicas).

One step = one velocity-Verlet step of the whole hot path: half kick + drift +
wrap, cell binning and neighbour table rebuild, fused descriptor kernel,
per-species network forward/backward, backward pair kernel with ScatterSum and
virial, final reductions, second half kick.  The neighbour table is rebuilt
every step inside the timed region.

Default workload: the 1,048,576-atom fcc cell (64^3, a = 4.05 A, sigma = 0.1 A
jitter, rc = 6 A, 1 A skin, K = 16, network 64-64-1 tanh, random weights).
Inputs are larger than L2 (the neighbour table alone is ~0.7 GB).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
(the only reference implementation: the paper ships no code) on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "force-eval atom-steps/s on 1 GB300 (plain FP32 vs BF16 form); serving p50/p99"
UNIT = "atom-steps/s"
CONV = 1.0 / 103.6427

# algorithmic flops per in-cutoff pair (FMA = 2 flops), from the operation
# counts of the tensor chain: forward P = sum H M (K x 20 FMA) + radial basis
# (~8 per channel) + geometry/moments (~50); backward U and V (2 x K x 20 FMA),
# H' (K FMA), radial basis with derivative (~10 per channel), M' contraction
# and projection (~120), virial (~45).
def fwd_flops_per_pair(K):
    return 2 * 20 * K + 8 * K + 50


def bwd_flops_per_pair(K):
    return 2 * (2 * 20 * K + K) + 10 * K + 165


def mlp_flops_per_atom(dims):
    # forward + input-gradient backward: 2 GEMV passes of sum(in*out) FMAs
    return 4 * sum(dims[i] * dims[i + 1] for i in range(len(dims) - 1))


def max_over_ranks(x, dist, device):
    """The slowest rank's value (times are reported as the max over ranks)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, atoms_per_rank, steps, seconds):
    """Whole-job atom-steps/s of `world` independent replicas (weak scaling)."""
    return world * atoms_per_rank * steps / seconds


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        import tempfile
        # TMD_CLOCKS_DIR keeps the samples (e.g. next to the bench output); default: a temporary directory
        self.path = os.path.join(os.environ.get("TMD_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def _lines(self):
        try:
            self.f.flush()
            with open(self.path) as fh:
                return fh.read().count("\n")
        except Exception:
            return 0

    def wait_first(self, timeout=3.0):
        """Block until nvidia-smi has written its first sample (its start-up
        takes longer than a short timed region) and remember how many lines
        precede the timed region: only later samples are kept."""
        self.skip = 0
        if self.proc is None:
            return
        t0 = time.time()
        while self._lines() == 0 and time.time() - t0 < timeout:
            time.sleep(0.02)
        self.skip = self._lines()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path).read().splitlines()[getattr(self, "skip", 0):]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_traffic(name):
    """Per-launch DRAM bytes of ``name`` from the committed ncu summary, if it was
    taken on the current sources of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    import hashlib
    with open(path) as f:
        d = json.load(f)
    k = d.get("kernels", {}).get(name)
    if k is None:
        return None
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2310_08439_gb300", "csrc")
    for fn in k.get("sources", []):
        fp = os.path.join(csrc, fn)
        if not os.path.exists(fp):
            return None
        h.update(open(fp, "rb").read())
    if k.get("sources_sha256") != h.hexdigest():
        return None
    return k.get("bytes_per_launch_full")


def workload(name, reps=64, rebuild_every=5):
    from paper_2310_08439_gb300 import inputs as I
    cadence = ("neighbour table rebuilt every step" if rebuild_every == 1 else
               f"neighbour table rebuilt every {rebuild_every} steps with a 1 A buffer (the paper's MD setting)")
    if name == "large":
        w = I.large(reps=reps)
        desc = (f"large: {reps}^3 fcc bulk, {w.systems[0].n:,} atoms, a=4.05 A, jitter 0.1 A, 1 species; rc 6 A, skin 1 A, "
                f"K=16, ranks 0-3, network 64-64-1 tanh (random init); velocity-Verlet dt=1 fs, {cadence}")
    elif name == "medium":
        w = I.medium()
        desc = ("medium: 16^3 fcc bulk, 16,384 atoms, a=3.61 A, 2 species, jitter 0.1 A; rc 6 A, skin 1 A, "
                f"K=16, network 64-64-1 per species; velocity-Verlet dt=1 fs, {cadence}")
    else:
        raise SystemExit(f"unknown config {name}")
    return w, desc


def compute_only_rate(tmd, model, sysm, s, w, steps, torch, stream, want_forces=False):
    """tmd_compute alone (descriptors + network + backward + scatter), table built once."""
    p, _, _ = sysm.get_state()
    pos = torch.as_tensor(np.mod(p, s.box), device="cuda")
    types = torch.as_tensor(s.types, device="cuda")
    nl = tmd.NeighborList()
    nl.build(pos, types, s.box, s.pbc, w.model.rc)
    n = s.n
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    W = torch.zeros(9, dtype=torch.float64, device="cuda")
    for _ in range(3):
        tmd.compute(model, nl, pos, types, s.box, E, None, F, W)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        tmd.compute(model, nl, pos, types, s.box, E, None, F, W)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    out = {"value": n / (ms * 1e-3), "unit": UNIT, "ms_per_eval": ms,
           "what": "tmd_compute on a fixed table (no neighbour build, no integration)"}
    if want_forces:
        out["forces"] = F.double().cpu().numpy()
    return out


def radial_table_measure(tmd, model, sysm, s, w, steps, torch, stream):
    """Tabulated radial basis (H and H' interpolated from a table, cutoff
    folded in) against direct evaluation of the Gaussians and the cutoff:
    tmd_compute rate on the same fixed neighbour table, and the largest force
    difference from the direct path on this workload."""
    out = {"what": "tmd_compute with H, H' from a table of ppa points per A (cubic Hermite) vs direct"}
    ref = compute_only_rate(tmd, model, sysm, s, w, steps, torch, stream, want_forces=True)
    rms = float(np.sqrt((ref["forces"] ** 2).mean()))
    out["direct"] = {"value": ref["value"], "ms_per_eval": ref["ms_per_eval"]}
    try:
        for ppa in (128, 1024):
            model.set_radial_table(ppa)
            r = compute_only_rate(tmd, model, sysm, s, w, steps, torch, stream, want_forces=True)
            out[f"ppa_{ppa}"] = {"value": r["value"], "ms_per_eval": r["ms_per_eval"],
                                 "speedup": ref["ms_per_eval"] / r["ms_per_eval"],
                                 "dF_max_over_rms_vs_direct": float(np.abs(r["forces"] - ref["forces"]).max()) / rms}
    finally:
        model.set_radial_table(0)
    return out


def batch_measure(tmd, torch, steps=5):
    """512 uneven systems (configs: batch) evaluated by one set of launches, FP32
    and BF16 network forms.  Returns the measurement and every system's energy
    and forces in both forms (compared with the FP64 oracle in the oracle leg,
    ``batch_errors``)."""
    from paper_2310_08439_gb300 import inputs as I
    w = I.batch()
    n_tot = int(sum(x.n for x in w.systems))
    ids = list(range(len(w.systems)))
    out = {"workload": "512 periodic systems, n ~ logU(32, 8192) (total %d atoms), fcc/bcc/hcp a ~ U(2.9, 4.1), "
                       "1-3 species, rc 6, K 16, network 192-128-128-1" % n_tot}
    m = tmd.Model(w.model)
    b = tmd.Batch(w.systems, skin=1.0)   # resident tables, built once (the positions do not move)
    sample = ids
    results = {}
    for prec in ("fp32", "bf16"):
        m.set_precision(prec)
        tuning = b.autotune(m, ids)   # tile shapes for this batch and form
        b.compute(m, ids)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            E, Wv = b.compute(m, ids)
        dt = (time.perf_counter() - t0) / steps
        results[prec] = {k: (float(E[k]), b.get_system(k)[2].astype(np.float64)) for k in sample}
        out[prec] = {"atom_evals_per_s": n_tot / dt, "ms_per_batch_eval": dt * 1e3, "tuning": tuning,
                     "errors": None}
    return out, (w, sample, results)


def batch_errors(extras_batch, sampled):
    """Oracle leg: every batch system's energy and force errors against the
    FP64 oracle, both network forms (per-system lists in system order, and
    their summary)."""
    from oracle import oracle as O
    w, sample, results = sampled
    om = O.OracleModel(w.model)
    t0 = time.perf_counter()
    rows = {prec: {"dE_rel": [], "dF_max_over_rms": []} for prec in results}
    for k in sample:
        s = w.systems[k]
        o = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
        rms = float(np.sqrt((o["forces"] ** 2).mean()))
        for prec, res in results.items():
            e, f = res[k]
            rows[prec]["dE_rel"].append(abs(e - o["energy"]) / abs(o["energy"]))
            rows[prec]["dF_max_over_rms"].append(float(np.abs(f - o["forces"]).max() / rms))
    secs = time.perf_counter() - t0
    for prec, r in rows.items():
        dE, dF = np.array(r["dE_rel"]), np.array(r["dF_max_over_rms"])
        extras_batch[prec]["errors"] = {
            "systems": len(sample), "atoms": int(sum(w.systems[k].n for k in sample)),
            "max_dE_rel": float(dE.max()), "median_dE_rel": float(np.median(dE)),
            "max_dF_over_rms": float(dF.max()), "median_dF_over_rms": float(np.median(dF)),
            "p99_dF_over_rms": float(np.percentile(dF, 99)),
            "systems_over_1e-5_dF": int((dF > 1e-5).sum()),
            "per_system": {"n": [int(w.systems[k].n) for k in sample],
                           "dE_rel": [float("%.3g" % x) for x in dE],
                           "dF_max_over_rms": [float("%.3g" % x) for x in dF]},
            "oracle_seconds": secs}


def paper_models_measure(tmd, torch, steps=5):
    """The paper's two potential geometries (Sec. "The Potential": k = 32 with a
    128-128-128-1 network, k = 128 with 128-128-128-128-1, SquarePlus) on
    random weights, on 1,024,000-atom bcc W lattices at the two lattice
    constants of the paper's weak-scaling runs; tmd_compute on a fixed table,
    FP32 and BF16 network forms."""
    from paper_2310_08439_gb300 import inputs as I

    def bcc_w(a, reps, seed):
        rng = np.random.default_rng(seed)
        pos, box = I.lattice("bcc", reps, a)
        return I.System(I.jitter_and_wrap(pos, box, 0.1, rng), np.zeros(len(pos), np.int32), box,
                        np.ones(3, np.int32))

    out = {"workload": "bcc W 80^3 x 2 = 1,024,000 atoms, jitter 0.1 A, rc 6 A (no skin), 1 species; "
                       "first layer normalised by the descriptor RMS of a 432-atom cell (GPU descriptors)"}
    for k, widths in ((32, [128, 128, 128]), (128, [128, 128, 128, 128])):
        for a in (3.1887, 2.8):
            small = bcc_w(a, (6, 6, 6), 1)
            p0 = I.random_model(1, k, 6.0, widths, seed=k, activation="squareplus", masses=[183.84])
            # first-layer scale: descriptor RMS over a 432-atom cell (descriptors do not depend on the weights)
            m0 = tmd.Model(p0)
            nl0 = tmd.NeighborList()
            pos0 = torch.as_tensor(small.pos, device="cuda")
            typ0 = torch.as_tensor(small.types, device="cuda")
            nl0.build(pos0, typ0, small.box, small.pbc, 6.0)
            G = tmd.descriptors(m0, nl0, pos0, typ0, small.box).double().cpu().numpy()
            del m0, nl0
            p = I.random_model(1, k, 6.0, widths, seed=k, activation="squareplus", masses=[183.84],
                               feature_scale=np.sqrt((G ** 2).mean(axis=0)).reshape(1, -1))
            s = bcc_w(a, (80, 80, 80), 2)
            m = tmd.Model(p)
            pos = torch.as_tensor(s.pos, device="cuda")
            types = torch.as_tensor(s.types, device="cuda")
            nl = tmd.NeighborList()
            nl.build(pos, types, s.box, s.pbc, 6.0)
            E = torch.zeros(1, dtype=torch.float64, device="cuda")
            F = torch.zeros((s.n, 3), dtype=torch.float32, device="cuda")
            W = torch.zeros(9, dtype=torch.float64, device="cuda")
            row = {"n": s.n, "pairs_listed": int(nl.size()[1])}
            for prec in ("fp32", "bf16"):
                m.set_precision(prec)
                for _ in range(2):
                    tmd.compute(m, nl, pos, types, s.box, E, None, F, W)
                torch.cuda.synchronize()
                tmd.profile_read(reset=True)
                tmd.profile_enable(True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(steps):
                    tmd.compute(m, nl, pos, types, s.box, E, None, F, W)
                e1.record()
                torch.cuda.synchronize()
                tmd.profile_enable(False)
                ks = tmd.profile_read(reset=True)
                ms = e0.elapsed_time(e1) / steps
                row[prec] = {"atom_evals_per_s": s.n / (ms * 1e-3), "ms_per_eval": ms,
                             "kernel_ms": {kk: v[1] / max(v[0], 1) for kk, v in ks.items()
                                           if kk in ("k_desc", "k_force", "k_mlp", "k_mlp_res", "k_mlp_bf16", "k_mlp_umma")}}
            out[f"k{k}_a{a}"] = row
            del nl, m, pos, types, E, F, W
            torch.cuda.empty_cache()
    return out


def graphs_measure(tmd, torch, steps=60):
    """Launch overhead: the medium cell (16,384 atoms) advanced one step per
    call with the skin check (rebuild only when an atom moved > skin/2), eager
    launches vs the captured CUDA graph of the evaluation + half kick."""
    from paper_2310_08439_gb300 import inputs as I
    w = I.medium()
    s = w.systems[0]
    m = tmd.Model(w.model)
    side = torch.cuda.Stream()
    out = {"workload": "medium: 16^3 fcc, 16,384 atoms, 2 species, K 16, 64-64-1; one MD step per call, skin 1 A"}
    for graphs in (False, True):
        tmd.set_graphs(graphs)
        g = tmd.System(s.n, s.box, s.pbc, skin=w.skin)
        g.set_state(s.pos, s.vel, s.types, s.masses, stream=side)
        for _ in range(4):
            g.step(m, w.dt_fs, 1, rebuild_every=0, stream=side, thermo=False)
        side.synchronize()
        r0 = tmd.graph_replays()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(side)
        for _ in range(steps):
            g.step(m, w.dt_fs, 1, rebuild_every=0, stream=side, thermo=False)
        e1.record(side)
        side.synchronize()
        ms = e0.elapsed_time(e1)
        out["graphs" if graphs else "eager"] = {"value": s.n * steps / (ms * 1e-3), "unit": UNIT,
                                               "ms_per_step": ms / steps, "replays": tmd.graph_replays() - r0}
    tmd.set_graphs(True)
    # many steps per call: runs of steps decided on the device (tmd_step),
    # with the paper's cadence (table every 5 steps) and with the skin
    # criterion alone
    for every, name in ((5, "runs_every_5"), (0, "runs_skin_criterion")):
        g = tmd.System(s.n, s.box, s.pbc, skin=w.skin)
        g.set_state(s.pos, s.vel, s.types, s.masses, stream=side)
        g.step(m, w.dt_fs, 12, rebuild_every=every, stream=side, thermo=False)   # captures
        side.synchronize()
        c0 = g.counters()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        nsteps = 10 * steps
        e0.record(side)
        g.step(m, w.dt_fs, nsteps, rebuild_every=every, stream=side, thermo=False)
        e1.record(side)
        side.synchronize()
        ms = e0.elapsed_time(e1)
        c1 = g.counters()
        out[name] = {"value": s.n * nsteps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / nsteps,
                     "steps": nsteps, "runs": c1["runs"] - c0["runs"], "reruns": c1["reruns"] - c0["reruns"],
                     "rebuilds": c1["rebuilds"] - c0["rebuilds"]}
    return out


def serving_measure(tmd, seconds, torch):
    """Serving workload (configs: serve): 256 systems of 64-50,000 atoms,
    Poisson requests of 1-10 MD steps on a uniformly chosen system.  Each arm's
    capacity is measured first (batched: every system stepped in every tick;
    per request: back-to-back calls), then a load sweep offers 0.25 / 0.5 /
    0.75 / 0.9 of that capacity over the same arrival window and reports the
    steady-state p50 / p99 latency; the batched FP32 arm also runs the per
    request arm's own request streams.  Systems are admitted by device memory
    (serve.Residency, half of the free memory) with resident tables (1 A skin,
    rebuilt every 5 steps or on the skin criterion)."""
    from paper_2310_08439_gb300 import inputs as I
    from paper_2310_08439_gb300 import serve
    w = I.serve()
    systems = w.systems
    free, _ = torch.cuda.mem_get_info()
    per = serve.bytes_per_atom(w.model)
    need = [int(x.n) * per for x in systems]
    budget = int(0.5 * free)
    m = tmd.Model(w.model)
    mean_work = float(np.mean([x.n for x in systems])) * 5.5          # atom-steps per request
    fracs = (0.25, 0.5, 0.75, 0.9)
    res = {"workload": "%d systems (%d atoms, 64-50,000 each, fcc/bcc, 1-2 species), Poisson requests of "
                       "U{1..10} MD steps, network 128-128-1; arrival window %.2f s per load point"
                       % (len(systems), sum(x.n for x in systems), seconds),
           "budget_bytes": budget, "estimated_bytes_all": int(sum(need)), "mean_atom_steps_per_request": mean_work}
    ids = list(range(len(systems)))

    def batched(prec):
        m.set_precision(prec)
        b = tmd.Batch(systems, skin=1.0, rebuild_every=5)
        b.step(m, ids, 1.0, 1)                      # tables, initial forces, graphs
        return b

    def sweep(arm, b, cap, seed0, rates=None):
        pts = []
        for i, f in enumerate(fracs):
            rate = (rates[i] if rates else f * cap / mean_work)
            reqs = serve.poisson_requests(len(systems), rate, seconds, seed=seed0 + i)
            if arm == "alone":
                _, st = serve.serve_alone(b, m, reqs)
            else:
                _, st = serve.serve_batched(b, m, reqs, residency=serve.Residency(b, need, budget))
            st.update(offered_fraction=f if not rates else None, rate_per_s=rate,
                      offered_atom_steps_per_s=rate * mean_work)
            pts.append(st)
        return pts

    for prec in ("fp32", "bf16"):
        b = batched(prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ticks = 4
        b.step(m, ids, 1.0, ticks)
        cap = ticks * float(sum(x.n for x in systems)) / (time.perf_counter() - t0)
        res["batched_" + prec] = {"capacity_atom_steps_per_s": cap, "sweep": sweep("batched", b, cap, 100)}
    m.set_precision("fp32")
    b = batched("fp32")
    burst = serve.poisson_requests(len(systems), 1e6, 1e-4 * 60, seed=7)    # ~60 requests at t ~ 0
    _, st = serve.serve_alone(b, m, burst, realtime=False)
    cap_alone = st["atom_steps"] / st["wall_s"]
    alone_pts = sweep("alone", b, cap_alone, 200)
    res["per_request_fp32"] = {"capacity_atom_steps_per_s": cap_alone, "sweep": alone_pts}
    b = batched("fp32")
    res["batched_fp32_at_per_request_loads"] = sweep("batched", b, None, 200,
                                                     rates=[p["rate_per_s"] for p in alone_pts])
    # the serving configuration's own rate, 2,000 requests/s, on every arm
    # (the same arrivals; the per-request arm is past its capacity there and
    # drains its queue after the window)
    res["at_2000_per_s"] = {}
    for arm, prec in (("batched_fp32", "fp32"), ("batched_bf16", "bf16"), ("per_request_fp32", "fp32")):
        b = batched(prec)
        reqs = serve.poisson_requests(len(systems), 2000.0, seconds, seed=300)
        if arm == "per_request_fp32":
            _, st = serve.serve_alone(b, m, reqs)
        else:
            _, st = serve.serve_batched(b, m, reqs, residency=serve.Residency(b, need, budget))
        st.update(rate_per_s=2000.0, offered_atom_steps_per_s=2000.0 * mean_work)
        res["at_2000_per_s"][arm] = st
    m.set_precision("fp32")
    return res


class OracleMD:
    """The FP64 oracle's MD loop on a bounded sample, with the neighbour
    cadence of the GPU loop: velocity-Verlet from the oracle's own functions;
    the table (radius rc + skin) is rebuilt every ``rebuild_every`` steps after
    wrapping the positions, and between rebuilds the drift leaves them
    unwrapped so that the table's image shifts stay valid (as on the GPU)."""

    def __init__(self, O, w, s, rebuild_every):
        self.O, self.w, self.s, self.R = O, w, s, max(1, int(rebuild_every))
        self.om = O.OracleModel(w.model)
        self.pos = s.pos.copy()
        self.vel = s.vel.copy() if s.vel is not None else np.zeros_like(s.pos)
        self.nopbc = np.zeros(3, np.int32)
        self.k = 0
        self._rebuild()
        self.forces = O.compute(self.om, self.pos, s.types, s.box, self.nl)["forces"]

    def _rebuild(self):
        s = self.s
        per = np.asarray(s.pbc, bool)
        self.pos[:, per] = np.mod(self.pos[:, per], np.asarray(s.box)[per])
        self.nl = self.O.neighbors(self.pos, s.box, s.pbc, self.w.model.rc + self.w.skin)

    def step(self):
        O, s = self.O, self.s
        O.vv_first(self.pos, self.vel, self.forces, s.masses, s.box, self.nopbc, 1.0)   # kick + drift
        self.k += 1
        if self.k % self.R == 0:
            self._rebuild()
        self.forces = O.compute(self.om, self.pos, s.types, s.box, self.nl)["forces"]
        O.vv_second(self.vel, self.forces, s.masses, 1.0)


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo where the kernel gives one)."""
    import platform
    arm = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
                if key in ("cpu implementer", "cpu part") and key not in arm:
                    arm[key] = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if arm:   # Arm cores name themselves by implementer and part number
        return (f"{platform.machine()} (CPU implementer {arm.get('cpu implementer', '?')}, "
                f"part {arm.get('cpu part', '?')})")
    return platform.processor() or platform.machine()


def oracle_sample_rate(wname, rebuild_every=5, min_seconds=10.0, max_steps=50):
    """Oracle MD steps (velocity-Verlet, evaluation, the neighbour table every
    ``rebuild_every`` steps) on a bounded sample of the workload: a 12^3 cell
    of the same lattice, model and jitter (6,912 atoms).  Returns
    (atom-steps/s, threads, description, atoms, steps, seconds)."""
    from oracle import oracle as O
    from paper_2310_08439_gb300 import inputs as I
    w, _ = workload(wname)
    s = I.large(reps=12).systems[0] if wname == "large" else w.systems[0]
    md = OracleMD(O, w, s, rebuild_every)
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        md.step()
        steps += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    dt = time.perf_counter() - t0
    desc = (f"FP64 C oracle (OpenMP), {steps} MD steps (evaluation + velocity-Verlet, O(N^2) neighbour search "
            f"every {md.R} steps) on a {s.n}-atom cell of the same lattice/model")
    return s.n * steps / dt, O.num_threads(), desc, s.n, steps, dt


def oracle_split(wname, reps=3):
    """The two parts of an oracle step timed apart on the same sample: the
    O(N^2) neighbour search and the FP64 evaluation on its table."""
    from oracle import oracle as O
    from paper_2310_08439_gb300 import inputs as I
    w, _ = workload(wname)
    s = I.large(reps=12).systems[0] if wname == "large" else w.systems[0]
    om = O.OracleModel(w.model)
    t0 = time.perf_counter()
    for _ in range(reps):
        nl = O.neighbors(s.pos, s.box, s.pbc, w.model.rc)
    t_nl = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        O.compute(om, s.pos, s.types, s.box, nl)
    t_c = (time.perf_counter() - t0) / reps
    return {"atoms": s.n, "neighbour_search_ms": t_nl * 1e3, "compute_ms": t_c * 1e3,
            "compute_atom_evals_per_s": s.n / t_c}


def size_sweep(tmd, torch, reps_list, steps, warmup, rebuild_every):
    """The FP32 MD step of the large lattice (same recipe, 4 reps^3 atoms) at
    several sizes: atom-steps/s, ms/step and the device memory the system,
    model and workspaces take.  Built-in tile shapes (no autotuning)."""
    out = []
    for reps in reps_list:
        w, _ = workload("large", reps, rebuild_every)
        s = w.systems[0]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        model = tmd.Model(w.model)
        sysm = tmd.System(s.n, s.box, s.pbc, skin=w.skin)
        sysm.set_state(s.pos, s.vel if s.vel is not None else np.zeros_like(s.pos), s.types, s.masses)
        for _ in range(warmup):
            sysm.step(model, w.dt_fs, 1, rebuild_every=rebuild_every, thermo=False)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sysm.step(model, w.dt_fs, 1, rebuild_every=rebuild_every, thermo=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        used = free0 - torch.cuda.mem_get_info()[0]
        out.append({"reps": reps, "atoms": s.n, "atom_steps_per_s": s.n / (ms * 1e-3), "ms_per_step": ms,
                    "device_bytes": int(used), "device_bytes_per_atom": used / s.n})
        del sysm, model
        torch.cuda.synchronize()
    return out


def nve_run(tmd, torch, total_steps, every, rebuild_every, precision="fp32"):
    """Energy conservation of the MD loop on the 1,048,576-atom lattice
    (300 K start, 1 fs steps): total energy per atom every ``every`` steps,
    with the table rebuilt every ``rebuild_every`` steps (0: only when an atom
    moved more than skin/2); ``precision`` is the network form."""
    w, _ = workload("large", 64, rebuild_every)
    s = w.systems[0]
    model = tmd.Model(w.model, precision=precision)
    sysm = tmd.System(s.n, s.box, s.pbc, skin=w.skin)
    sysm.set_state(s.pos, s.vel, s.types, s.masses)
    th = sysm.step(model, w.dt_fs, 0)
    rows = [{"step": 0, "e_tot_per_atom": (th["e_pot"] + th["e_kin"]) / s.n, "temperature": th["temperature"]}]
    done = 0
    while done < total_steps:
        k = min(every, total_steps - done)
        th = sysm.step(model, w.dt_fs, k, rebuild_every=rebuild_every)
        done += k
        rows.append({"step": done, "e_tot_per_atom": (th["e_pot"] + th["e_kin"]) / s.n,
                     "temperature": th["temperature"], "rebuilds": th["rebuilds"]})
    torch.cuda.synchronize()
    e = np.array([r["e_tot_per_atom"] for r in rows])
    return {"atoms": s.n, "dt_fs": w.dt_fs, "rebuild_every": rebuild_every, "precision": precision,
            "steps": total_steps,
            "max_abs_drift_per_atom_eV": float(np.abs(e - e[0]).max()), "trace": rows}


def decompose_run(args, tmd, torch, dist, rank, world):
    """Strong scaling of one system over the ranks (the paper's spatial
    decomposition): the large lattice cut into slabs along x; per evaluation
    every rank exchanges its ghost halo (rc wide), builds its table and runs
    tmd_compute_owned, hands the ghost forces back and all-reduces E and W.
    Returns the JSON line (rank 0)."""
    from paper_2310_08439_gb300 import domain as Dm
    w, desc = workload(args.config, args.reps, rebuild_every=1)
    s = w.systems[0]
    model = tmd.Model(w.model, precision=args.precision)
    slabs = Dm.Slabs(s.box, s.pbc, world, w.model.rc)
    d = Dm.split(slabs, s.pos, np.zeros_like(s.pos), s.types, s.masses)[rank]
    comm = Dm.TorchComm(dist, device="cuda") if dist is not None else Dm.LocalComm()
    engine = Dm.gpu_engine(tmd, model, torch, w.model.rc)
    for _ in range(args.warmup):
        Dm.evaluate(comm, d, engine)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, E, W = Dm.evaluate(comm, d, engine)
    torch.cuda.synchronize()
    t = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    value = s.n * args.steps / t
    return {"metric": "decomposed force evaluations, atom-evals/s (one system over the ranks)", "value": value,
            "unit": "atom-evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": desc, "atoms": s.n, "slabs": world, "halo_A": w.model.rc,
                       "owned_atoms_rank0": int(d.n)},
            "energy": E}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2310_08439_gb300 import inputs as I
    w, desc = workload(args.config, rebuild_every=args.rebuild_every)
    sw = I.large(reps=12) if args.config == "large" else w
    s = sw.systems[0]
    md = OracleMD(O, w, s, args.rebuild_every)
    step = md.step

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = s.n * args.steps / dt
    sample = (f"{s.n}-atom cell of the same lattice and model, {args.steps} MD steps per run, neighbour table "
              f"every {md.R} steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "reference": "FP64 CPU oracle (no code ships "
                                            "with the paper)", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                             "cpu": cpu_model(), "nproc": os.cpu_count(),
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="large", choices=["large", "medium"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16"])
    ap.add_argument("--rebuild-every", type=int, default=5,
                    help="neighbour rebuild cadence of the timed MD loop (the paper's setting: 5)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reps", type=int, default=64, help="fcc repeats of the large cell (64 = 1,048,576 atoms)")
    ap.add_argument("--no-extras", action="store_true", help="skip the batch and serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=1.0, help="arrival window of each serving load point")
    ap.add_argument("--size-sweep", default="",
                    help="instead of the bench line: the FP32 MD step of the large lattice at these fcc repeats "
                         "(e.g. 32,64,128,160), throughput and device memory per size")
    ap.add_argument("--tuning", default="auto",
                    help="tile shapes 'ROWS,BLOCKS_PER_SM' instead of the autotuner (e.g. for profiler captures)")
    ap.add_argument("--nve", default="",
                    help="instead of the bench line: 'STEPS,EVERY' of an NVE run of the large lattice, total energy "
                         "per atom every EVERY steps (table cadence from --rebuild-every)")
    ap.add_argument("--decompose", action="store_true",
                    help="instead of the bench line: one system split into slabs over the ranks (strong scaling "
                         "of the decomposed force evaluation; ghost halo and reverse force exchange)")
    ap.add_argument("--force-kernel", default="auto", choices=["auto", "simt", "tensor"],
                    help="force pass of the unbatched evaluation (tmd_set_force_kernel)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2310_08439_gb300 import build as B
    from paper_2310_08439_gb300 import tmd
    B.build()
    tmd.set_force_kernel(args.force_kernel)
    if args.nve:
        if rank == 0:
            steps_n, every = (int(x) for x in args.nve.split(","))
            print(json.dumps({"nve": nve_run(tmd, torch, steps_n, every, args.rebuild_every, args.precision)}),
                  flush=True)
        return
    if args.decompose:
        line = decompose_run(args, tmd, torch, dist, rank, world)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    if args.size_sweep:
        if rank == 0:
            reps = [int(x) for x in args.size_sweep.split(",")]
            print(json.dumps({"size_sweep": size_sweep(tmd, torch, reps, args.steps, args.warmup,
                                                       args.rebuild_every)}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return
    w, desc = workload(args.config, args.reps, rebuild_every=args.rebuild_every)
    R = args.rebuild_every
    s = w.systems[0]
    n = s.n
    model = tmd.Model(w.model, precision=args.precision)
    sysm = tmd.System(n, s.box, s.pbc, skin=w.skin)
    vel = s.vel if s.vel is not None else np.zeros_like(s.pos)
    sysm.set_state(s.pos, vel, s.types, s.masses)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        sysm.step(model, w.dt_fs, 1, rebuild_every=R, thermo=False)
    torch.cuda.synchronize()
    # tile shapes picked by the autotuner on this system (kept in the model)
    if args.tuning == "auto":
        p_w, _, _ = sysm.get_state()
        nl_t = tmd.NeighborList()
        pos_t = torch.as_tensor(np.mod(p_w, s.box), device=dev)   # unwrapped since the last rebuild
        types_t = torch.as_tensor(s.types, device=dev)
        nl_t.build(pos_t, types_t, s.box, s.pbc, w.model.rc + w.skin)
        tuning = tmd.autotune(model, nl_t, pos_t, types_t, s.box)
        del nl_t, pos_t, types_t
    else:
        rows, bps = (int(x) for x in args.tuning.split(","))
        model.tuning = {"tile_rows": rows, "pair_blocks_per_sm": bps}
        tuning = dict(model.tuning, ms=None)
    for _ in range(args.warmup):
        sysm.step(model, w.dt_fs, 1, rebuild_every=R, thermo=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    tmd.profile_read(reset=True)
    tmd.profile_enable(True)
    launches0 = tmd.launch_count()
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    clocks.wait_first()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        sysm.step(model, w.dt_fs, 1, rebuild_every=R, thermo=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = tmd.launch_count() - launches0
    tmd.profile_enable(False)
    kstats = tmd.profile_read(reset=True)
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    value = replica_throughput(world, n, args.steps, elapsed_ms * 1e-3)

    # the BF16-network form of the same step (same state, same timing rules)
    other = "bf16" if args.precision == "fp32" else "fp32"
    model.set_precision(other)
    for _ in range(args.warmup):
        sysm.step(model, w.dt_fs, 1, rebuild_every=R, thermo=False)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sysm.step(model, w.dt_fs, 1, rebuild_every=R, thermo=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_other = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    forms = {args.precision: {"value": value, "ms_per_step": elapsed_ms / args.steps},
             other: {"value": replica_throughput(world, n, args.steps, t_other * 1e-3),
                     "ms_per_step": t_other / args.steps}}
    model.set_precision(args.precision)

    # the same MD loop with a neighbour rebuild in every step (no reuse of the
    # table at all)
    for _ in range(args.warmup):
        sysm.step(model, w.dt_fs, 1, rebuild_every=1, thermo=False)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sysm.step(model, w.dt_fs, 1, rebuild_every=1, thermo=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_every = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    forms[args.precision + "_rebuild_every_step"] = {
        "value": replica_throughput(world, n, args.steps, t_every * 1e-3), "ms_per_step": t_every / args.steps,
        "what": "neighbour table rebuilt in every step"}

    # the same MD loop with the skin criterion of the velocity-Verlet step
    # (rebuild only once an atom moved more than skin/2 since the last build):
    # a longer run, so that the rebuilds it needs fall inside the timed region
    skin_steps = max(4 * args.steps, 40)
    for _ in range(args.warmup - 1):
        sysm.step(model, w.dt_fs, 1, rebuild_every=0, thermo=False)
    builds0 = sysm.step(model, w.dt_fs, 1, rebuild_every=0, thermo=True)["rebuilds"]
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(skin_steps):
        sysm.step(model, w.dt_fs, 1, rebuild_every=0, thermo=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_skin = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    # one more (untimed) step reads the rebuild counter: the count covers the
    # timed steps and that one
    builds1 = sysm.step(model, w.dt_fs, 1, rebuild_every=0, thermo=True)["rebuilds"]
    forms[args.precision + "_skin_rebuild"] = {
        "value": replica_throughput(world, n, skin_steps, t_skin * 1e-3), "ms_per_step": t_skin / skin_steps,
        "steps": skin_steps, "rebuilds_in_timed_steps_plus_one": int(builds1 - builds0),
        "what": "neighbour table rebuilt only when an atom moved more than skin/2 (the MD loop's own criterion); "
                "the host reads the rebuild flag once per step"}

    # end to end through the host-buffer C-ABI call (pinned host state)
    e2e = None
    if not args.no_e2e:
        th = tmd.Thermo  # noqa: F841
        pos_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        vel_h = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        f_h = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        p_, v_, f_ = sysm.get_state()
        pos_h.numpy()[:] = np.mod(p_, s.box)   # unwrapped since the last rebuild
        vel_h.numpy()[:] = v_
        f_h.numpy()[:] = f_
        sysm.step_host(model, pos_h, vel_h, f_h, w.dt_fs, 1, rebuild_every=R)  # warm
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sysm.step_host(model, pos_h, vel_h, f_h, w.dt_fs, 1, rebuild_every=R)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": replica_throughput(world, n, args.steps, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": int(n * (24 + 24 + 12)), "d2h_bytes_per_step": int(n * (24 + 24 + 12))}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel
    peaks = load_peaks()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = nsm * 128 * 2 * clk_mhz * 1e6 / 1e12  # TFLOP/s
    # units: in-cutoff pairs of the configuration at the timed state
    nl = tmd.NeighborList()
    p_now, _, _ = sysm.get_state()
    pos_d = torch.as_tensor(np.mod(p_now, s.box), device=dev)   # unwrapped since the last rebuild
    types_d = torch.as_tensor(s.types, device=dev)
    nl.build(pos_d, types_d, s.box, s.pbc, w.model.rc)
    pairs = nl.size()[1]          # entries inside rc = in-cutoff pairs
    nl.build(pos_d, types_d, s.box, s.pbc, w.model.rc + w.skin)
    entries = nl.size()[1]        # table entries screened per step (rc + skin)
    K = w.model.n_radial
    dims = [w.model.n_desc] + list(w.model.widths) + [1]
    per_launch_flops = {"k_force": pairs * bwd_flops_per_pair(K), "k_desc": pairs * fwd_flops_per_pair(K),
                        "k_mlp": n * mlp_flops_per_atom(dims), "k_mlp_res": n * mlp_flops_per_atom(dims)}
    ranked = sorted(kstats.items(), key=lambda kv: -kv[1][1])
    dom, (dl, dms) = ranked[0]
    avg_ms = dms / max(dl, 1)
    roof = None
    if dom in per_launch_flops:
        ach = per_launch_flops[dom] / (avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": kernel_traffic(dom),
                "peak_source": f"FP32 FMA peak {nsm} SMs x 128 lanes x 2 flops x {clk_mhz:.0f} MHz "
                               f"(max SM clock, {peaks['source']} peaks file)"}
        # the descriptor and force passes take nearly equal time, so the
        # dominant one can change between runs: every pair/network kernel's
        # figures, the same way
        roof["all"] = {}
        for kn, fl in per_launch_flops.items():
            if kn in kstats:
                a = fl / (kstats[kn][1] / max(kstats[kn][0], 1) * 1e-3) / 1e12
                roof["all"][kn] = {"achieved": a, "frac": a / fp32_peak, "traffic": kernel_traffic(kn)}
        # the in-cutoff screen is a stream: table entries in (nbr int32 +
        # shift char4), pair-cache entries out (float4 + float2 per pair), per
        # atom its split position (2 float4), segment bounds and pair count
        if "k_screen" in kstats:
            sb = entries * 8 + pairs * 24 + n * (32 + 16 + 4)
            a = sb / (kstats["k_screen"][1] / max(kstats["k_screen"][0], 1) * 1e-3) / 1e9
            roof["all"]["k_screen"] = {"bound": "hbm", "achieved": a, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                       "frac": a / peaks["hbm_gbs"], "bytes_per_launch": sb,
                                       "traffic": kernel_traffic("k_screen")}
    total_ms = sum(v[1] for v in kstats.values())
    kernels = {k: {"launches": v[0], "ms_per_launch": v[1] / max(v[0], 1), "share": v[1] / total_ms}
               for k, v in ranked}

    compute_only = compute_only_rate(tmd, model, sysm, s, w, args.steps, torch, stream)
    extras = {}
    if not args.no_extras and world == 1:
        extras["batch"], batch_sample = batch_measure(tmd, torch)
        extras["radial_table"] = radial_table_measure(tmd, model, sysm, s, w, args.steps, torch, stream)
        extras["paper_models"] = paper_models_measure(tmd, torch)
        extras["graphs"] = graphs_measure(tmd, torch)
        extras["serving"] = serving_measure(tmd, args.serve_seconds, torch)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, cores, sdesc, sn, ssteps, sdt = oracle_sample_rate(args.config, rebuild_every=R)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sdesc,
               "cpu": cpu_model(), "nproc": os.cpu_count(), "split": oracle_split(args.config)}
        if "batch" in extras:   # errors of the batch sample against the oracle
            batch_errors(extras["batch"], batch_sample)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f32+bf16-network",
            "data": "synthetic",
            "config": {"workload": desc, "atoms_per_gpu": n, "precision": args.precision,
                       "l2": "inputs larger than L2 (neighbour table ~%.2f GB, %d in-cutoff pairs)"
                             % (nl.size()[1] * 8 / 1e9, pairs),
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "forms": forms, "compute_only": compute_only, "tuning": tuning, "roofline": roof, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk}
    line.update(extras)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
