"""Continuous-batching MD force server over resident systems.

Systems are admitted into one resident batch (``tmd.Batch``) while their
device memory fits the budget.  Requests (system id, number of MD steps)
arrive open-loop; every tick the server advances all systems that have an
active request by one velocity-Verlet step in a single batched call (one set
of launches over the union of their atoms), retires the requests that are
done and admits the ones that arrived meanwhile.  Requests for the same
system are served in arrival order, so every system's trajectory is the one
it would have alone.  ``serve_alone`` is the baseline: each request as its
own plain FP32 call, first come first served.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import tmd

# device bytes per resident atom (state, workspace, neighbour table) for the
# admission estimate: positions/velocities/masses 56, forces 12, per-atom
# energy/virial 40, positions split 32, P/G/G' ~ (S K 20 + 2 Dd) 4, list ~ 8 per entry
def bytes_per_atom(model_params, entries_per_atom=80):
    S, K = model_params.n_species, model_params.n_radial
    Dd = model_params.n_desc
    return 56 + 12 + 40 + 32 + 4 * (S * K * 20 + 2 * Dd) + 24 + 8 * entries_per_atom + 64


@dataclass
class Request:
    rid: int
    system: int
    steps: int
    arrival: float                 # seconds since the start
    start: float = -1.0
    done: float = -1.0
    thermo: dict = field(default_factory=dict)


def poisson_requests(n_systems, rate, duration, seed, max_steps=10):
    """Open-loop arrivals: exponential gaps (mean 1/rate), uniform system,
    U{1..max_steps} MD steps each."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        out.append(Request(len(out), int(rng.integers(0, n_systems)), int(rng.integers(1, max_steps + 1)), t))
    return out


def admit(systems, model_params, budget_bytes):
    """Indices of the systems admitted by the device-memory budget (in order)."""
    per = bytes_per_atom(model_params)
    used, ids = 0, []
    for k, s in enumerate(systems):
        need = s.n * per
        if used + need > budget_bytes:
            continue
        used += need
        ids.append(k)
    return ids, used


def serve_batched(batch, model, requests, dt=1.0, clock=time.perf_counter, realtime=True):
    """Run the continuous-batching loop; returns (requests, stats)."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    queues = collections.defaultdict(collections.deque)   # system -> waiting requests
    active = {}                                           # system -> [request, steps left]
    t0 = clock()
    atom_steps, ticks = 0, 0
    finished = []
    while pending or queues or active:
        now = clock() - t0
        if not realtime and not active and pending:
            now = max(now, pending[0].arrival)
        while pending and pending[0].arrival <= now:
            r = pending.popleft()
            queues[r.system].append(r)
        for sysid in list(queues):
            if sysid not in active and queues[sysid]:
                r = queues[sysid].popleft()
                r.start = now
                active[sysid] = [r, r.steps]
            if not queues[sysid]:
                del queues[sysid]
        if not active:
            if pending and realtime:
                time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.002)))
            continue
        ids = sorted(active)
        th = batch.step(model, ids, dt, 1)
        ticks += 1
        atom_steps += int(sum(batch.n[k] for k in ids))
        t_done = clock() - t0
        for k, sysid in enumerate(ids):
            entry = active[sysid]
            entry[1] -= 1
            if entry[1] == 0:
                r = entry[0]
                r.done = t_done
                r.thermo = th[k]
                finished.append(r)
                del active[sysid]
    wall = clock() - t0
    return finished, _stats(finished, atom_steps, wall, ticks)


def serve_alone(batch, model, requests, dt=1.0, clock=time.perf_counter, realtime=True):
    """Baseline: each request as its own call (one system per call), FIFO."""
    order = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    atom_steps = 0
    for r in order:
        now = clock() - t0
        if now < r.arrival:
            if realtime:
                time.sleep(r.arrival - now)
                now = clock() - t0
            else:
                now = r.arrival
        r.start = now
        th = batch.step(model, [r.system], dt, r.steps)
        r.done = clock() - t0
        r.thermo = th[0]
        atom_steps += int(batch.n[r.system]) * r.steps
    wall = clock() - t0
    return order, _stats(order, atom_steps, wall, len(order))


def _stats(reqs, atom_steps, wall, ticks):
    lat = np.array([r.done - r.arrival for r in reqs]) * 1e3
    return {"requests": len(reqs), "atom_steps": atom_steps, "wall_s": wall,
            "atom_steps_per_s": atom_steps / wall if wall > 0 else 0.0, "calls": ticks,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else math.nan,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else math.nan,
            "mean_ms": float(lat.mean()) if lat.size else math.nan}
