"""Continuous-batching MD force server over resident systems.

Every system's state lives in one batch (``tmd.Batch``); its neighbour table
and the evaluation workspace of its atoms are what a system holds on the
device while it is *resident*.  Requests (system id, number of MD steps)
arrive open-loop.  Every tick the server
- queues the requests that arrived,
- admits systems with queued requests while the device-memory budget allows
  (releasing the tables of idle resident systems, least recently used first,
  when it does not), so a request whose system cannot be admitted waits,
- advances all systems that have an active request by one velocity-Verlet
  step in a single batched call (one set of launches over the union of their
  atoms; tables kept between ticks with the batch's skin policy),
- retires the requests that are done.
Requests for the same system are served in arrival order, so every system's
trajectory is the one it would have alone.  ``serve_alone`` is the baseline:
each request as its own call, first come first served.
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


class Residency:
    """Device-memory admission: which systems hold a table and workspace.

    need[k] = bytes system k holds while resident.  A system is admitted when
    the resident total plus its need fits the budget; otherwise idle resident
    systems (no active or queued request) are released, least recently used
    first, until it fits.  A system larger than the whole budget is refused
    at construction (it could never run)."""

    def __init__(self, batch, need, budget_bytes):
        self.batch, self.need, self.budget = batch, list(need), budget_bytes
        self.resident = collections.OrderedDict()     # system -> last use (LRU order)
        self.used = 0
        self.admissions = self.releases = 0
        too_big = [k for k, b in enumerate(self.need) if budget_bytes is not None and b > budget_bytes]
        if too_big:
            raise ValueError(f"systems {too_big} need more than the whole budget of {budget_bytes} bytes")

    def admit(self, k, busy):
        """True when system k is (now) resident; busy = systems that must stay."""
        if k in self.resident:
            self.resident.move_to_end(k)
            return True
        if self.budget is not None:
            if self.used + self.need[k] > self.budget:
                idle = [j for j in self.resident if j not in busy]
                freed = sum(self.need[j] for j in idle)
                if self.used - freed + self.need[k] > self.budget:
                    return False                      # wait: not enough idle memory to release
                for j in idle:
                    if self.used + self.need[k] <= self.budget:
                        break
                    self.batch.release(j)
                    self.used -= self.need[j]
                    del self.resident[j]
                    self.releases += 1
        self.resident[k] = True
        self.used += self.need[k]
        self.admissions += 1
        return True


def serve_batched(batch, model, requests, dt=1.0, clock=time.perf_counter, realtime=True, residency=None):
    """Run the continuous-batching loop; returns (requests, stats).
    residency: a Residency (device-memory admission), or None (no budget)."""
    pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
    queues = collections.defaultdict(collections.deque)   # system -> waiting requests
    active = {}                                           # system -> [request, steps left]
    t0 = clock()
    atom_steps, ticks, waited = 0, 0, set()
    finished = []
    while pending or queues or active:
        now = clock() - t0
        if not realtime and not active and pending and not queues:
            now = max(now, pending[0].arrival)
        while pending and pending[0].arrival <= now:
            r = pending.popleft()
            queues[r.system].append(r)
        for sysid in sorted(queues, key=lambda k: queues[k][0].arrival):
            if sysid not in active and queues[sysid]:
                if residency is not None and not residency.admit(sysid, set(active) | set(queues)):
                    waited.add(queues[sysid][0].rid)
                    continue
                r = queues[sysid].popleft()
                r.start = now
                active[sysid] = [r, r.steps]
            if not queues[sysid]:
                del queues[sysid]
        if not active:
            if pending and realtime:
                time.sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.002)))
            elif not pending and queues:
                raise RuntimeError("requests wait on memory that no idle system can free")
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
    st = _stats(finished, atom_steps, wall, ticks)
    if residency is not None:
        st.update(admissions=residency.admissions, releases=residency.releases, waited_on_memory=len(waited))
    return finished, st


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
