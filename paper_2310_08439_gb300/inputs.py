"""Seeded synthetic inputs shared by the CUDA path and the FP64 oracle.

This module builds atom configurations (fcc / bcc / hcp lattices with Gaussian
jitter, species assignment, Maxwell-Boltzmann velocities) and random-init model
parameters.  It holds none of the potential's arithmetic: no radial function,
moment, descriptor, network evaluation or force is computed here.  Everything
is a NumPy array drawn from ``numpy.random.default_rng(seed)``.

Workload shapes follow the bulk-metal systems the paper simulates (bulk W
lattices, Sec. "Evaluation"; binning with a 1 A buffer, 1 fs steps) but use
Cu/Al-like lattice constants and random weights: the trained W potentials and
the DFT data set are not available.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

# Boltzmann constant in eV/K and the conversion from eV/amu to A^2/fs^2.
KB_EV = 8.617333262e-5
EV_PER_AMU_TO_A2_PER_FS2 = 1.0 / 103.6427

_DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")

# ---------------------------------------------------------------------------
# lattices
# ---------------------------------------------------------------------------
_BASIS = {
    "fcc": (np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]),
            (1.0, 1.0, 1.0)),
    "bcc": (np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.5]]), (1.0, 1.0, 1.0)),
    # orthohexagonal hcp cell (a, sqrt(3) a, sqrt(8/3) a), 4 atoms
    "hcp": (np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0],
                      [0.0, 1.0 / 3.0, 0.5], [0.5, 5.0 / 6.0, 0.5]]),
            (1.0, math.sqrt(3.0), math.sqrt(8.0 / 3.0))),
}


def lattice(kind: str, reps, a: float):
    """Replicate a conventional cell ``reps = (nx, ny, nz)`` times.

    Returns (positions [N,3] float64, box [3] float64).  Atom order is
    cell-major (x fastest), basis atoms innermost.
    """
    basis, cell = _BASIS[kind]
    nx, ny, nz = (int(r) for r in reps)
    cell = np.array(cell) * a
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    origins = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    pos = (origins[:, None, :] + basis[None, :, :]).reshape(-1, 3) * cell
    box = cell * np.array([nx, ny, nz], dtype=np.float64)
    return pos, box


def jitter_and_wrap(pos, box, sigma: float, rng):
    """Add N(0, sigma^2) to every coordinate and wrap into [0, L)."""
    out = pos + rng.normal(0.0, sigma, size=pos.shape)
    out = np.mod(out, box)
    # np.mod can return exactly L for tiny negative inputs; fold those to 0
    out[out >= box] -= box[np.nonzero(out >= box)[1]]
    return np.ascontiguousarray(out)


def maxwell_velocities(masses_per_atom, temperature: float, rng):
    """Maxwell-Boltzmann velocities in A/fs with zero total momentum."""
    m = np.asarray(masses_per_atom, dtype=np.float64)
    sd = np.sqrt(KB_EV * temperature / m * EV_PER_AMU_TO_A2_PER_FS2)
    v = rng.normal(size=(m.size, 3)) * sd[:, None]
    p = (m[:, None] * v).sum(axis=0)
    v -= p / m.sum()
    return np.ascontiguousarray(v)


# ---------------------------------------------------------------------------
# model parameters
# ---------------------------------------------------------------------------
@dataclass
class ModelParams:
    """Random-init potential parameters (all float64).

    mu, eta: [S, S, K] Gaussian centres / widths indexed (centre species,
    neighbour species, channel).  weights[s] is one flat array per centre
    species holding, for layer l = 0..L, W_l [out, in] row-major then b_l [out].
    Descriptor column c = ((b * K) + k) * 4 + m (b = neighbour species).
    """
    n_species: int
    n_radial: int
    rc: float
    widths: list
    mu: np.ndarray
    eta: np.ndarray
    weights: list
    activation: str = "tanh"
    squareplus_b: float = 4.0
    masses: list = field(default_factory=list)

    @property
    def n_desc(self) -> int:
        return self.n_species * self.n_radial * 4

    def layer_shapes(self):
        dims = [self.n_desc] + list(self.widths) + [1]
        return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]

    def unpack(self, s: int):
        """Split species ``s`` weights into [(W_l, b_l), ...]."""
        out, o = [], 0
        flat = self.weights[s]
        for (r, c) in self.layer_shapes():
            W = flat[o:o + r * c].reshape(r, c); o += r * c
            b = flat[o:o + r]; o += r
            out.append((W, b))
        assert o == flat.size
        return out


def default_radial(n_species: int, n_radial: int, rc: float):
    """Evenly spaced Gaussian centres mu_k = k rc/(K-1), eta = 1/(2 delta^2)."""
    delta = rc / (n_radial - 1)
    mu = np.arange(n_radial, dtype=np.float64) * delta
    eta = np.full(n_radial, 1.0 / (2.0 * delta * delta))
    S = n_species
    return (np.ascontiguousarray(np.broadcast_to(mu, (S, S, n_radial))).copy(),
            np.ascontiguousarray(np.broadcast_to(eta, (S, S, n_radial))).copy())


def random_model(n_species, n_radial, rc, widths, seed, feature_scale=None,
                 out_bias=-4.0, activation="tanh", masses=None, scale_floor=0.1, out_scale=0.1):
    """W_l ~ N(0, 1/fan_in); first-layer columns divided by ``feature_scale``;
    output layer ~ N(0, out_scale^2/fan_in).

    ``feature_scale`` ([S, Dd] or None) is the per-column RMS of the descriptor
    over the workload's initial configuration (a stored model statistic, the
    way trained potentials store input normalisation), floored at
    ``scale_floor`` so that channels that are nearly empty in that
    configuration (short-range radial channels, odd ranks in symmetric
    environments) are not amplified more than 10x: with a 1e-2 floor a pair
    that closes to 1.5 A during MD lights up channels whose weights were
    scaled by 100 and dominates the forces.
    ``out_bias`` is the output-layer bias, a cohesive-energy-like offset in
    eV/atom.  ``out_scale`` = 0.1 gives forces of ~0.1 eV/A RMS on the jittered
    lattices, like thermal forces of a metal near equilibrium; with 1.0 the
    random potential drives 300 K runs of the medium cell to pair distances
    below 1 A within 50 fs.
    """
    rng = np.random.default_rng(seed)
    mu, eta = default_radial(n_species, n_radial, rc)
    Dd = n_species * n_radial * 4
    dims = [Dd] + list(widths) + [1]
    weights = []
    for s in range(n_species):
        parts = []
        for l in range(len(dims) - 1):
            fan_in, fan_out = dims[l], dims[l + 1]
            W = rng.normal(0.0, 1.0 / math.sqrt(fan_in), size=(fan_out, fan_in))
            if l == len(dims) - 2:
                W = W * out_scale
            if l == 0 and feature_scale is not None:
                sc = np.maximum(np.asarray(feature_scale[s], dtype=np.float64), scale_floor)
                W = W / sc[None, :]
            b = rng.normal(0.0, 0.1, size=fan_out)
            if l == len(dims) - 2:
                b = b * 0.0 + out_bias
            parts += [W.ravel(), b]
        weights.append(np.ascontiguousarray(np.concatenate(parts)))
    return ModelParams(n_species, n_radial, rc, list(widths), mu, eta, weights,
                       activation=activation,
                       masses=list(masses) if masses is not None else [63.546] * n_species)


def load_feature_scale(name: str, n_species: int, n_desc: int):
    """Stored per-column descriptor RMS for workload ``name`` (or None)."""
    path = os.path.join(_DATA_DIR, "feature_scales.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        table = json.load(f)
    if name not in table:
        return None
    arr = np.asarray(table[name], dtype=np.float64).reshape(n_species, n_desc)
    arr[arr <= 0.0] = 1.0
    return arr


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
@dataclass
class System:
    """One periodic system: positions (wrapped), species, box, pbc, masses."""
    pos: np.ndarray
    types: np.ndarray
    box: np.ndarray
    pbc: np.ndarray
    vel: np.ndarray | None = None
    masses: np.ndarray | None = None  # per atom, amu

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class Workload:
    name: str
    systems: list
    model: ModelParams
    skin: float = 1.0
    dt_fs: float = 1.0
    md_steps: int = 0


def _system(kind, reps, a, sigma, seed_pos, n_species=1, seed_types=None,
            masses=None, temperature=None, seed_vel=None):
    pos, box = lattice(kind, reps, a)
    pos = jitter_and_wrap(pos, box, sigma, np.random.default_rng(seed_pos))
    n = pos.shape[0]
    if n_species == 1:
        types = np.zeros(n, dtype=np.int32)
    else:
        types = np.random.default_rng(seed_types).integers(0, n_species, size=n).astype(np.int32)
    sysm = System(pos, types, box, np.ones(3, dtype=np.int32))
    if masses is not None:
        sysm.masses = np.asarray(masses, dtype=np.float64)[types]
        if temperature is not None:
            sysm.vel = maxwell_velocities(sysm.masses, temperature, np.random.default_rng(seed_vel))
    return sysm


def _mass_for_a(a: float) -> float:
    if abs(a - 3.61) < 1e-9:
        return 63.546
    if abs(a - 4.05) < 1e-9:
        return 26.982
    return 55.845


def tiny(feature_scale=True):
    """32-atom fcc 2x2x2, a=3.61, sigma=0.05 (seed 0); rc 5, K 8, 32-32-1 tanh (seed 1)."""
    s = _system("fcc", (2, 2, 2), 3.61, 0.05, seed_pos=0, masses=[63.546])
    fs = load_feature_scale("tiny", 1, 32) if feature_scale else None
    m = random_model(1, 8, 5.0, [32, 32], seed=1, feature_scale=fs, masses=[63.546])
    return Workload("tiny", [s], m, skin=0.0)


def medium(feature_scale=True):
    """16^3 fcc (16,384 atoms), a=3.61, two species 50/50 (seed 2), sigma 0.1
    (seed 3), 300 K velocities (seed 4); rc 6, skin 1, K 16, 64-64-1 per species."""
    s = _system("fcc", (16, 16, 16), 3.61, 0.1, seed_pos=3, n_species=2, seed_types=2,
                masses=[63.546, 63.546], temperature=300.0, seed_vel=4)
    fs = load_feature_scale("medium", 2, 128) if feature_scale else None
    m = random_model(2, 16, 6.0, [64, 64], seed=11, feature_scale=fs, masses=[63.546, 63.546])
    return Workload("medium", [s], m, skin=1.0, dt_fs=1.0, md_steps=100)


def large(feature_scale=True, reps=64):
    """64^3 fcc (1,048,576 atoms), a=4.05, sigma 0.1 (seed 5); rc 6, K 16, 64-64-1."""
    s = _system("fcc", (reps, reps, reps), 4.05, 0.1, seed_pos=5, masses=[26.982],
                temperature=300.0, seed_vel=15)
    fs = load_feature_scale("large", 1, 64) if feature_scale else None
    m = random_model(1, 16, 6.0, [64, 64], seed=12, feature_scale=fs, masses=[26.982])
    return Workload(f"large" if reps == 64 else f"large_{reps}", [s], m, skin=1.0,
                    dt_fs=1.0, md_steps=20)


def sparse_gas(n=400, L=60.0, dmin=2.2, seed=23):
    """Random dilute gas of two species in a periodic cube (no two atoms closer
    than dmin, seed 23): about 1.7 neighbours within 6 A and 2.7 within 7 A
    per atom, so that many atoms have no pair within 6 A, some of them with
    table entries in a 1 A skin shell."""
    rng = np.random.default_rng(seed)
    box = np.array([L, L, L])
    pos = []
    while len(pos) < n:
        x = rng.uniform(0.0, L, 3)
        if pos:
            d = np.array(pos) - x
            d -= np.round(d / box) * box
            if (d * d).sum(axis=1).min() < dmin * dmin:
                continue
        pos.append(x)
    return System(np.array(pos), rng.integers(0, 2, n).astype(np.int32), box, np.ones(3, np.int32))


def _best_reps(n_target, n_basis, cell):
    """(nx, ny, nz) minimising |basis*nx*ny*nz - n| with box aspect ratio <= 2
    (ties: the first found scanning nx, ny ascending)."""
    best, best_err = (1, 1, 1), None
    lim = max(1, int(round((n_target / n_basis) ** (1.0 / 3.0) * 2.5)) + 1)
    cell = np.asarray(cell)
    for nx in range(1, lim + 1):
        for ny in range(1, lim + 1):
            z0 = max(1, int(round(n_target / (n_basis * nx * ny))))
            for nz in (z0 - 1, z0, z0 + 1):
                if nz < 1:
                    continue
                L = np.array([nx, ny, nz]) * cell
                if L.max() > 2.0 * L.min():
                    continue
                err = abs(n_basis * nx * ny * nz - n_target)
                if best_err is None or err < best_err:
                    best, best_err = (nx, ny, nz), err
    return best


def batch(n_systems=512, seed=6, feature_scale=True):
    """Uneven periodic systems: n ~ logU(32, 8192), fcc/bcc/hcp, a ~ U(2.9, 4.1),
    sigma ~ U(0.05, 0.15), 1-3 species; rc 6, K 16, model 3 species 128-128-1."""
    rng = np.random.default_rng(seed)
    systems = []
    for i in range(n_systems):
        n_t = math.exp(rng.uniform(math.log(32), math.log(8192)))
        kind = ["fcc", "bcc", "hcp"][int(rng.integers(0, 3))]
        a = rng.uniform(2.9, 4.1)
        sigma = rng.uniform(0.05, 0.15)
        ns = int(rng.integers(1, 4))
        basis, cell = _BASIS[kind]
        reps = _best_reps(n_t, basis.shape[0], cell)
        pos, box = lattice(kind, reps, a)
        pos = jitter_and_wrap(pos, box, sigma, rng)
        types = rng.integers(0, ns, size=pos.shape[0]).astype(np.int32)
        masses = np.array([55.845, 63.546, 26.982])[types]
        systems.append(System(pos, types, box, np.ones(3, dtype=np.int32), masses=masses))
    fs = load_feature_scale("batch", 3, 192) if feature_scale else None
    m = random_model(3, 16, 6.0, [128, 128], seed=13, feature_scale=fs,
                     masses=[55.845, 63.546, 26.982])
    return Workload("batch", systems, m, skin=1.0)


def serve(n_systems=256, seed=7, feature_scale=True, n_max=50000):
    """Resident systems for the serving loop: n ~ logU(64, n_max), fcc/bcc,
    1-2 species, sigma 0.1, a ~ U(2.9, 4.1); model 2 species 128-128-1."""
    rng = np.random.default_rng(seed)
    systems = []
    for i in range(n_systems):
        n_t = math.exp(rng.uniform(math.log(64), math.log(n_max)))
        kind = ["fcc", "bcc"][int(rng.integers(0, 2))]
        a = rng.uniform(2.9, 4.1)
        ns = int(rng.integers(1, 3))
        basis, cell = _BASIS[kind]
        reps = _best_reps(n_t, basis.shape[0], cell)
        pos, box = lattice(kind, reps, a)
        pos = jitter_and_wrap(pos, box, 0.1, rng)
        types = rng.integers(0, ns, size=pos.shape[0]).astype(np.int32)
        masses = np.array([55.845, 63.546])[types]
        vel = maxwell_velocities(masses, 300.0, rng)
        systems.append(System(pos, types, box, np.ones(3, dtype=np.int32), vel=vel, masses=masses))
    fs = load_feature_scale("serve", 2, 128) if feature_scale else None
    m = random_model(2, 16, 6.0, [128, 128], seed=14, feature_scale=fs, masses=[55.845, 63.546])
    return Workload("serve", systems, m, skin=1.0)


def cluster(n_atoms, radius, seed, n_species=1):
    """Open-boundary random cluster (pbc off) inside a sphere, min spacing 1.2 A."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n_atoms:
        p = rng.uniform(-radius, radius, size=3)
        if np.linalg.norm(p) > radius:
            continue
        if all(np.linalg.norm(p - q) > 1.2 for q in pts):
            pts.append(p)
    pos = np.array(pts) + radius + 1.0
    box = np.full(3, 2.0 * radius + 2.0)
    types = rng.integers(0, n_species, size=n_atoms).astype(np.int32)
    return System(np.ascontiguousarray(pos), types, box, np.zeros(3, dtype=np.int32))


WORKLOADS = {"tiny": tiny, "medium": medium, "large": large, "batch": batch, "serve": serve}


def embedding_radial_table(S, K, rc, ppa, seed):
    """Radial functions from a small DP-style embedding network, as a table:
    per species pair m(R) = tanh(W2 tanh(W1 R + b1) + b2) (1 -> 8 -> K, seeded
    random weights) times the smooth step (1 - (R/rc)^2)^2, which reaches zero
    with zero slope at rc.  Returns (H, dH) [S][S][n][K] at R_g = g / ppa,
    n = ceil(rc ppa), with the exact derivative."""
    rng = np.random.default_rng(seed)
    n = int(math.ceil(rc * ppa))
    r = np.arange(n) / ppa
    H = np.zeros((S, S, n, K))
    dH = np.zeros_like(H)
    w = np.clip(1.0 - (r / rc) ** 2, 0.0, None)
    sw, dsw = w * w, -4.0 * w * r / (rc * rc)
    for a in range(S):
        for b in range(S):
            W1, b1 = rng.normal(0, 1.0, 8), rng.normal(0, 0.5, 8)
            W2, b2 = rng.normal(0, 0.5, (K, 8)), rng.normal(0, 0.3, K)
            u = np.tanh(np.outer(r, W1) + b1)
            m = np.tanh(u @ W2.T + b2)
            dm = (1 - m * m) * (((1 - u * u) * W1) @ W2.T)
            H[a, b] = sw[:, None] * m
            dH[a, b] = dsw[:, None] * m + sw[:, None] * dm
    return H, dH
