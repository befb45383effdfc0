"""ctypes wrapper of the FP64 CPU oracle (tmd_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the CUDA product path.  It shares no
code with the CUDA library.  The C source is compiled with gcc
(-O2 -ffp-contract=off -fopenmp) into oracle/_build/ on first use.

Every wrapper below names the paper passage its C function follows (TensorMD,
arXiv 2310.08439, Sec. "The Tensor Formalism"):
  moments / moment_grad / tdm      -> Eq. T_dm (moment tensor M_d, multiplicities)
  radial                           -> H_abck = f_k(R) f_c(R); with radial_table > 0
                                      the tabulated H of Sec. "The H_abck tensor
                                      and Batch Rational 1D Interpolation"
  hermite                          -> the interpolation step of that section
                                      (cubic Hermite: a reading, see radial_tab)
  neighbors / neighbors_of         -> the neighbour table R_abc (all images)
  compute / atom_terms             -> Eqs. tensor_formalism, sigma_function,
                                      dP_abkd, U_abck, F1_abcx, F2_abcx, ScatterSum
  vv_first / vv_second             -> velocity-Verlet (Sec. Evaluation, 1 fs steps)
Functions without an independent pin would say "parity unpinned"; none do
(the pins live in tests/test_oracle_pins.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtmd_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-D_GNU_SOURCE", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _CModel(C.Structure):
    _fields_ = [("S", C.c_int32), ("K", C.c_int32), ("L", C.c_int32), ("act", C.c_int32),
                ("rc", C.c_double), ("sp_b", C.c_double),
                ("mu", C.POINTER(C.c_double)), ("eta", C.POINTER(C.c_double)),
                ("widths", C.POINTER(C.c_int32)), ("w", C.POINTER(C.POINTER(C.c_double))),
                ("tab_ppa", C.c_int32), ("tab_n", C.c_int32),
                ("tab_H", C.POINTER(C.c_double)), ("tab_dH", C.POINTER(C.c_double))]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _lp(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _bp(a):
    return a.ctypes.data_as(C.POINTER(C.c_int8))


def lib():
    global _lib
    if _lib is None:
        # TMD_ORACLE_LIB lets the mutation tests load a deliberately broken build
        override = os.environ.get("TMD_ORACLE_LIB")
        _lib = C.CDLL(override if override else build())
        L = _lib
        L.tmdo_neighbors_of.restype = C.c_int64
        L.tmdo_neighbors.restype = C.c_int64
        L.tmdo_atom_terms.restype = C.c_double
        L.tmdo_compute.restype = C.c_int
        L.tmdo_num_threads.restype = C.c_int
    return _lib


class OracleModel:
    """Holds a C view of ``inputs.ModelParams`` (keeps the arrays alive).
    radial_table = 0: H evaluated directly; > 0: H and H' interpolated from a
    table with that many grid points per Angstrom."""

    def __init__(self, params, radial_table=0, table_values=None):
        self.params = params
        self.radial_table = int(radial_table)
        # table_values = (H, dH) [S][S][n][K]: the caller's radial functions at
        # r_g = g / radial_table instead of the Gaussians
        self._tab = None
        if table_values is not None:
            H, dH = (np.ascontiguousarray(a, dtype=np.float64) for a in table_values)
            if H.shape != dH.shape or H.ndim != 4:
                raise ValueError("table values must both be [S][S][n][K]")
            self._tab = (H, dH)
        S, K = params.n_species, params.n_radial
        self._mu = np.ascontiguousarray(params.mu, dtype=np.float64).reshape(S * S * K)
        self._eta = np.ascontiguousarray(params.eta, dtype=np.float64).reshape(S * S * K)
        self._widths = np.ascontiguousarray(params.widths, dtype=np.int32)
        if max([params.n_desc] + list(params.widths)) > 656 or K > 256 or len(params.widths) > 7:
            raise ValueError("oracle limits: widths <= 656, K <= 256, <= 7 hidden layers")
        self._w = [np.ascontiguousarray(w, dtype=np.float64) for w in params.weights]
        self._wptr = (C.POINTER(C.c_double) * S)(*[_dp(w) for w in self._w])
        act = {"tanh": 0, "squareplus": 1}[params.activation]
        self.c = _CModel(S, K, len(params.widths), act, float(params.rc),
                         float(params.squareplus_b), _dp(self._mu), _dp(self._eta),
                         _ip(self._widths), C.cast(self._wptr, C.POINTER(C.POINTER(C.c_double))),
                         self.radial_table, 0 if self._tab is None else self._tab[0].shape[2],
                         None if self._tab is None else _dp(self._tab[0]),
                         None if self._tab is None else _dp(self._tab[1]))

    @property
    def n_desc(self):
        return self.params.n_desc


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


# --------------------------------------------------------------------------
# building blocks (Eq. T_dm; H_abck)
# --------------------------------------------------------------------------
def moments(u):
    u = _f64(u, 3)
    out = np.zeros(20)
    lib().tmdo_moments(_dp(u), _dp(out))
    return out


def moment_grad(u):
    u = _f64(u, 3)
    out = np.zeros((20, 3))
    lib().tmdo_moment_grad(_dp(u), _dp(out))
    return out


def tdm():
    out = np.zeros((20, 4))
    lib().tmdo_tdm(_dp(out))
    return out


def radial(model: OracleModel, ti: int, tj: int, r: float):
    K = model.params.n_radial
    H, dH = np.zeros(K), np.zeros(K)
    lib().tmdo_radial(C.byref(model.c), C.c_int(ti), C.c_int(tj), C.c_double(r), _dp(H), _dp(dH))
    return H, dH


def hermite(y0, d0, y1, d1, h, t):
    """Cubic Hermite interpolant on [x0, x0 + h] at x0 + t h: (y, dy/dx)."""
    y, dy = C.c_double(), C.c_double()
    lib().tmdo_hermite(C.c_double(y0), C.c_double(d0), C.c_double(y1), C.c_double(d1), C.c_double(h),
                       C.c_double(t), C.byref(y), C.byref(dy))
    return y.value, dy.value


# --------------------------------------------------------------------------
# neighbour table
# --------------------------------------------------------------------------
def neighbors(pos, box, pbc, r_list):
    """All (i, j, s) with |x_j + s L - x_i| < r_list; CSR (off, nbr, shift[nnz,3])."""
    pos = _f64(pos)
    n = pos.shape[0]
    box = _f64(box, 3)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    counts = np.zeros(n, dtype=np.int64)
    L = lib()
    L.tmdo_neighbors(C.c_int64(n), _dp(pos), _dp(box), _ip(pbc), C.c_double(r_list),
                     _lp(counts), None, None, None)
    off = np.zeros(n + 1, dtype=np.int64)
    nnz = int(counts.sum())
    nbr = np.zeros(max(nnz, 1), dtype=np.int32)
    shift = np.zeros((max(nnz, 1), 3), dtype=np.int8)
    L.tmdo_neighbors(C.c_int64(n), _dp(pos), _dp(box), _ip(pbc), C.c_double(r_list),
                     _lp(counts), _lp(off), _ip(nbr), _bp(shift))
    return off, nbr[:nnz], shift[:nnz]


def neighbors_of(pos, box, pbc, r_list, i):
    """Neighbour entries (nbr, shift) of one atom, ordered by (j, sx, sy, sz)."""
    pos = _f64(pos)
    n = pos.shape[0]
    box = _f64(box, 3)
    pbc = np.ascontiguousarray(pbc, dtype=np.int32)
    L = lib()
    cnt = L.tmdo_neighbors_of(C.c_int64(n), _dp(pos), _dp(box), _ip(pbc), C.c_double(r_list),
                              C.c_int64(i), C.c_int64(0), None, None)
    nbr = np.zeros(max(cnt, 1), dtype=np.int32)
    shift = np.zeros((max(cnt, 1), 3), dtype=np.int8)
    L.tmdo_neighbors_of(C.c_int64(n), _dp(pos), _dp(box), _ip(pbc), C.c_double(r_list),
                        C.c_int64(i), C.c_int64(cnt), _ip(nbr), _bp(shift))
    return nbr[:cnt], shift[:cnt]


# --------------------------------------------------------------------------
# energy / forces / virial
# --------------------------------------------------------------------------
def compute(model: OracleModel, pos, types, box, nl, want_G=False):
    """E, E_a, F [n,3], W [3,3] (and G, dE/dG [n,Dd]) for a neighbour list ``nl``."""
    off, nbr, shift = nl
    pos = _f64(pos)
    n = pos.shape[0]
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box, 3)
    off = np.ascontiguousarray(off, dtype=np.int64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    shift = np.ascontiguousarray(shift, dtype=np.int8).reshape(-1, 3)
    if nbr.size == 0:
        nbr = np.zeros(1, dtype=np.int32)
        shift = np.zeros((1, 3), dtype=np.int8)
    E = C.c_double(0.0)
    ea = np.zeros(n)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    G = np.zeros((n, model.n_desc)) if want_G else None
    dG = np.zeros((n, model.n_desc)) if want_G else None
    lib().tmdo_compute(C.byref(model.c), C.c_int64(n), _dp(pos), _ip(types), _dp(box), _lp(off),
                       _ip(nbr), _bp(shift), C.byref(E), _dp(ea), _dp(F), _dp(W),
                       _dp(G) if want_G else None, _dp(dG) if want_G else None)
    out = {"energy": E.value, "e_atom": ea, "forces": F, "virial": W.reshape(3, 3)}
    if want_G:
        out["G"] = G
        out["dEdG"] = dG
    return out


def evaluate(model: OracleModel, pos, types, box, pbc, want_G=False):
    """Neighbour list at r_list = rc, then ``compute``."""
    nl = neighbors(pos, box, pbc, model.params.rc)
    return compute(model, pos, types, box, nl, want_G=want_G)


def atom_terms(model: OracleModel, pos, types, box, a, nbr, shift, want_G=False):
    """(E_a, g [deg,3] = dE_a/dD_c, G_a) for one centre atom."""
    pos = _f64(pos)
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box, 3)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    shift = np.ascontiguousarray(shift, dtype=np.int8).reshape(-1, 3)
    deg = nbr.size
    g = np.zeros((max(deg, 1), 3))
    G = np.zeros(model.n_desc)
    Ea = lib().tmdo_atom_terms(C.byref(model.c), _dp(pos), _ip(types), _dp(box), C.c_int64(a),
                               C.c_int64(deg), _ip(nbr if deg else np.zeros(1, np.int32)),
                               _bp(shift if deg else np.zeros((1, 3), np.int8)), _dp(G), _dp(g), None)
    return (Ea, g[:deg], G) if want_G else (Ea, g[:deg])


def sampled(model: OracleModel, pos, types, box, pbc, atoms, r_list=None):
    """E_a and F_a for a sample of atoms of an arbitrarily large system.

    F_i = sum_j g_ij - sum_{a: (a, i, s) listed} g_{a,(i,s)}: the atom's own
    pair gradients plus those of every atom that lists i as a neighbour.  Each
    neighbour search is the O(N) brute-force definition for one atom.
    """
    rc = model.params.rc if r_list is None else r_list
    e_out, f_out = [], []
    cache = {}

    def terms(a):
        if a not in cache:
            nb, sh = neighbors_of(pos, box, pbc, rc, a)
            Ea, g = atom_terms(model, pos, types, box, a, nb, sh)
            cache[a] = (nb, sh, Ea, g)
        return cache[a]

    for i in atoms:
        i = int(i)
        nb, sh, Ea, g = terms(i)
        F = g.sum(axis=0) if len(nb) else np.zeros(3)
        for j in sorted(set(int(x) for x in nb)):
            nbj, shj, _, gj = terms(j)
            mask = nbj == i
            if mask.any():
                F = F - gj[mask].sum(axis=0)
        e_out.append(Ea)
        f_out.append(F)
    return np.array(e_out), np.array(f_out)


# --------------------------------------------------------------------------
# velocity-Verlet
# --------------------------------------------------------------------------
def vv_first(pos, vel, forces, mass, box, pbc, dt):
    """Half kick, drift, wrap (in place)."""
    n = pos.shape[0]
    lib().tmdo_vv_first(C.c_int64(n), _dp(pos), _dp(vel), _dp(_f64(forces)), _dp(_f64(mass)),
                        _dp(_f64(box, 3)), _ip(np.ascontiguousarray(pbc, dtype=np.int32)),
                        C.c_double(dt))


def vv_second(vel, forces, mass, dt):
    n = vel.shape[0]
    lib().tmdo_vv_second(C.c_int64(n), _dp(vel), _dp(_f64(forces)), _dp(_f64(mass)), C.c_double(dt))


def md(model: OracleModel, system, n_steps, dt):
    """Plain NVE velocity-Verlet with a fresh neighbour list every step."""
    pos = system.pos.copy()
    vel = system.vel.copy()
    mass = system.masses
    out = evaluate(model, pos, system.types, system.box, system.pbc)
    for _ in range(n_steps):
        vv_first(pos, vel, out["forces"], mass, system.box, system.pbc, dt)
        out = evaluate(model, pos, system.types, system.box, system.pbc)
        vv_second(vel, out["forces"], mass, dt)
    return pos, vel, out


def num_threads():
    return int(lib().tmdo_num_threads())
