"""Thin ctypes binding of libtmd.so (include/tmd.h).

Argument marshalling only: every step of the energy / force / virial path runs
in the CUDA library.  PyTorch supplies device memory and the current stream.
There is no CPU fallback: if libtmd.so is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmd.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tmd.h")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNIMPLEMENTED = range(7)
ACT = {"tanh": 0, "squareplus": 1}
PREC = {"fp32": 0, "bf16": 1}

_lib = None


class TmdError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(what)


class _Desc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_radial", C.c_int32), ("rc", C.c_double),
                ("mu", C.POINTER(C.c_double)), ("eta", C.POINTER(C.c_double)),
                ("n_hidden", C.c_int32), ("widths", C.POINTER(C.c_int32)),
                ("weights", C.POINTER(C.POINTER(C.c_double))), ("activation", C.c_int32),
                ("squareplus_b", C.c_double), ("precision", C.c_int32)]


class Thermo(C.Structure):
    _fields_ = [("e_pot", C.c_double), ("e_kin", C.c_double), ("temperature", C.c_double),
                ("virial", C.c_double * 9), ("pressure", C.c_double * 9), ("step", C.c_int64),
                ("rebuilds", C.c_int64)]

    def as_dict(self):
        return {"e_pot": self.e_pot, "e_kin": self.e_kin, "temperature": self.temperature,
                "virial": np.array(self.virial[:]).reshape(3, 3),
                "pressure": np.array(self.pressure[:]).reshape(3, 3),
                "step": self.step, "rebuilds": self.rebuilds}


class Tuning(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("pair_blocks_per_sm", C.c_int32), ("ms", C.c_float)]

    def as_dict(self):
        return {"tile_rows": self.tile_rows, "pair_blocks_per_sm": self.pair_blocks_per_sm, "ms": self.ms}


_P = C.c_void_p
_SIGS = {
    "tmd_status_string": (C.c_char_p, [C.c_int]),
    "tmd_last_error": (C.c_char_p, []),
    "tmd_version": (C.c_char_p, []),
    "tmd_model_create": (C.c_int, [C.POINTER(_Desc), C.POINTER(_P)]),
    "tmd_model_destroy": (C.c_int, [_P]),
    "tmd_model_set_precision": (C.c_int, [_P, C.c_int32]),
    "tmd_model_set_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "tmd_model_set_radial_table": (C.c_int, [_P, C.c_int32]),
    "tmd_model_set_radial_table_values": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_double),
                                                    C.POINTER(C.c_double)]),
    "tmd_set_network_kernel": (C.c_int, [C.c_int32]),
    "tmd_set_force_kernel": (C.c_int, [C.c_int32]),
    "tmd_device_status": (C.c_int, [C.POINTER(C.c_int32)]),
    "tmd_selftest_bounded_wait": (C.c_int, [C.POINTER(C.c_int32)]),
    "tmd_model_get_tuning": (C.c_int, [_P, C.POINTER(Tuning)]),
    "tmd_autotune": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_double), C.POINTER(Tuning), _P]),
    "tmd_batch_autotune": (C.c_int, [_P, _P, _P, C.c_int32, C.POINTER(Tuning), _P]),
    "tmd_nlist_create": (C.c_int, [C.POINTER(_P)]),
    "tmd_nlist_destroy": (C.c_int, [_P]),
    "tmd_neighbors": (C.c_int, [_P, _P, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                C.c_double, _P, _P]),
    "tmd_nlist_size": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tmd_nlist_export": (C.c_int, [_P, _P, _P, _P]),
    "tmd_compute": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_double), _P, _P, _P, _P, _P]),
    "tmd_descriptors": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_double), _P, _P, _P]),
    "tmd_compute_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int64, _P, _P, C.c_int64, C.POINTER(C.c_double),
                                      _P, _P, _P, _P, _P]),
    "tmd_evaluate_host": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.POINTER(C.c_double),
                                    C.POINTER(C.c_int32), _P, _P, _P, _P]),
    "tmd_system_create": (C.c_int, [C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.c_double,
                                    C.POINTER(_P)]),
    "tmd_system_destroy": (C.c_int, [_P]),
    "tmd_system_set_state": (C.c_int, [_P, _P, _P, _P, _P, C.c_int32, _P]),
    "tmd_system_get_state": (C.c_int, [_P, _P, _P, _P, C.c_int32, _P]),
    "tmd_step": (C.c_int, [_P, _P, C.c_double, C.c_int32, C.c_int32, C.POINTER(Thermo), _P]),
    "tmd_step_host": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int32, C.c_int32,
                                C.POINTER(Thermo), _P]),
    "tmd_batch_create": (C.c_int, [C.c_int32, _P, _P, _P, C.POINTER(_P)]),
    "tmd_batch_destroy": (C.c_int, [_P]),
    "tmd_batch_set_system": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, _P]),
    "tmd_batch_get_system": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "tmd_batch_compute": (C.c_int, [_P, _P, _P, C.c_int32, _P, _P, _P]),
    "tmd_batch_step": (C.c_int, [_P, _P, _P, C.c_int32, C.c_double, C.c_int32, _P, _P]),
    "tmd_batch_set_skin": (C.c_int, [_P, C.c_double, C.c_int32]),
    "tmd_system_counters": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64)]),
    "tmd_compute_owned": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int64, C.POINTER(C.c_double), _P, _P, _P, _P,
                                    _P]),
    "tmd_batch_release": (C.c_int, [_P, C.c_int32]),
    "tmd_batch_table_info": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                       C.POINTER(C.c_int64)]),
    "tmd_profile_enable": (C.c_int, [C.c_int32]),
    "tmd_profile_read": (C.c_int, [_P, C.c_int32, C.POINTER(C.c_int32), C.c_int32]),
    "tmd_launch_count": (C.c_int64, []),
    "tmd_set_graphs": (C.c_int, [C.c_int32]),
    "tmd_graph_replays": (C.c_int64, []),
}


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double)]


def profile_enable(on=True):
    check(lib().tmd_profile_enable(1 if on else 0))


def profile_read(reset=True):
    """{kernel name: (launches, total device ms)} recorded since the last reset."""
    arr = (KernelStat * 64)()
    n = C.c_int32(0)
    check(lib().tmd_profile_read(C.cast(arr, C.c_void_p), 64, C.byref(n), 1 if reset else 0))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(min(n.value, 64))}


def launch_count():
    return int(lib().tmd_launch_count())


NET = {"auto": 0, "tcgen05": 1, "mma_sync": 2}


def set_network_kernel(kind="auto"):
    """BF16 network kernel: "auto" (tcgen05 when the shapes allow), "tcgen05", "mma_sync"."""
    check(lib().tmd_set_network_kernel(NET[kind]))


FORCE = {"auto": 0, "simt": 1, "tensor": 2}


def set_force_kernel(kind="auto"):
    """Force pass of the unbatched evaluation: "auto", "simt" (FP32 FMAs) or
    "tensor" (per-atom products on TF32 tensor cores with split operands)."""
    check(lib().tmd_set_force_kernel(FORCE[kind]))


def device_status():
    """Raw status bits of the tensor-core kernels since the last call (raises on a timeout)."""
    b = C.c_int32(0)
    check(lib().tmd_device_status(C.byref(b)))
    return int(b.value)


def selftest_bounded_wait():
    """Run the bounded-wait self-test kernel; True when its wait gave up as designed."""
    g = C.c_int32(0)
    check(lib().tmd_selftest_bounded_wait(C.byref(g)))
    return g.value == 1


def set_graphs(on=True):
    """Process-wide switch for the captured CUDA graphs of the MD / batch loops."""
    check(lib().tmd_set_graphs(1 if on else 0))


def graph_replays():
    return int(lib().tmd_graph_replays())


def lib():
    """Load libtmd.so (built by ``paper_2310_08439_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2310_08439_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/tmd.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(tmd_\w+)\s*\(", txt, flags=re.M)))


def check(status):
    if status != OK:
        L = lib()
        raise TmdError(status, f"{L.tmd_status_string(status).decode()}: {L.tmd_last_error().decode()}")


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _box(box):
    return (C.c_double * 3)(*[float(x) for x in box])


def _pbc(pbc):
    return (C.c_int32 * 3)(*[int(x) for x in pbc])


class Model:
    """Device copy of a potential (``inputs.ModelParams``)."""

    def __init__(self, params, precision="fp32"):
        self.params = params
        S, K = params.n_species, params.n_radial
        self._mu = np.ascontiguousarray(params.mu, dtype=np.float64).ravel()
        self._eta = np.ascontiguousarray(params.eta, dtype=np.float64).ravel()
        self._widths = np.ascontiguousarray(params.widths, dtype=np.int32)
        self._w = [np.ascontiguousarray(w, dtype=np.float64) for w in params.weights]
        wp = (C.POINTER(C.c_double) * S)(*[w.ctypes.data_as(C.POINTER(C.c_double)) for w in self._w])
        d = _Desc(S, K, float(params.rc), self._mu.ctypes.data_as(C.POINTER(C.c_double)),
                  self._eta.ctypes.data_as(C.POINTER(C.c_double)), len(params.widths),
                  self._widths.ctypes.data_as(C.POINTER(C.c_int32)),
                  C.cast(wp, C.POINTER(C.POINTER(C.c_double))), ACT[params.activation],
                  float(params.squareplus_b), PREC[precision])
        h = _P()
        check(lib().tmd_model_create(C.byref(d), C.byref(h)))
        self.handle = h
        self.precision = precision
        self.radial_table = 0

    def set_precision(self, precision):
        check(lib().tmd_model_set_precision(self.handle, PREC[precision]))
        self.precision = precision

    def set_radial_table(self, points_per_angstrom):
        """Read H and H' from a table with this many points per Angstrom
        (a power of two in [16, 1024]); 0 returns to direct evaluation."""
        check(lib().tmd_model_set_radial_table(self.handle, int(points_per_angstrom)))
        self.radial_table = int(points_per_angstrom)

    def set_radial_table_values(self, points_per_angstrom, H, dH):
        """Table from the caller's radial functions: H, dH [S][S][n_points][K]
        (float64) at r_g = g / points_per_angstrom."""
        H = np.ascontiguousarray(H, dtype=np.float64)
        dH = np.ascontiguousarray(dH, dtype=np.float64)
        if H.shape != dH.shape or H.ndim != 4:
            raise ValueError("H and dH must both be [S][S][n_points][K]")
        check(lib().tmd_model_set_radial_table_values(self.handle, int(points_per_angstrom), int(H.shape[2]),
                                                      H.ctypes.data_as(C.POINTER(C.c_double)),
                                                      dH.ctypes.data_as(C.POINTER(C.c_double))))
        self.radial_table = int(points_per_angstrom)

    @property
    def tuning(self):
        """Tile shapes in use: {tile_rows, pair_blocks_per_sm} (0 = built-in choice)."""
        t = Tuning()
        check(lib().tmd_model_get_tuning(self.handle, C.byref(t)))
        d = t.as_dict()
        d.pop("ms")
        return d

    @tuning.setter
    def tuning(self, d):
        t = Tuning(int(d.get("tile_rows", 0)), int(d.get("pair_blocks_per_sm", 0)), 0.0)
        check(lib().tmd_model_set_tuning(self.handle, C.byref(t)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tmd_model_destroy(self.handle)
            self.handle = None


class NeighborList:
    """Device neighbour table + compute workspace (opaque tmd_nlist)."""

    def __init__(self):
        h = _P()
        check(lib().tmd_nlist_create(C.byref(h)))
        self.handle = h

    def build(self, pos, types, box, pbc, r_list, stream=None):
        """pos: cuda float64 [n,3]; types: cuda int32 [n]."""
        check(lib().tmd_neighbors(_dptr(pos), _dptr(types), int(pos.shape[0]), _box(box), _pbc(pbc),
                                  float(r_list), self.handle, _stream(stream)))
        return self

    def size(self):
        n, nnz = C.c_int64(0), C.c_int64(0)
        check(lib().tmd_nlist_size(self.handle, C.byref(n), C.byref(nnz)))
        return n.value, nnz.value

    def export(self):
        n, nnz = self.size()
        off = np.zeros(n + 1, dtype=np.int64)
        nbr = np.zeros(max(nnz, 1), dtype=np.int32)
        sh = np.zeros((max(nnz, 1), 3), dtype=np.int8)
        check(lib().tmd_nlist_export(self.handle, off.ctypes.data_as(_P), nbr.ctypes.data_as(_P),
                                     sh.ctypes.data_as(_P)))
        return off, nbr[:nnz], sh[:nnz]

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tmd_nlist_destroy(self.handle)
            self.handle = None


def compute(model, nl, pos, types, box, energy=None, e_atom=None, forces=None, virial=None, stream=None):
    """tmd_compute into caller-provided cuda tensors (any may be None)."""
    check(lib().tmd_compute(model.handle, nl.handle, _dptr(pos), _dptr(types), int(pos.shape[0]), _box(box),
                            _dptr(energy), _dptr(e_atom), _dptr(forces), _dptr(virial), _stream(stream)))


def compute_owned(model, nl, pos, types, n_owned, box, energy=None, e_atom=None, forces=None, virial=None,
                  stream=None):
    """tmd_compute_owned: atoms [0, n_owned) are centres, the rest ghosts."""
    check(lib().tmd_compute_owned(model.handle, nl.handle, _dptr(pos), _dptr(types), int(pos.shape[0]),
                                  int(n_owned), _box(box), _dptr(energy), _dptr(e_atom), _dptr(forces),
                                  _dptr(virial), _stream(stream)))


def autotune(model, nl, pos, types, box, stream=None):
    """Time every candidate tile shape on this system and keep the fastest in the model."""
    t = Tuning()
    check(lib().tmd_autotune(model.handle, nl.handle, _dptr(pos), _dptr(types), int(pos.shape[0]), _box(box),
                             C.byref(t), _stream(stream)))
    return t.as_dict()


def descriptors(model, nl, pos, types, box, stream=None, with_grad=False):
    """G [n, Dd] float32 cuda tensor (tmd_descriptors); with_grad also returns dE/dG."""
    import torch
    G = torch.zeros((pos.shape[0], model.params.n_desc), dtype=torch.float32, device=pos.device)
    dG = torch.zeros_like(G) if with_grad else None
    check(lib().tmd_descriptors(model.handle, nl.handle, _dptr(pos), _dptr(types), int(pos.shape[0]), _box(box),
                                _dptr(G), _dptr(dG), _stream(stream)))
    return (G, dG) if with_grad else G


def evaluate(model, nl, pos, types, box, stream=None):
    """Allocate outputs and run tmd_compute; returns dict of cuda tensors."""
    import torch
    n = pos.shape[0]
    dev = pos.device
    out = {"energy": torch.zeros(1, dtype=torch.float64, device=dev),
           "e_atom": torch.zeros(n, dtype=torch.float32, device=dev),
           "forces": torch.zeros((n, 3), dtype=torch.float32, device=dev),
           "virial": torch.zeros(9, dtype=torch.float64, device=dev)}
    compute(model, nl, pos, types, box, out["energy"], out["e_atom"], out["forces"], out["virial"], stream)
    return out


def compute_noalloc(model, off, nbr, shift4, pos, types, box, energy=None, e_atom=None, forces=None, virial=None,
                    stream=None):
    """tmd_compute_noalloc: cuda tensors off [n+1] int64, nbr [nnz] int32,
    shift4 [nnz, 4] int8 (sx, sy, sz, species of j); outputs as ``compute``.
    Shapes, dtypes and contiguity are checked here, before the library reads
    off[n] or shift4[nnz - 1] on the device."""
    import torch
    n, nnz = int(pos.shape[0]), int(nbr.shape[0])
    want = [(off, (n + 1,), torch.int64, "off"), (nbr, (nnz,), torch.int32, "nbr"),
            (shift4, (nnz, 4), torch.int8, "shift4"), (pos, (n, 3), torch.float64, "pos"),
            (types, (n,), torch.int32, "types")]
    for t, shape, dtype, name in want:
        if tuple(t.shape) != shape or t.dtype != dtype or not t.is_contiguous() or not t.is_cuda:
            raise TmdError(ERR_INVALID_ARG, f"{name}: want a contiguous cuda {dtype} tensor of shape {shape}, "
                                            f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    check(lib().tmd_compute_noalloc(model.handle, _dptr(off), _dptr(nbr), _dptr(shift4), int(nbr.shape[0]),
                                    _dptr(pos), _dptr(types), int(pos.shape[0]), _box(box), _dptr(energy),
                                    _dptr(e_atom), _dptr(forces), _dptr(virial), _stream(stream)))


def evaluate_host(model, nl, pos, types, box, pbc, energy, forces, virial, stream=None):
    """tmd_evaluate_host with host numpy (or pinned torch CPU) buffers."""
    def hp(a):
        if a is None:
            return None
        return C.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(_P)
    check(lib().tmd_evaluate_host(model.handle, nl.handle, hp(pos), hp(types), int(pos.shape[0]), _box(box),
                                  _pbc(pbc), hp(energy), hp(forces), hp(virial), _stream(stream)))


class System:
    """Resident MD state (opaque tmd_system)."""

    def __init__(self, n, box, pbc, skin):
        h = _P()
        check(lib().tmd_system_create(int(n), _box(box), _pbc(pbc), float(skin), C.byref(h)))
        self.handle = h
        self.n = int(n)

    def set_state(self, pos, vel, types, masses, stream=None):
        """Tensors on the GPU (on_device) or numpy arrays (host)."""
        on_dev = hasattr(pos, "is_cuda") and pos.is_cuda

        def p(a):
            if a is None:
                return None
            return C.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(_P)
        check(lib().tmd_system_set_state(self.handle, p(pos), p(vel), p(types), p(masses), int(on_dev),
                                         _stream(stream)))

    def get_state(self, stream=None):
        pos = np.zeros((self.n, 3))
        vel = np.zeros((self.n, 3))
        f = np.zeros((self.n, 3), dtype=np.float32)
        check(lib().tmd_system_get_state(self.handle, pos.ctypes.data_as(_P), vel.ctypes.data_as(_P),
                                         f.ctypes.data_as(_P), 0, _stream(stream)))
        return pos, vel, f

    def counters(self):
        """{steps, rebuilds, runs, reruns} (tmd_system_counters)."""
        v = [C.c_int64() for _ in range(4)]
        check(lib().tmd_system_counters(self.handle, *[C.byref(x) for x in v]))
        return dict(zip(("steps", "rebuilds", "runs", "reruns"), (int(x.value) for x in v)))

    def step(self, model, dt, nsteps, rebuild_every=0, stream=None, thermo=True):
        th = Thermo()
        check(lib().tmd_step(model.handle, self.handle, float(dt), int(nsteps), int(rebuild_every),
                             C.byref(th) if thermo else None, _stream(stream)))
        return th.as_dict() if thermo else None

    def step_host(self, model, pos, vel, forces, dt, nsteps, rebuild_every=0, stream=None):
        def hp(a):
            if a is None:
                return None
            return C.c_void_p(a.data_ptr()) if hasattr(a, "data_ptr") else a.ctypes.data_as(_P)
        th = Thermo()
        check(lib().tmd_step_host(model.handle, self.handle, hp(pos), hp(vel), hp(forces), float(dt),
                                  int(nsteps), int(rebuild_every), C.byref(th), _stream(stream)))
        return th.as_dict()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tmd_system_destroy(self.handle)
            self.handle = None


class Batch:
    """Many resident systems evaluated / advanced together (tmd_batch)."""

    def __init__(self, systems, skin=0.0, rebuild_every=0):
        """systems: list of inputs.System (pos, types, box, pbc, vel, masses);
        skin / rebuild_every: the resident tables' policy (tmd_batch_set_skin)."""
        S = len(systems)
        n = np.array([x.n for x in systems], dtype=np.int64)
        boxes = np.ascontiguousarray(np.array([x.box for x in systems], dtype=np.float64))
        pbc = np.ascontiguousarray(np.array([x.pbc for x in systems], dtype=np.int32))
        h = _P()
        check(lib().tmd_batch_create(S, n.ctypes.data_as(_P), boxes.ctypes.data_as(_P), pbc.ctypes.data_as(_P),
                                     C.byref(h)))
        self.handle = h
        self.n = n
        for k, x in enumerate(systems):
            self.set_system(k, x)
        if skin or rebuild_every:
            self.set_skin(skin, rebuild_every)

    def set_skin(self, skin, rebuild_every=0):
        check(lib().tmd_batch_set_skin(self.handle, float(skin), int(rebuild_every)))

    def release(self, k):
        """Give back system k's resident table (tmd_batch_release)."""
        check(lib().tmd_batch_release(self.handle, int(k)))

    def table_info(self, k):
        """(region entries of system k, pool entries, table builds of k)."""
        r, p, b = C.c_int64(), C.c_int64(), C.c_int64()
        check(lib().tmd_batch_table_info(self.handle, int(k), C.byref(r), C.byref(p), C.byref(b)))
        return int(r.value), int(p.value), int(b.value)

    def set_system(self, k, x, stream=None):
        pos = np.ascontiguousarray(x.pos, dtype=np.float64)
        vel = None if x.vel is None else np.ascontiguousarray(x.vel, dtype=np.float64)
        types = np.ascontiguousarray(x.types, dtype=np.int32)
        masses = np.ascontiguousarray(x.masses if x.masses is not None else np.full(x.n, 55.845), dtype=np.float64)
        check(lib().tmd_batch_set_system(self.handle, int(k), pos.ctypes.data_as(_P),
                                         None if vel is None else vel.ctypes.data_as(_P),
                                         types.ctypes.data_as(_P), masses.ctypes.data_as(_P), _stream(stream)))

    def get_system(self, k, stream=None):
        m = int(self.n[k])
        pos = np.zeros((m, 3)); vel = np.zeros((m, 3)); f = np.zeros((m, 3), dtype=np.float32)
        check(lib().tmd_batch_get_system(self.handle, int(k), pos.ctypes.data_as(_P), vel.ctypes.data_as(_P),
                                         f.ctypes.data_as(_P), _stream(stream)))
        return pos, vel, f

    def compute(self, model, systems, stream=None):
        ids = np.ascontiguousarray(systems, dtype=np.int32)
        e = np.zeros(ids.size); w = np.zeros((ids.size, 9))
        check(lib().tmd_batch_compute(model.handle, self.handle, ids.ctypes.data_as(_P), int(ids.size),
                                      e.ctypes.data_as(_P), w.ctypes.data_as(_P), _stream(stream)))
        return e, w.reshape(-1, 3, 3)

    def step(self, model, systems, dt, nsteps, stream=None):
        ids = np.ascontiguousarray(systems, dtype=np.int32)
        th = (Thermo * max(ids.size, 1))()
        check(lib().tmd_batch_step(model.handle, self.handle, ids.ctypes.data_as(_P), int(ids.size), float(dt),
                                   int(nsteps), C.cast(th, _P), _stream(stream)))
        return [th[k].as_dict() for k in range(ids.size)]

    def autotune(self, model, systems, stream=None):
        """Time every candidate tile shape on these systems and keep the fastest in the model."""
        ids = np.ascontiguousarray(systems, dtype=np.int32)
        t = Tuning()
        check(lib().tmd_batch_autotune(model.handle, self.handle, ids.ctypes.data_as(_P), int(ids.size), C.byref(t),
                                       _stream(stream)))
        return t.as_dict()

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tmd_batch_destroy(self.handle)
            self.handle = None
