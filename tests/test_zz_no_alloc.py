"""tmd_compute_noalloc: the force evaluation for callers that cannot allocate
device memory while they run (codes that hand all GPU memory to their own pool
at start-up, or that must not allocate inside their time-stepping loop).  Its
scratch is one static device array; these checks call it through the C ABI and
compare it with tmd_compute, twice in a row (the array keeps the previous
call's contents, so the second call shows that it is cleared correctly).
"""
import numpy as np
import pytest

from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu

E_TOL, F_TOL, W_TOL = 1e-6, 1e-5, 1e-5


def _torch():
    import torch
    return torch


def _table(tmd, s, r_list):
    """Neighbour table in the caller's format: CSR offsets, ids, (sx, sy, sz, species of j)."""
    torch = _torch()
    nl = tmd.NeighborList()
    pos = torch.as_tensor(s.pos, dtype=torch.float64, device="cuda")
    types = torch.as_tensor(s.types, dtype=torch.int32, device="cuda")
    nl.build(pos, types, s.box, s.pbc, r_list)
    off, nbr, sh = nl.export()
    shift4 = np.zeros((len(nbr), 4), np.int8)
    shift4[:, :3] = sh
    shift4[:, 3] = s.types[nbr]
    dev = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device="cuda")
    return nl, pos, types, dev(off, torch.int64), dev(nbr, torch.int32), dev(shift4, torch.int8)


def _outputs(n):
    torch = _torch()
    return (torch.zeros(1, dtype=torch.float64, device="cuda"), torch.zeros(n, dtype=torch.float32, device="cuda"),
            torch.zeros((n, 3), dtype=torch.float32, device="cuda"), torch.zeros(9, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("wname,precision,force_kernel", [("tiny", "fp32", "auto"), ("medium", "fp32", "auto"),
                                                         ("tiny", "bf16", "auto"), ("medium", "bf16", "auto"),
                                                         ("tiny", "fp32", "tensor"), ("large", "fp32", "auto")])
def test_noalloc_matches_compute_two_calls(tmdlib, wname, precision, force_kernel):
    """Both network forms; with the tensor-core force pass chosen, tmd_compute
    runs it and the allocation-free call runs the SIMT pass (it keeps no pair
    cache), and the two still agree within the FP32 bars."""
    torch = _torch()
    # "large": 2,048 atoms of the 1M-atom cell's lattice and model, whose
    # 64-wide network runs on the resident-weight kernel
    w = I.large(reps=8) if wname == "large" else getattr(I, wname)()
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    if precision == "bf16":
        m.set_precision("bf16")
    nl, pos, types, off, nbr, shift4 = _table(tmdlib, s, w.model.rc + (0.0 if wname == "tiny" else 1.0))
    tmdlib.set_force_kernel(force_kernel)
    try:
        ref = _outputs(s.n)
        tmdlib.compute(m, nl, pos, types, s.box, *ref)
        torch.cuda.synchronize()
        rE, rEa, rF, rW = (t.double().cpu().numpy() for t in ref)
        rms = np.sqrt((rF ** 2).mean())
        for call in range(2):
            out = _outputs(s.n)
            tmdlib.compute_noalloc(m, off, nbr, shift4, pos, types, s.box, *out)
            torch.cuda.synchronize()
            E, Ea, F, W = (t.double().cpu().numpy() for t in out)
            # The caller's table is the exported one, sorted per atom, so the
            # descriptor sums run in another order than tmd_compute's; FP32
            # results agree to rounding, while in the BF16 form a descriptor
            # that rounds to the neighbouring BF16 value moves that atom's
            # energy and forces by a few 1e-3 relative (the BF16 form's own
            # error against the oracle is ~1e-2 of RMS(F)).
            et, ft, wt, at = (E_TOL, F_TOL, W_TOL, 1e-5) if precision == "fp32" else (1e-5, 1e-2, 1e-3, 1e-2)
            assert abs(E[0] - rE[0]) <= et * abs(rE[0]), call
            assert np.abs(F - rF).max() <= ft * rms, call
            assert np.abs(W - rW).max() <= wt * np.abs(rW).max(), call
            assert np.abs(Ea - rEa).max() <= at * np.abs(rEa).max(), call
    finally:
        tmdlib.set_force_kernel("auto")


def test_noalloc_rejects_oversized_and_bad_tables(tmdlib):
    torch = _torch()
    w = I.large(reps=8)  # S = 1, K = 16
    m = tmdlib.Model(w.model)
    n = 40000            # above the static scratch bound for this model
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    types = torch.zeros(n, dtype=torch.int32, device="cuda")
    off = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    nbr = torch.zeros(0, dtype=torch.int32, device="cuda")
    sh = torch.zeros((0, 4), dtype=torch.int8, device="cuda")
    box = [100.0, 100.0, 100.0]
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.compute_noalloc(m, off, nbr, sh, pos, types, box, *_outputs(n))
    assert e.value.status == tmdlib.ERR_CAPACITY
    # a species id in shift4 beyond the model's species count is rejected on the device
    s = w.systems[0]
    nl, pos, types, off, nbr, shift4 = _table(tmdlib, s, 6.0)
    bad = shift4.clone()
    bad[5, 3] = 3
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.compute_noalloc(m, off, nbr, bad, pos, types, s.box, *_outputs(s.n))
    assert e.value.status == tmdlib.ERR_INVALID_ARG
    # and a good table still works afterwards
    out = _outputs(s.n)
    tmdlib.compute_noalloc(m, off, nbr, shift4, pos, types, s.box, *out)
    torch.cuda.synchronize()
    assert np.isfinite(out[0].item())


def test_noalloc_rejects_mismatched_species_and_bad_shapes(tmdlib):
    """A species byte that is a valid species but not that of j is rejected on
    the device (check code 16); tensors of the wrong shape or dtype are
    rejected by the binding before the library reads them."""
    torch = _torch()
    w = I.medium()       # two species
    s = w.systems[0]
    m = tmdlib.Model(w.model)
    nl, pos, types, off, nbr, shift4 = _table(tmdlib, s, w.model.rc)
    bad = shift4.clone()
    bad[7, 3] = 1 - bad[7, 3]
    with pytest.raises(tmdlib.TmdError) as e:
        tmdlib.compute_noalloc(m, off, nbr, bad, pos, types, s.box, *_outputs(s.n))
    assert e.value.status == tmdlib.ERR_INVALID_ARG and "16" in str(e.value)
    for args in [(off[:-1], nbr, shift4), (off, nbr, shift4[:, :3].contiguous()), (off.int(), nbr, shift4)]:
        with pytest.raises(tmdlib.TmdError) as e:
            tmdlib.compute_noalloc(m, *args, pos, types, s.box, *_outputs(s.n))
        assert e.value.status == tmdlib.ERR_INVALID_ARG
    out = _outputs(s.n)
    tmdlib.compute_noalloc(m, off, nbr, shift4, pos, types, s.box, *out)
    torch.cuda.synchronize()
    assert np.isfinite(out[0].item())


def test_noalloc_sparse_gas_matches_compute(tmdlib):
    """A dilute gas (many atoms whose table entries all lie in the skin shell):
    the allocation-free call, which screens the table itself, equals
    tmd_compute within the FP32 bars."""
    torch = _torch()
    w = I.medium()
    s = I.sparse_gas()
    m = tmdlib.Model(w.model)
    nl, pos, types, off, nbr, shift4 = _table(tmdlib, s, w.model.rc + 1.0)
    ref = _outputs(s.n)
    tmdlib.compute(m, nl, pos, types, s.box, *ref)
    out = _outputs(s.n)
    tmdlib.compute_noalloc(m, off, nbr, shift4, pos, types, s.box, *out)
    torch.cuda.synchronize()
    rE, rEa, rF, rW = (t.double().cpu().numpy() for t in ref)
    E, Ea, F, W = (t.double().cpu().numpy() for t in out)
    rms = np.sqrt((rF ** 2).mean())
    assert abs(E[0] - rE[0]) <= E_TOL * abs(rE[0])
    assert np.abs(F - rF).max() <= F_TOL * rms
    assert np.abs(W - rW).max() <= W_TOL * np.abs(rW).max()
