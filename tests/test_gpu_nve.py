"""Energy conservation of the MD loop (velocity-Verlet, Sec. "Evaluation":
1 fs steps, a 1 A buffer, the table rebuilt every 5 steps) on the large
lattice at 32^3 (131,072 atoms) from 300 K: the total energy per atom stays
within 1e-5 eV of its start over 500 steps, for both network forms and for
both table cadences (every 5 steps; only when an atom moved more than
skin/2)."""
import numpy as np
import pytest

from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,rebuild_every", [("fp32", 5), ("fp32", 0), ("bf16", 5)])
def test_nve_energy_is_conserved(tmdlib, precision, rebuild_every):
    w = I.large(reps=32)
    s = w.systems[0]
    m = tmdlib.Model(w.model, precision=precision)
    g = tmdlib.System(s.n, s.box, s.pbc, skin=w.skin)
    g.set_state(s.pos, s.vel, s.types, s.masses)
    th = g.step(m, w.dt_fs, 0)
    e = [(th["e_pot"] + th["e_kin"]) / s.n]
    temps = [th["temperature"]]
    for _ in range(5):
        th = g.step(m, w.dt_fs, 100, rebuild_every=rebuild_every)
        e.append((th["e_pot"] + th["e_kin"]) / s.n)
        temps.append(th["temperature"])
    drift = np.abs(np.array(e) - e[0]).max()
    assert drift < 1e-5, (drift, e)
    assert th["step"] == 500
    if rebuild_every == 5:
        assert th["rebuilds"] >= 100
    else:
        assert 1 <= th["rebuilds"] < 100
    assert max(temps) - min(temps) > 10.0   # the system is moving, not frozen
