"""The oracle's MD loop used by bench.py's reference arm and CPU baseline: with
the table rebuilt every 5 steps (positions left unwrapped in between, the
table's image shifts kept) it follows the same trajectory as with a rebuild
in every step (CPU only)."""
import numpy as np

import bench
from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I


def test_oracle_md_cadence_does_not_change_the_trajectory():
    w, _ = bench.workload("medium")
    s = I.tiny().systems[0]
    s.types = np.zeros(s.n, np.int32)
    s.vel = I.maxwell_velocities(s.masses, 600.0, np.random.default_rng(3))
    w.model = I.tiny().model
    w.skin = 1.0
    a = bench.OracleMD(O, w, s, 5)
    b = bench.OracleMD(O, w, s, 1)
    for _ in range(12):
        a.step()
        b.step()
    box = np.asarray(s.box)
    da = np.mod(a.pos - b.pos + 0.5 * box, box) - 0.5 * box   # same positions up to whole periods
    assert np.abs(da).max() < 1e-9
    assert np.abs(a.vel - b.vel).max() < 1e-9
    assert np.abs(a.forces - b.forces).max() < 1e-8 * max(1.0, np.abs(b.forces).max())
