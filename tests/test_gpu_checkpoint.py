"""Checkpoint and resume of a resident MD system through the C ABI: the state
read back after k steps (positions, velocities, species, masses), loaded into
a fresh system, continues exactly as the uninterrupted run.  With a
neighbour rebuild every step the two runs see the same tables and every
result is bitwise equal (forces accumulate in fixed point)."""
import numpy as np
import pytest

from paper_2310_08439_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_resume_equals_uninterrupted(tmdlib, precision):
    w = I.medium()
    s = w.systems[0]
    vel = I.maxwell_velocities(s.masses, 300.0, np.random.default_rng(12))
    m = tmdlib.Model(w.model, precision=precision)

    def fresh(pos, v):
        g = tmdlib.System(s.n, s.box, s.pbc, skin=w.skin)
        g.set_state(pos, v, s.types, s.masses)
        return g

    ref = fresh(s.pos, vel)
    th_ref = ref.step(m, w.dt_fs, 8, rebuild_every=1)
    p_ref, v_ref, f_ref = ref.get_state()

    a = fresh(s.pos, vel)
    a.step(m, w.dt_fs, 5, rebuild_every=1)
    p_ck, v_ck, _ = a.get_state()                    # the checkpoint
    del a
    b = fresh(p_ck, v_ck)                            # resume in a new system
    th_b = b.step(m, w.dt_fs, 3, rebuild_every=1)
    p_b, v_b, f_b = b.get_state()
    assert np.array_equal(p_b, p_ref) and np.array_equal(v_b, v_ref) and np.array_equal(f_b, f_ref)
    assert th_b["e_pot"] == th_ref["e_pot"] and th_b["e_kin"] == th_ref["e_kin"]
