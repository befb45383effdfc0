"""The pins catch plausible mistakes: each case plants one bug in a private
copy of the oracle's C source (on the CPU), builds it, and checks that the pin
suite then fails.  The committed oracle is never modified."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tmd_oracle.c")

MUTANTS = {
    "tdm_xy_multiplicity": ("{0, 0, 1, 0}, {0, 0, 2, 0}, {0, 0, 2, 0}", "{0, 0, 1, 0}, {0, 0, 1, 0}, {0, 0, 2, 0}"),
    "sigma_no_sqrt": ("(mm == 0) ? sqrt(s) : s", "s"),
    "cutoff_derivative_sign": ("dfc = -0.5 * (M_PI / rc)", "dfc = 0.5 * (M_PI / rc)"),
    "scatter_sign": ("forces[3 * (size_t)j + x] -= g[3 * c + x]", "forces[3 * (size_t)j + x] += g[3 * c + x]"),
    "projection_dropped": ("(dEdu[x] - u[x] * udotg) / R", "dEdu[x] / R"),
    "virial_sign": ("W[al * 3 + be] -= Dv[al]", "W[al * 3 + be] += Dv[al]"),
    "self_pair_kept": ("if (j == i && sx == 0 && sy == 0 && sz == 0) continue;", ""),
    "min_image_floor": ("-(int)rint((pos[3 * j + x]", "-(int)floor((pos[3 * j + x]"),
    "act_derivative_wrong_layer": ("g[c] = gn[c] * act_df(m, z[l - 1][c])", "g[c] = gn[c] * act_df(m, z[l][c])"),
    "rank3_moment_transposed": ("{1, 2, 0}, {1, 1, 1}, {1, 0, 2}", "{1, 1, 1}, {1, 2, 0}, {1, 0, 2}"),
    "hermite_end_slope_sign": ("+ (t3 - t2) * h * d1;", "- (t3 - t2) * h * d1;"),
    "hermite_slope_unscaled": ("(t3 - 2.0 * t2 + t) * h * d0", "(t3 - 2.0 * t2 + t) * d0"),
    "table_wrong_upper_node": ("r1 = (g + 1.0) * h;", "r1 = (g + 2.0) * h;"),
    "table_values_pair_transposed": ("const size_t base = ((size_t)ti * m->S + tj)",
                                     "const size_t base = ((size_t)tj * m->S + ti)"),
}

# Mutants that must be caught by one named pin (not only by a finite-difference
# tolerance somewhere): name -> ([(old, new, occurrences)], pin test).
TARGETED = {
    # SquarePlus with b^2 in place of b, in the value and the derivative alike
    "squareplus_b_squared": ([("m->sp_b", "m->sp_b * m->sp_b", 2)], "test_squareplus_special_values_and_slope"),
    # SquarePlus slope halved at every z (value intact)
    "squareplus_slope_halved": ([("return 0.5 * (1.0 + z / sqrt(z * z + m->sp_b));",
                                  "return 0.25 * (1.0 + z / sqrt(z * z + m->sp_b));", 1)],
                                "test_squareplus_special_values_and_slope"),
    # Gaussian twice as wide, exp(-eta t^2 / 2), with the derivative to match
    "gaussian_width_halved": ([("const double fk = exp(-eta * (r - mu) * (r - mu));",
                                "const double fk = exp(-0.5 * eta * (r - mu) * (r - mu));", 1),
                               ("const double dfk = -2.0 * eta * (r - mu) * fk;",
                                "const double dfk = -eta * (r - mu) * fk;", 1)],
                              "test_radial_gaussian_width_away_from_centre"),
    # pair type b taken from the centre atom instead of the neighbour, in the
    # forward and backward passes alike (still a smooth, invariant potential
    # whose forces are its gradient: only the column placement can tell)
    "pair_type_is_centre_species": ([("const int b = types[j];", "const int b = ti;", 2)],
                                    "test_descriptor_equals_double_sum"),
    # pair types beyond the third folded onto the first ones (a three-species
    # limit left in the indexing): seen only with four or more species
    "pair_type_wraps_at_three": ([("const int b = types[j];", "const int b = types[j] % 3;", 2)],
                                 "test_five_species_pins"),
    # Gaussian centres and widths of pair (neighbour, centre) instead of
    # (centre, neighbour): invisible while the parameters are symmetric
    "radial_params_pair_transposed": ([("((size_t)ti * m->S + tj) * K + k]", "((size_t)tj * m->S + ti) * K + k]", 2)],
                                      "test_radial_parameters_follow_centre_then_neighbour"),
    # the network of species 0 evaluated for every atom (invisible with one
    # species, and still a consistent potential with several)
    "network_of_species_zero": ([("const double *p = m->w[s];", "const double *p = m->w[0];", 1)],
                                "test_centre_species_selects_its_network"),
    # every weight matrix read as [in][out] instead of [out][in], forward and
    # backward alike (again a consistent potential)
    "weights_read_transposed": ([("W[l][(size_t)o * dims[l] + c]", "W[l][(size_t)c * dims[l + 1] + o]", 2)],
                                "test_network_bias_only_and_single_unit"),
}


def _run_pins(edits, tmp_path, select=None):
    src = open(SRC).read()
    for old, new, count in edits:
        assert src.count(old) == count, old
        src = src.replace(old, new)
    mut = tmp_path / "mut.c"
    mut.write_text(src)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                    "-D_GNU_SOURCE", "-o", str(so), str(mut), "-lm"], check=True)
    env = dict(os.environ, TMD_ORACLE_LIB=str(so), OMP_NUM_THREADS="2")
    target = os.path.join(ROOT, "tests", "test_oracle_pins.py")
    if select:
        target += "::" + select
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", target],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_bug(name, tmp_path):
    old, new = MUTANTS[name]
    r = _run_pins([(old, new, 1)], tmp_path)
    assert r.returncode != 0, f"planted bug {name} survived the pins"


@pytest.mark.parametrize("name", sorted(TARGETED))
def test_named_pin_rejects_planted_bug(name, tmp_path):
    edits, pin = TARGETED[name]
    r = _run_pins(edits, tmp_path, select=pin)
    assert r.returncode != 0, f"planted bug {name} survived {pin}"
    assert "1 failed" in r.stdout, r.stdout[-2000:]
