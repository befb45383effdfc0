"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types an oracle formula: each compares the oracle with
an independent fact (the printed T_dm table, the double-sum angular form the
tensor formalism replaces, closed-form 2- and 3-atom descriptors, crystal shell
counts, brute-force image enumeration, invariances, finite differences of the
energy, strain derivatives, velocity-Verlet reversibility).
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_08439_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _small_model(S=1, K=6, rc=4.0, widths=(8, 8), seed=3, activation="tanh"):
    p = I.random_model(S, K, rc, list(widths), seed=seed, activation=activation)
    return p, O.OracleModel(p)


# ---------------------------------------------------------------- T_dm, M_d
def test_tdm_matches_printed_table():
    """Eq. T_dm: the oracle's table equals the one printed in the paper."""
    rows = _read_table("tdm_table.txt")
    T = np.array([[float(x) for x in r[1:]] for r in rows])
    assert np.array_equal(O.tdm(), T)


def test_moment_contraction_identity():
    """sum_d T_dm M_d(u) M_d(v) = (u.v)^m for unit u, v: the identity that turns
    the double angular sum into the squared single sums (Eq.
    double_to_single_simplification, moment_s_formalism).  A wrong monomial,
    a wrong multiplicity or a swapped row fails it."""
    rng = np.random.default_rng(0)
    T = O.tdm()
    for _ in range(50):
        u, v = _unit(rng), _unit(rng)
        Mu, Mv = O.moments(u), O.moments(v)
        c = float(u @ v)
        for m in range(4):
            lhs = float((T[:, m] * Mu * Mv).sum())
            assert abs(lhs - c ** m) < 1e-14


def test_moment_grad_finite_difference():
    rng = np.random.default_rng(1)
    for _ in range(10):
        u = rng.normal(size=3)
        dM = O.moment_grad(u)
        h = 1e-6
        for y in range(3):
            e = np.zeros(3); e[y] = h
            fd = (O.moments(u + e) - O.moments(u - e)) / (2 * h)
            assert np.allclose(dM[:, y], fd, atol=1e-8)


# ---------------------------------------------------------------- H_abck
def test_radial_special_values_and_derivative():
    """h_k = f_k f_c: at r = mu_k the Gaussian is 1 so H = f_c(mu_k); f_c is 1
    at r = 0, 1/2 at rc/2 and 0 beyond rc; dH/dr is the derivative of H."""
    p, m = _small_model(K=5, rc=4.0)
    H0, _ = O.radial(m, 0, 0, 0.0)
    assert H0[0] == 1.0
    Hh, _ = O.radial(m, 0, 0, 2.0)
    k = int(np.argmin(abs(p.mu[0, 0] - 2.0)))
    assert p.mu[0, 0, k] == 2.0 and abs(Hh[k] - 0.5) < 1e-15
    Hc, dHc = O.radial(m, 0, 0, 4.0)
    assert np.all(Hc == 0.0) and np.all(dHc == 0.0)
    for r in [0.3, 1.7, 2.9, 3.999]:
        H, dH = O.radial(m, 0, 0, r)
        hp, _ = O.radial(m, 0, 0, r + 1e-6)
        hm, _ = O.radial(m, 0, 0, r - 1e-6)
        assert np.allclose(dH, (hp - hm) / 2e-6, atol=1e-8)


def test_radial_parameters_follow_centre_then_neighbour():
    """The radial parameters of a pair are those of (centre species, neighbour
    species) (the H_abck subscripts: centre atom a, pair type b).  Two atoms of
    species 0 and 1 at r = rc/2, where f_c = 1/2: channel 0 of pair (0, 1) is
    centred on r and channel 0 of pair (1, 0) one width away, so the rank-0
    descriptor of atom 0 reads 1/2 and that of atom 1 reads e^-1/2 in the
    column of the other species, and both read 0 in their own species' one."""
    p, _ = _small_model(S=2, K=4, rc=5.0, widths=(4,))
    r = 2.5
    p.mu[0, 1, 0], p.eta[0, 1, 0] = r, 1.0
    p.mu[1, 0, 0], p.eta[1, 0, 0] = r + 1.0, 1.0
    om = O.OracleModel(p)
    pos = np.array([[10.0, 10.0, 10.0], [10.0, 10.0 + r, 10.0]])
    G = O.evaluate(om, pos, np.array([0, 1], np.int32), np.full(3, 40.0), np.zeros(3, np.int32),
                   want_G=True)["G"].reshape(2, 2, 4, 4)   # [atom][b][k][m]
    assert abs(G[0, 1, 0, 0] - 0.5) < 1e-15
    assert abs(G[1, 0, 0, 0] - 0.5 * math.exp(-1.0)) < 1e-15
    assert np.all(G[0, 0] == 0.0) and np.all(G[1, 1] == 0.0)


def test_radial_gaussian_width_away_from_centre():
    """The width of f_k = exp(-eta (r - mu)^2) (reading c2), checked away from
    the centres, where H = 1 at mu cannot see it:
    - two channels at the same r share f_c, so ln(H_k / H_l) equals
      -eta_k (r - mu_k)^2 + eta_l (r - mu_l)^2 for arbitrary centres and widths;
    - one standard deviation out, r = mu_k + 1/sqrt(2 eta_k), the Gaussian is
      e^(-1/2), and f_c there is the closed form (cos(pi r / rc) + 1) / 2;
    - with the default spacing (eta = 1/(2 delta^2)) neighbouring channels
      cross half way between their centres at e^(-1/8) f_c, and at mu_k the
      next channel has fallen to e^(-1/2) of channel k."""
    rc = 4.0
    p, m = _small_model(K=5, rc=rc)
    fc = lambda r: 0.5 * (math.cos(math.pi * r / rc) + 1.0)
    delta = p.mu[0, 0, 1] - p.mu[0, 0, 0]
    for k in range(4):
        mid = 0.5 * (p.mu[0, 0, k] + p.mu[0, 0, k + 1])
        H, _ = O.radial(m, 0, 0, mid)
        assert abs(H[k] - math.exp(-0.125) * fc(mid)) < 1e-14
        assert abs(H[k + 1] - math.exp(-0.125) * fc(mid)) < 1e-14
        H, _ = O.radial(m, 0, 0, p.mu[0, 0, k])
        assert abs(H[k + 1] / H[k] - math.exp(-0.5)) < 1e-14
    assert abs(delta - rc / 4) < 1e-15
    rng = np.random.default_rng(11)
    p.mu[:] = rng.uniform(0.0, rc, size=p.mu.shape)
    p.eta[:] = rng.uniform(0.3, 3.0, size=p.eta.shape)
    m = O.OracleModel(p)
    for k in range(5):
        eta, mu = p.eta[0, 0, k], p.mu[0, 0, k]
        r = mu + 1.0 / math.sqrt(2.0 * eta)
        if r < rc:
            H, _ = O.radial(m, 0, 0, r)
            assert abs(H[k] - math.exp(-0.5) * fc(r)) < 1e-14
    for r in rng.uniform(0.2, rc - 0.2, size=20):
        H, _ = O.radial(m, 0, 0, r)
        for k in range(5):
            for l in range(5):
                want = -p.eta[0, 0, k] * (r - p.mu[0, 0, k]) ** 2 + p.eta[0, 0, l] * (r - p.mu[0, 0, l]) ** 2
                assert abs(math.log(H[k] / H[l]) - want) < 1e-11


# ---------------------------------------------------------------- tabulated H
def test_hermite_reproduces_cubics_and_quartic_error():
    """Cubic Hermite interpolation from end values and slopes reproduces every
    cubic (value and slope) on the interval; for x^4 on [0, 1] its error is the
    closed form t^2 (t - 1)^2 (the remainder f^(4)/4! (x - x0)^2 (x - x1)^2)."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        p = np.polynomial.Polynomial(rng.normal(size=4))
        dp = p.deriv()
        x0, h = rng.uniform(-2.0, 2.0), rng.uniform(0.01, 1.0)
        for t in (0.0, 0.13, 0.5, 0.77, 1.0):
            y, dy = O.hermite(p(x0), dp(x0), p(x0 + h), dp(x0 + h), h, t)
            x = x0 + t * h
            assert abs(y - p(x)) <= 1e-12 * (1.0 + abs(p(x)))
            assert abs(dy - dp(x)) <= 1e-10 * (1.0 + abs(dp(x)))
    for t in (0.1, 0.5, 0.8):
        y, dy = O.hermite(0.0, 0.0, 1.0, 4.0, 1.0, t)
        assert abs((t ** 4 - y) - t * t * (t - 1.0) ** 2) < 1e-14
        assert abs((4 * t ** 3 - dy) - (2 * t * (t - 1.0) ** 2 + 2 * t * t * (t - 1.0))) < 1e-14


def test_radial_table_nodes_order_and_cutoff():
    """Tabulated H (Sec. "The H_abck tensor and Batch Rational 1D
    Interpolation"): equal to the direct H and H' at every grid point, zero
    from rc on, and converging to the direct values as h^4 (H) and h^3 (H')
    when the spacing h = 1/ppa halves."""
    w = I.medium()
    direct = O.OracleModel(w.model)
    rc = w.model.rc
    for ppa in (16, 64):
        tab = O.OracleModel(w.model, radial_table=ppa)
        for g in (7, 40, int(rc * ppa) - 1):
            r = g / ppa
            Ht, dHt = O.radial(tab, 0, 1, r)
            Hd, dHd = O.radial(direct, 0, 1, r)
            assert np.allclose(Ht, Hd, rtol=0, atol=1e-15) and np.allclose(dHt, dHd, rtol=0, atol=1e-14)
        for r in (rc, rc + 0.3):
            Ht, dHt = O.radial(tab, 1, 0, r)
            assert np.all(Ht == 0.0) and np.all(dHt == 0.0)
        Ht, _ = O.radial(tab, 1, 0, rc - 1e-9)
        assert np.abs(Ht).max() < 1e-12
    rs = np.linspace(0.8, rc - 1e-3, 1201)
    ref = [O.radial(direct, 1, 1, r) for r in rs]
    errs = []
    for ppa in (32, 64, 128):
        tab = O.OracleModel(w.model, radial_table=ppa)
        eH = eD = 0.0
        for r, (Hd, dHd) in zip(rs, ref):
            Ht, dHt = O.radial(tab, 1, 1, r)
            eH, eD = max(eH, np.abs(Ht - Hd).max()), max(eD, np.abs(dHt - dHd).max())
        errs.append((eH, eD))
    for (h1, d1), (h2, d2) in zip(errs, errs[1:]):
        assert 12.0 < h1 / h2 < 20.0 and 6.0 < d1 / d2 < 10.0, errs


def test_tabulated_forces_are_negative_energy_gradient():
    """With the tabulated H the slope used for forces is the derivative of the
    interpolant itself, so the forces stay the exact gradient of the
    (interpolated) energy."""
    p = I.random_model(2, 6, 4.5, [12, 10], seed=3)
    om = O.OracleModel(p, radial_table=32)
    c = I.cluster(16, 3.6, seed=5, n_species=2)
    F = O.evaluate(om, c.pos, c.types, c.box, c.pbc)["forces"]
    rng = np.random.default_rng(2)
    for _ in range(8):
        i, x = int(rng.integers(c.n)), int(rng.integers(3))
        fd = _fd_force(om, c.pos, c.types, c.box, c.pbc, i, x)
        assert abs(fd - F[i, x]) <= 1e-7 * max(1.0, abs(F[i, x])) + 1e-8


def test_table_values_match_the_gaussian_table_and_forces_are_gradients():
    """Given the Gaussians' own values at the grid points, the table built from
    caller values equals the Gaussian table (species pairs and channels kept
    apart); with an embedding-network radial basis the forces are -grad E."""
    p = I.random_model(2, 6, 4.5, [12, 10], seed=3)
    p.mu = p.mu + 0.05 * np.arange(4).reshape(2, 2, 1)
    p.eta = p.eta * (1.0 + 0.1 * np.arange(4).reshape(2, 2, 1))
    ppa = 32
    n = int(math.ceil(4.5 * ppa))
    direct = O.OracleModel(p)
    H = np.zeros((2, 2, n, 6))
    dH = np.zeros_like(H)
    for a in range(2):
        for b in range(2):
            for g in range(n):
                H[a, b, g], dH[a, b, g] = O.radial(direct, a, b, g / ppa)
    gauss = O.OracleModel(p, radial_table=ppa)
    given = O.OracleModel(p, radial_table=ppa, table_values=(H, dH))
    for r in (0.9, 1.7, 3.33, 4.49):
        for a, b in ((0, 1), (1, 0), (1, 1)):
            x, y = O.radial(gauss, a, b, r), O.radial(given, a, b, r)
            assert np.array_equal(x[0], y[0]) and np.array_equal(x[1], y[1])
    He, dHe = I.embedding_radial_table(2, 6, 4.5, ppa, seed=8)
    om = O.OracleModel(p, radial_table=ppa, table_values=(He, dHe))
    c = I.cluster(16, 3.6, seed=5, n_species=2)
    F = O.evaluate(om, c.pos, c.types, c.box, c.pbc)["forces"]
    rng = np.random.default_rng(3)
    for _ in range(8):
        i, x = int(rng.integers(c.n)), int(rng.integers(3))
        fd = _fd_force(om, c.pos, c.types, c.box, c.pbc, i, x)
        assert abs(fd - F[i, x]) <= 1e-7 * max(1.0, abs(F[i, x])) + 1e-8


# ---------------------------------------------------------------- neighbours
def _brute_pairs(pos, box, pbc, r):
    """Independent image enumeration: every s in a generous cube."""
    n = len(pos)
    R = [int(math.ceil(r / box[x])) + 2 if pbc[x] else 0 for x in range(3)]
    out = set()
    for i in range(n):
        for j in range(n):
            for sx in range(-R[0], R[0] + 1):
                for sy in range(-R[1], R[1] + 1):
                    for sz in range(-R[2], R[2] + 1):
                        if i == j and sx == sy == sz == 0:
                            continue
                        d = pos[j] + np.array([sx, sy, sz]) * box - pos[i]
                        if float(d @ d) < r * r:
                            out.add((i, j, sx, sy, sz))
    return out


def _as_set(nl):
    off, nbr, sh = nl
    s = set()
    for i in range(len(off) - 1):
        for c in range(off[i], off[i + 1]):
            s.add((i, int(nbr[c]), int(sh[c, 0]), int(sh[c, 1]), int(sh[c, 2])))
    return s


@pytest.mark.parametrize("L,r", [(7.22, 5.0), (4.0, 5.0), (11.0, 5.0), (3.0, 6.5)])
def test_neighbors_vs_brute_force_images(L, r):
    rng = np.random.default_rng(7)
    pos = rng.uniform(0, L, size=(6, 3))
    box = np.array([L, L * 1.1, L * 0.9])
    pos = np.mod(pos, box)
    pbc = np.array([1, 1, 1])
    nl = O.neighbors(pos, box, pbc, r)
    assert _as_set(nl) == _brute_pairs(pos, box, pbc, r)


def test_neighbors_open_and_mixed_boundaries():
    rng = np.random.default_rng(8)
    box = np.array([6.0, 7.0, 8.0])
    pos = rng.uniform(0, 1, size=(7, 3)) * box
    for pbc in ([0, 0, 0], [1, 0, 1]):
        nl = O.neighbors(pos, box, np.array(pbc), 4.5)
        assert _as_set(nl) == _brute_pairs(pos, box, pbc, 4.5)


def test_neighbors_symmetric_and_ordered():
    w = I.tiny()
    s = w.systems[0]
    nl = O.neighbors(s.pos, s.box, s.pbc, 5.0)
    st = _as_set(nl)
    assert all((j, i, -a, -b, -c) in st for (i, j, a, b, c) in st)
    off, nbr, sh = nl
    for i in range(s.n):
        keys = [(int(nbr[c]), *map(int, sh[c])) for c in range(off[i], off[i + 1])]
        assert keys == sorted(keys)


def test_fcc_shell_counts():
    for a, rc, cnt in _read_table("fcc_shell_counts.txt"):
        a, rc, cnt = float(a), float(rc), int(cnt)
        pos, box = I.lattice("fcc", (4, 4, 4), a)
        off, nbr, sh = O.neighbors(pos, box, np.ones(3, np.int32), rc)
        assert np.all(np.diff(off) == cnt)


def test_neighbors_relabel_invariant():
    w = I.tiny()
    s = w.systems[0]
    perm = np.random.default_rng(3).permutation(s.n)
    inv = np.argsort(perm)
    a = _as_set(O.neighbors(s.pos, s.box, s.pbc, 5.0))
    b = _as_set(O.neighbors(s.pos[perm], s.box, s.pbc, 5.0))
    b = {(int(perm[i]), int(perm[j]), x, y, z) for (i, j, x, y, z) in b}
    assert a == b and inv is not None


# ---------------------------------------------------------------- descriptors
def _double_sum_G(model_params, om, pos, types, box, pbc, a):
    """BP/MEAM angular double sum (Eq. general_atomic_descriptor_functions with
    P_m = cos^m, diagonal j = l included):  G_bkm = sum_{j,l in b} h_k(r_j)
    h_k(r_l) (u_j.u_l)^m for m >= 1 and sum_j h_k(r_j) for m = 0."""
    S, K = model_params.n_species, model_params.n_radial
    nb, sh = O.neighbors_of(pos, box, pbc, model_params.rc, a)
    G = np.zeros((S, K, 4))
    by_b = {b: [] for b in range(S)}
    for j, s in zip(nb, sh):
        d = pos[j] + s * box - pos[a]
        r = np.linalg.norm(d)
        H, _ = O.radial(om, int(types[a]), int(types[j]), r)
        by_b[int(types[j])].append((H, d / r))
    for b in range(S):
        for (Hj, uj) in by_b[b]:
            G[b, :, 0] += Hj
            for (Hl, ul) in by_b[b]:
                c = float(uj @ ul)
                for m in range(1, 4):
                    G[b, :, m] += Hj * Hl * c ** m
    return G.reshape(-1)


def test_descriptor_equals_double_sum():
    """Tensor form (Eq. tensor_formalism) == the angular double sum it replaces."""
    p, om = _small_model(S=2, K=5, rc=4.5)
    c = I.cluster(14, 3.5, seed=4, n_species=2)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc, want_G=True)
    for a in range(c.n):
        ref = _double_sum_G(p, om, c.pos, c.types, c.box, c.pbc, a)
        assert np.allclose(out["G"][a], ref, rtol=1e-12, atol=1e-14)
    # and on a periodic cell with self images (L < 2 rc)
    w = I.tiny(feature_scale=False)
    s = w.systems[0]
    om2 = O.OracleModel(w.model)
    out = O.evaluate(om2, s.pos, s.types, s.box, s.pbc, want_G=True)
    for a in [0, 5, 31]:
        ref = _double_sum_G(w.model, om2, s.pos, s.types, s.box, s.pbc, a)
        assert np.allclose(out["G"][a], ref, rtol=1e-12, atol=1e-14)


def test_two_and_three_atom_closed_forms():
    """2 atoms at r: G_k0 = h_k(r), G_km = h_k(r)^2.  3 atoms (neighbours at r1,
    r2, angle theta): G_k0 = h1 + h2, G_km = h1^2 + h2^2 + 2 h1 h2 cos^m theta."""
    p, om = _small_model(K=4, rc=5.0)
    box = np.array([50.0, 50.0, 50.0])
    pbc = np.zeros(3, np.int32)
    pos = np.array([[10.0, 10.0, 10.0], [12.3, 10.0, 10.0]])
    G = O.evaluate(om, pos, np.zeros(2, np.int32), box, pbc, want_G=True)["G"].reshape(2, -1, 4)
    h, _ = O.radial(om, 0, 0, 2.3)
    assert np.allclose(G[0, :, 0], h, rtol=1e-14)
    for m in (1, 2, 3):
        assert np.allclose(G[0, :, m], h * h, rtol=1e-13)
    r1, r2, th = 2.1, 3.3, 1.1
    pos = np.array([[10.0, 10.0, 10.0], [10.0 + r1, 10.0, 10.0],
                    [10.0 + r2 * math.cos(th), 10.0 + r2 * math.sin(th), 10.0]])
    G = O.evaluate(om, pos, np.zeros(3, np.int32), box, pbc, want_G=True)["G"].reshape(3, -1, 4)
    h1, _ = O.radial(om, 0, 0, r1)
    h2, _ = O.radial(om, 0, 0, r2)
    assert np.allclose(G[0, :, 0], h1 + h2, rtol=1e-13)
    for m in (1, 2, 3):
        assert np.allclose(G[0, :, m], h1 ** 2 + h2 ** 2 + 2 * h1 * h2 * math.cos(th) ** m,
                           rtol=1e-12)


def test_radial_only_limit():
    """Eq. G_radial_tensor_form: the m = 0 column is G_abk = sum_c H_abck."""
    w = I.tiny(feature_scale=False)
    s = w.systems[0]
    om = O.OracleModel(w.model)
    out = O.evaluate(om, s.pos, s.types, s.box, s.pbc, want_G=True)
    for a in [0, 11]:
        nb, sh = O.neighbors_of(s.pos, s.box, s.pbc, 5.0, a)
        acc = np.zeros(8)
        for j, t in zip(nb, sh):
            acc += O.radial(om, 0, 0, np.linalg.norm(s.pos[j] + t * s.box - s.pos[a]))[0]
        assert np.allclose(out["G"][a].reshape(8, 4)[:, 0], acc, rtol=1e-13)


# ---------------------------------------------------------------- network
def test_network_bias_only_and_single_unit():
    """All weights zero except the output bias: E = N b, F = 0.  One hidden unit
    fed by one descriptor column: E_a = w2 tanh(w1 G_c) + b (closed form)."""
    p, om = _small_model(K=4, rc=4.5, widths=(3,))
    for s in range(p.n_species):
        p.weights[s][:] = 0.0
        p.weights[s][-1] = -2.5
    om = O.OracleModel(p)
    c = I.cluster(8, 3.0, seed=2)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc, want_G=True)
    assert abs(out["energy"] - (-2.5 * c.n)) < 1e-12
    assert np.all(out["forces"] == 0.0)
    Dd = p.n_desc
    col = 4 * 2 + 2
    w = p.weights[0]
    w[:] = 0.0
    w[0 * Dd + col] = 0.7                # W1[0, col]
    w[3 * Dd + 3 + 0] = 1.3              # W2[0, 0] (after W1 [3xDd], b1 [3])
    w[-1] = 0.25
    om = O.OracleModel(p)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc, want_G=True)
    ref = 1.3 * np.tanh(0.7 * out["G"][:, col]) + 0.25
    assert np.allclose(out["e_atom"], ref, rtol=1e-14, atol=1e-15)


def test_centre_species_selects_its_network():
    """E_a = NNP_{species of a}(G_a): with every weight zero but the output
    biases (-1 for species 0, -3 for species 1), each atom's energy is the
    bias of its own species' network; then a one-unit first layer in species
    1 alone changes the energies of species-1 atoms only."""
    p, _ = _small_model(S=2, K=4, rc=4.5, widths=(3,))
    for s, b in enumerate((-1.0, -3.0)):
        p.weights[s][:] = 0.0
        p.weights[s][-1] = b
    c = I.cluster(12, 3.2, seed=6, n_species=2)
    assert set(c.types.tolist()) == {0, 1}
    out = O.evaluate(O.OracleModel(p), c.pos, c.types, c.box, c.pbc, want_G=True)
    assert np.array_equal(out["e_atom"], np.where(c.types == 0, -1.0, -3.0))
    Dd = p.n_desc
    p.weights[1][0 * Dd + 1] = 0.9        # W1[0, column 1] of species 1
    p.weights[1][3 * Dd + 3 + 0] = 2.0    # W2[0, 0] of species 1
    out = O.evaluate(O.OracleModel(p), c.pos, c.types, c.box, c.pbc, want_G=True)
    want = np.where(c.types == 0, -1.0, 2.0 * np.tanh(0.9 * out["G"][:, 1]) - 3.0)
    assert np.allclose(out["e_atom"], want, rtol=1e-14, atol=1e-15)


def test_squareplus_special_values_and_slope():
    """SquarePlus (Barron's smooth ReLU, the activation of the paper's
    potentials in Sec. "Evaluation") through a one-unit network whose hidden
    input is fixed by its bias (E_a = sp(z0)):
    - sp(0) = sqrt(b)/2;
    - sp(z) - z -> b / (4 z) for z >> sqrt(b) (so sp(z) -> z);
    - sp(-z) -> b / (4 z) for z >> sqrt(b) (so sp -> 0 on the left).
    The slope at 0 is 1/2: with a tiny first-layer weight eps on one column
    (z = eps G), every force of the SquarePlus network is half the force of
    the same network with tanh (slope 1 at 0), up to O(eps)."""
    for b in (4.0, 2.5):
        p, _ = _small_model(K=4, rc=4.5, widths=(1,), activation="squareplus")
        p.squareplus_b = b
        c = I.cluster(6, 2.5, seed=4)
        Dd = p.n_desc
        for z0, want, tol in [(0.0, 0.5 * math.sqrt(b), 1e-15),
                              (1e4, 1e4 + b / 4e4, 1e-10),
                              (-1e4, b / 4e4, 1e-10)]:
            w = p.weights[0]
            w[:] = 0.0
            w[Dd] = z0            # b1[0] (after W1 [1 x Dd])
            w[Dd + 1] = 1.0       # W2[0, 0]
            out = O.evaluate(O.OracleModel(p), c.pos, c.types, c.box, c.pbc)
            assert np.all(np.abs(out["e_atom"] - want) < tol), (b, z0)
    eps = 1e-7
    col = 4 * 1 + 0                       # channel 1, rank 0
    Dd = 4 * 4
    F = {}
    for act in ("squareplus", "tanh"):
        p, _ = _small_model(K=4, rc=4.5, widths=(1,), activation=act)
        w = p.weights[0]
        w[:] = 0.0
        w[col] = eps              # W1[0, col]
        w[Dd + 1] = 1.0           # W2[0, 0]
        c = I.cluster(10, 3.0, seed=6)
        F[act] = O.evaluate(O.OracleModel(p), c.pos, c.types, c.box, c.pbc)["forces"]
    assert np.abs(F["tanh"]).max() > 0
    assert np.allclose(F["squareplus"], 0.5 * F["tanh"], rtol=1e-5, atol=1e-6 * np.abs(F["tanh"]).max())


# ---------------------------------------------------------------- forces
def _fd_force(om, pos, types, box, pbc, i, x, h=1e-5):
    pp, pm = pos.copy(), pos.copy()
    pp[i, x] += h
    pm[i, x] -= h
    ep = O.evaluate(om, pp, types, box, pbc)["energy"]
    em = O.evaluate(om, pm, types, box, pbc)["energy"]
    return -(ep - em) / (2 * h)


@pytest.mark.parametrize("act", ["tanh", "squareplus"])
def test_forces_are_negative_energy_gradient(act):
    p, om = _small_model(S=2, K=6, rc=4.5, widths=(12, 10), activation=act)
    c = I.cluster(16, 3.6, seed=5, n_species=2)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc)
    F = out["forces"]
    rng = np.random.default_rng(0)
    for _ in range(12):
        i, x = int(rng.integers(c.n)), int(rng.integers(3))
        fd = _fd_force(om, c.pos, c.types, c.box, c.pbc, i, x)
        assert abs(fd - F[i, x]) <= 1e-7 * max(1.0, abs(F[i, x])) + 1e-8
    assert np.abs(F.sum(axis=0)).max() < 1e-12 * c.n * max(1.0, np.sqrt((F ** 2).mean()))


def test_forces_fd_periodic_self_images():
    w = I.tiny()
    s = w.systems[0]
    om = O.OracleModel(w.model)
    F = O.evaluate(om, s.pos, s.types, s.box, s.pbc)["forces"]
    rng = np.random.default_rng(1)
    for _ in range(8):
        i, x = int(rng.integers(s.n)), int(rng.integers(3))
        fd = _fd_force(om, s.pos, s.types, s.box, s.pbc, i, x)
        assert abs(fd - F[i, x]) <= 1e-7 * max(1.0, abs(F[i, x]))


def test_virial_is_strain_derivative():
    """W_ab = -dE/d eps_ab under x -> (I + eps) x, L -> (I + eps) L."""
    w = I.tiny()
    s = w.systems[0]
    om = O.OracleModel(w.model)
    W = O.evaluate(om, s.pos, s.types, s.box, s.pbc)["virial"]
    assert np.allclose(W, W.T, atol=1e-10 * abs(W).max())
    h = 1e-6
    for (a, b) in [(0, 0), (1, 1), (2, 2)]:
        es = []
        for sgn in (1, -1):
            eps = np.eye(3)
            eps[a, b] += sgn * h
            pos = s.pos @ eps.T
            box = s.box * np.diag(eps)
            es.append(O.evaluate(om, pos, s.types, box, s.pbc)["energy"])
        fd = -(es[0] - es[1]) / (2 * h)
        assert abs(fd - W[a, b]) <= 1e-7 * abs(W).max()
    # shear: an open cluster has no box constraint, so any (I + eps) applies
    c = I.cluster(12, 3.4, seed=9)
    p, om = _small_model(K=5, rc=4.5)
    W = O.evaluate(om, c.pos, c.types, c.box, c.pbc)["virial"]
    for (a, b) in [(0, 1), (1, 2), (2, 0), (1, 0)]:
        es = []
        for sgn in (1, -1):
            eps = np.eye(3)
            eps[a, b] += sgn * h
            es.append(O.evaluate(om, c.pos @ eps.T, c.types, c.box, c.pbc)["energy"])
        fd = -(es[0] - es[1]) / (2 * h)
        assert abs(fd - W[a, b]) <= 1e-7 * max(1.0, abs(W).max())


# ---------------------------------------------------------------- invariances
def _rot(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_rotation_invariance_cluster():
    p, om = _small_model(S=2, K=6, rc=4.5)
    c = I.cluster(15, 3.6, seed=6, n_species=2)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc)
    Rm = _rot(np.random.default_rng(2))
    ctr = c.pos.mean(axis=0)
    pos2 = (c.pos - ctr) @ Rm.T + ctr
    out2 = O.evaluate(om, pos2, c.types, c.box, c.pbc)
    assert abs(out2["energy"] - out["energy"]) < 1e-12 * abs(out["energy"])
    assert np.allclose(out2["forces"], out["forces"] @ Rm.T, atol=1e-11)
    assert np.allclose(out2["virial"], Rm @ out["virial"] @ Rm.T, atol=1e-10)


def test_translation_and_cubic_symmetry_periodic():
    w = I.tiny()
    s = w.systems[0]
    om = O.OracleModel(w.model)
    out = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
    pos_t = np.mod(s.pos + np.array([1.3, -2.2, 0.7]), s.box)
    out_t = O.evaluate(om, pos_t, s.types, s.box, s.pbc)
    assert abs(out_t["energy"] - out["energy"]) < 1e-12 * abs(out["energy"])
    assert np.allclose(out_t["forces"], out["forces"], atol=1e-11)
    # cubic cell: axis permutation (x, y, z) -> (y, z, x) is a symmetry of the box
    P = np.array([[0, 1, 0], [0, 0, 1], [1, 0, 0]], dtype=float)
    out_p = O.evaluate(om, s.pos @ P.T, s.types, s.box, s.pbc)
    assert abs(out_p["energy"] - out["energy"]) < 1e-12 * abs(out["energy"])
    assert np.allclose(out_p["forces"], out["forces"] @ P.T, atol=1e-11)


def test_permutation_invariance():
    w = I.medium()
    p = w.model
    om = O.OracleModel(p)
    c = I.cluster(18, 4.0, seed=10, n_species=2)
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc)
    perm = np.random.default_rng(4).permutation(c.n)
    out2 = O.evaluate(om, c.pos[perm], c.types[perm], c.box, c.pbc)
    assert abs(out2["energy"] - out["energy"]) < 1e-12 * abs(out["energy"])
    assert np.allclose(out2["e_atom"], out["e_atom"][perm], atol=1e-12)
    assert np.allclose(out2["forces"], out["forces"][perm], atol=1e-11)


def test_energy_is_sum_of_atomic_energies_and_cutoff_continuity():
    p, om = _small_model(K=5, rc=4.0)
    box = np.array([40.0, 40.0, 40.0])
    pbc = np.zeros(3, np.int32)
    es = []
    for r in [4.0 - 1e-6, 4.0, 4.0 + 1e-6]:
        pos = np.array([[10.0, 10, 10], [10.0 + r, 10, 10], [10.0, 12.0, 10.0]])
        out = O.evaluate(om, pos, np.zeros(3, np.int32), box, pbc)
        assert abs(out["energy"] - out["e_atom"].sum()) < 1e-13
        es.append(out["energy"])
    assert abs(es[0] - es[1]) < 1e-9 and abs(es[1] - es[2]) < 1e-9


def test_sampled_forces_match_full_evaluation():
    w = I.tiny()
    s = w.systems[0]
    om = O.OracleModel(w.model)
    out = O.evaluate(om, s.pos, s.types, s.box, s.pbc)
    atoms = [0, 7, 19, 31]
    ea, fa = O.sampled(om, s.pos, s.types, s.box, s.pbc, atoms)
    assert np.allclose(ea, out["e_atom"][atoms], rtol=1e-14)
    assert np.allclose(fa, out["forces"][atoms], atol=1e-12)


# ---------------------------------------------------------------- MD
def test_velocity_verlet_reversible_and_conserving():
    """Velocity-Verlet is time-reversible: n steps, negate v, n steps returns
    the start; and NVE energy drift over 40 fs stays small."""
    w = I.tiny()
    s = w.systems[0]
    om = O.OracleModel(w.model)
    rng = np.random.default_rng(0)
    s.vel = I.maxwell_velocities(s.masses, 300.0, rng)
    pos, vel = s.pos.copy(), s.vel.copy()
    conv = 1.0 / 103.6427

    def etot(p, v, e):
        return e + 0.5 * (s.masses[:, None] * v * v).sum() / conv

    out = O.evaluate(om, pos, s.types, s.box, s.pbc)
    e0 = etot(pos, vel, out["energy"])
    dt = 0.5
    for _ in range(20):
        O.vv_first(pos, vel, out["forces"], s.masses, s.box, s.pbc, dt)
        out = O.evaluate(om, pos, s.types, s.box, s.pbc)
        O.vv_second(vel, out["forces"], s.masses, dt)
    e1 = etot(pos, vel, out["energy"])
    assert abs(e1 - e0) < 2e-3 * s.n
    vel = -vel
    for _ in range(20):
        O.vv_first(pos, vel, out["forces"], s.masses, s.box, s.pbc, dt)
        out = O.evaluate(om, pos, s.types, s.box, s.pbc)
        O.vv_second(vel, out["forces"], s.masses, dt)
    d = pos - s.pos
    d -= np.rint(d / s.box) * s.box
    assert np.abs(d).max() < 1e-9
    assert np.allclose(-vel, s.vel, atol=1e-10)


def test_five_species_pins():
    """Five species (the paper's pair-type index b = 1..5): the descriptor
    equals the angular double sum column by column for every pair type, the
    forces are the negative energy gradient, and relabelling atoms of equal
    species leaves E_a and F permuted alike."""
    p, om = _small_model(S=5, K=4, rc=4.5, widths=(10, 8), seed=7)
    c = I.cluster(20, 3.8, seed=8, n_species=5)
    assert set(c.types.tolist()) == {0, 1, 2, 3, 4}
    out = O.evaluate(om, c.pos, c.types, c.box, c.pbc, want_G=True)
    assert out["G"].shape == (c.n, 5 * 4 * 4)
    for a in range(c.n):
        ref = _double_sum_G(p, om, c.pos, c.types, c.box, c.pbc, a)
        assert np.allclose(out["G"][a], ref, rtol=1e-12, atol=1e-14)
    F = out["forces"]
    rng = np.random.default_rng(2)
    for _ in range(10):
        i, x = int(rng.integers(c.n)), int(rng.integers(3))
        fd = _fd_force(om, c.pos, c.types, c.box, c.pbc, i, x)
        assert abs(fd - F[i, x]) <= 1e-7 * max(1.0, abs(F[i, x])) + 1e-8
    perm = rng.permutation(c.n)
    out2 = O.evaluate(om, c.pos[perm], c.types[perm], c.box, c.pbc)
    assert abs(out2["energy"] - out["energy"]) < 1e-12 * abs(out["energy"])
    assert np.allclose(out2["e_atom"], out["e_atom"][perm], atol=1e-12)
    assert np.allclose(out2["forces"], F[perm], atol=1e-11)
