"""Pins of the oracle's lattice algebra against exact arithmetic and the
paper's printed tables (App. A).  CPU only."""
import os
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from oracle import lattice as L
from oracle import lbm

GOLD = os.path.join(os.path.dirname(__file__), "golden", "d3q19_flux_tables.txt")


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_weights_exact_moments(lat):
    """sum w = 1, sum w c_a c_b = c_s^2 d_ab and the fourth-order isotropy
    sum w c_a c_b c_g c_d = c_s^4 (d_ab d_gd + d_ag d_bd + d_ad d_bg), in
    exact rationals (this is what fixes the weights of Eq. wi, whose printed
    list is garbled)."""
    cs2 = Fraction(1, 3)
    D = lat.D
    w = lat.w_exact
    assert sum(w) == 1
    d = lambda p, q: 1 if p == q else 0
    for a, b in product(range(D), repeat=2):
        s = sum(w[i] * int(lat.c[i, a]) * int(lat.c[i, b]) for i in range(lat.Q))
        assert s == cs2 * d(a, b)
    for a, b, g, e in product(range(D), repeat=4):
        s = sum(w[i] * int(lat.c[i, a] * lat.c[i, b] * lat.c[i, g] * lat.c[i, e]) for i in range(lat.Q))
        assert s == cs2 * cs2 * (d(a, b) * d(g, e) + d(a, g) * d(b, e) + d(a, e) * d(b, g))


def test_d3q19_ordering_opposites():
    """Eq. cid3q19: the opposite of population i (1..9) is i + 9."""
    for i in range(1, 10):
        assert L.D3Q19.opp[i] == i + 9


def test_h3r_norms_exact():
    """Lattice norms of the Eq. hi3 combinations, computed in exact rationals
    by brute force: 2 c_s^6 for the '+' and 6 c_s^6 for the '-' combinations
    (D3Q19), 2 c_s^6 for H_xxy, H_xyy (D2Q9); mutual orthogonality."""
    cs2 = Fraction(1, 3)
    for lat, expect in ((L.D3Q19, [2, 2, 2, 6, 6, 6]), (L.D2Q9, [2, 2])):
        rows = []
        for combo in lat.H3r_idx:
            h = []
            for i in range(lat.Q):
                v = Fraction(0)
                for s, (a, b, g) in combo:
                    c = [int(x) for x in lat.c[i]]
                    dd = lambda p, q: 1 if p == q else 0
                    v += s * (c[a] * c[b] * c[g] - cs2 * (dd(a, b) * c[g] + dd(b, g) * c[a] + dd(a, g) * c[b]))
                h.append(v)
            rows.append(h)
        for k, h in enumerate(rows):
            n = sum(lat.w_exact[i] * h[i] * h[i] for i in range(lat.Q))
            assert n == expect[k] * cs2 ** 3
            assert abs(float(n) - lat.N3r[k]) < 1e-15
            for k2 in range(k + 1, len(rows)):
                assert sum(lat.w_exact[i] * h[i] * rows[k2][i] for i in range(lat.Q)) == 0


def _read_gold():
    tab = {0: [], 1: [], 2: []}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        ax, coef, i, dx, dy, dz = line.split()
        tab["xyz".index(ax)].append((int(i), (int(dx), int(dy), int(dz)), float(coef)))
    return tab


def test_flux_tables_match_paper():
    """The generic face-crossing rule reproduces Eqs. fluxx, fluxy, fluxz
    term for term (as multisets)."""
    gold = _read_gold()
    for axis in range(3):
        gen = sorted(L.D3Q19.flux_table(axis))
        ref = sorted(gold[axis])
        assert gen == ref


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_equilibrium_moments(lat):
    """Eq. feq moments: sum f = rho, sum c f = rho u,
    sum c c f = rho u u + rho c_s^2 theta I; H3r projections equal the
    combinations of rho u u u (orthogonal projection, reading Q3)."""
    rng = np.random.default_rng(1)
    D = lat.D
    rho = 1.0 + 0.2 * rng.random(5)
    u = 0.2 * rng.standard_normal((D, 5))
    th = 0.5 + rng.random(5)
    feq = lbm.equilibrium(lat, rho, u, th)
    c = lat.c.astype(float)
    assert np.allclose(feq.sum(0), rho, rtol=0, atol=1e-14)
    for a in range(D):
        assert np.allclose((c[:, a, None] * feq).sum(0), rho * u[a], atol=1e-14)
        for b in range(D):
            m = (c[:, a, None] * c[:, b, None] * feq).sum(0)
            ref = rho * u[a] * u[b] + (rho * th / 3.0 if a == b else 0.0)
            assert np.allclose(m, ref, atol=1e-14)
    for k, combo in enumerate(lat.H3r_idx):
        proj = (lat.H3r[k][:, None] * feq).sum(0)
        ref = sum(s * rho * u[a] * u[b] * u[g] for s, (a, b, g) in combo)
        assert np.allclose(proj, ref, atol=1e-14)


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_regularized_neq_idempotent(lat):
    """Eq. fneq: second and third (H3r) moments of the reconstructed
    off-equilibrium equal the traceless Pi and the combinations of Eq. pi3;
    its mass and momentum are zero."""
    rng = np.random.default_rng(2)
    D = lat.D
    u = 0.2 * rng.standard_normal((D, 4))
    A = rng.standard_normal((D, D, 4)) * 1e-3
    Pi = [[A[a, b] + A[b, a] for b in range(D)] for a in range(D)]
    tr = sum(Pi[a][a] for a in range(D))
    Pi = [[Pi[a][b] - (tr / D if a == b else 0) for b in range(D)] for a in range(D)]
    fneq = lbm.regularized_neq(lat, u, Pi)
    c = lat.c.astype(float)
    assert np.allclose(fneq.sum(0), 0, atol=1e-16)
    for a in range(D):
        assert np.allclose((c[:, a, None] * fneq).sum(0), 0, atol=1e-16)
        for b in range(D):
            H = lat.H2(a, b)
            assert np.allclose((H[:, None] * fneq).sum(0), Pi[a][b], atol=1e-16)
    for k, combo in enumerate(lat.H3r_idx):
        proj = (lat.H3r[k][:, None] * fneq).sum(0)
        ref = sum(s * (u[a] * Pi[b][g] + u[b] * Pi[g][a] + u[g] * Pi[a][b]) for s, (a, b, g) in combo)
        assert np.allclose(proj, ref, atol=1e-16)


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19])
def test_force_population_moments(lat):
    """Eq. fi: sum F = 0, sum c F = f_u, sum c c F = a^F (symmetric)."""
    rng = np.random.default_rng(3)
    D = lat.D
    fu = rng.standard_normal((D, 3))
    A = rng.standard_normal((D, D, 3))
    aF = [[A[a, b] + A[b, a] for b in range(D)] for a in range(D)]
    F = lbm.force_populations(lat, fu, aF)
    c = lat.c.astype(float)
    assert np.allclose(F.sum(0), 0, atol=1e-14)
    for a in range(D):
        assert np.allclose((c[:, a, None] * F).sum(0), fu[a], atol=1e-14)
        for b in range(D):
            assert np.allclose((c[:, a, None] * c[:, b, None] * F).sum(0), aF[a][b], atol=1e-14)
