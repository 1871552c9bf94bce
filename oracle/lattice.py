"""Lattice definitions for the oracle (App. A of the paper).

D3Q19 velocities follow the paper's ordering (Eq. cid3q19), in which the
opposite of population i (1 <= i <= 9) is i + 9.  The printed weight list
(Eq. wi) is garbled (it sums to 37/36); the weights used here are the ones
fixed by |c_i|^2 (1/3, 1/18, 1/36), which are the only ones that satisfy
sum w = 1 and sum w c c = c_s^2 I for these velocities.

D2Q9 is not given by the paper (it works in 3D only); the standard set is
used: 0 rest, 1..4 axis links (+x, +y, -x, -y), 5..8 diagonals
(1,1), (-1,1), (-1,-1), (1,-1); weights 4/9, 1/9, 1/36.

Lattice units: dx = dt = 1, c_s^2 = 1/3 (App. A: c_s = dx / (sqrt(3) dt)).
"""
from fractions import Fraction

import numpy as np

CS2 = 1.0 / 3.0

_D3Q19_CX = [0, 1, 1, 0, -1, 0, 0, 0, 1, -1, -1, -1, 0, 1, 0, 0, 0, -1, 1]
_D3Q19_CY = [0, 0, 0, 0, 0, 1, 1, -1, 1, 1, 0, 0, 0, 0, -1, -1, 1, -1, -1]
_D3Q19_CZ = [0, 0, 1, 1, 1, 0, 1, 1, 0, 0, 0, -1, -1, -1, 0, -1, -1, 0, 0]

_D2Q9_C = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


class Lattice:
    """Velocity set with weights, Hermite tensors and the flux tables.

    Attributes
    ----------
    D, Q    : dimension and number of velocities
    c       : int array (Q, D), c[i, a] = component a (0=x, 1=y, 2=z) of c_i
    w       : float array (Q,)
    w_exact : list of Fractions (for exact moment pins)
    H3r     : float array (n3, Q) of the third-order combinations used by the
              equilibrium and the regularized off-equilibrium (Eq. hi3)
    H3r_idx : list of tuples of (sign, (a, b, g)) components of each combination
    N3r     : lattice norms sum_i w_i H3r_k,i^2 of each combination
    """

    def __init__(self, name):
        self.name = name
        if name == "D3Q19":
            self.c = np.array([_D3Q19_CX, _D3Q19_CY, _D3Q19_CZ], dtype=np.int64).T.copy()
        elif name == "D2Q9":
            self.c = np.array(_D2Q9_C, dtype=np.int64)
        else:
            raise ValueError(name)
        self.Q, self.D = self.c.shape
        c2 = (self.c ** 2).sum(axis=1)
        if self.D == 3:
            table = {0: Fraction(1, 3), 1: Fraction(1, 18), 2: Fraction(1, 36)}
        else:
            table = {0: Fraction(4, 9), 1: Fraction(1, 9), 2: Fraction(1, 36)}
        self.w_exact = [table[int(k)] for k in c2]
        self.w = np.array([float(v) for v in self.w_exact])
        self.opp = np.array([int(np.where((self.c == -self.c[i]).all(axis=1))[0][0])
                             for i in range(self.Q)])
        self._build_hermite()

    # -- Hermite polynomials (Eq. hi) --------------------------------------
    def H2(self, a, b):
        """H^(2)_{i,ab} = c_ia c_ib - c_s^2 delta_ab, over all i."""
        c = self.c.astype(np.float64)
        return c[:, a] * c[:, b] - CS2 * (1.0 if a == b else 0.0)

    def H3(self, a, b, g):
        """H^(3)_{i,abg} = c_a c_b c_g - c_s^2 (d_ab c_g + d_bg c_a + d_ag c_b)."""
        c = self.c.astype(np.float64)
        d = lambda p, q: 1.0 if p == q else 0.0
        return (c[:, a] * c[:, b] * c[:, g]
                - CS2 * (d(a, b) * c[:, g] + d(b, g) * c[:, a] + d(a, g) * c[:, b]))

    def _build_hermite(self):
        X, Y, Z = 0, 1, 2
        if self.D == 3:
            # Eq. hi3: the six D3Q19 combinations, in the paper's order.
            self.H3r_idx = [
                [(+1, (X, X, Y)), (+1, (Y, Z, Z))],
                [(+1, (X, Z, Z)), (+1, (X, Y, Y))],
                [(+1, (Y, Y, Z)), (+1, (X, X, Z))],
                [(+1, (X, X, Y)), (-1, (Y, Z, Z))],
                [(+1, (X, Z, Z)), (-1, (X, Y, Y))],
                [(+1, (Y, Y, Z)), (-1, (X, X, Z))],
            ]
        else:
            # D2Q9 supports exactly the two mixed third-order polynomials.
            self.H3r_idx = [[(+1, (X, X, Y))], [(+1, (X, Y, Y))]]
        rows = []
        for combo in self.H3r_idx:
            h = np.zeros(self.Q)
            for s, (a, b, g) in combo:
                h = h + s * self.H3(a, b, g)
            rows.append(h)
        self.H3r = np.array(rows)
        # lattice norms N_k = sum_i w_i H3r_k,i^2 (reading Q3): exact
        # rationals (weights k/36, polynomials in thirds), rounded once
        cs2 = Fraction(1, 3)
        d = lambda p, q: 1 if p == q else 0
        norms = []
        for combo in self.H3r_idx:
            n = Fraction(0)
            for i in range(self.Q):
                ci = [int(v) for v in self.c[i]]
                h = Fraction(0)
                for s, (a, b, g) in combo:
                    h += s * (ci[a] * ci[b] * ci[g] - cs2 * (d(a, b) * ci[g] + d(b, g) * ci[a] + d(a, g) * ci[b]))
                n += self.w_exact[i] * h * h
            norms.append(n)
        self.N3r_exact = norms
        self.N3r = np.array([float(v) for v in norms])

    def combo3(self, T3):
        """Contract a full symmetric third-order tensor T3[a,b,g] into the
        H3r combinations (same signs as Eq. hi3)."""
        out = []
        for combo in self.H3r_idx:
            v = 0.0
            for s, (a, b, g) in combo:
                v = v + s * T3[a][b][g]
            out.append(v)
        return out

    # -- Face-crossing flux tables (Eqs. fluxx, fluxy, fluxz) --------------
    def flux_table(self, axis):
        """Terms of the LB mass flux through the face x + e_axis / 2.

        Returns a list of (i, offset, coef): F^rho_{+axis/2}(x) =
        sum coef * f^col_i(x + offset).  Rule (reproduces the printed D3Q19
        tables term for term, see tests): a population with c_{i,axis} = +1
        leaves from x, one with -1 from x + e_axis; the coefficient carries
        the sign c_{i,axis}; a population with one transverse component t
        is split in halves between its source node and the source node
        shifted by -c_{i,t} e_t.
        """
        terms = []
        for i in range(self.Q):
            ca = int(self.c[i, axis])
            if ca == 0:
                continue
            base = [0] * self.D
            if ca < 0:
                base[axis] = 1
            trans = [t for t in range(self.D) if t != axis and self.c[i, t] != 0]
            if not trans:
                terms.append((i, tuple(base), float(ca)))
            else:
                assert len(trans) == 1
                t = trans[0]
                other = list(base)
                other[t] -= int(self.c[i, t])
                terms.append((i, tuple(base), 0.5 * ca))
                terms.append((i, tuple(other), 0.5 * ca))
        return terms


D2Q9 = Lattice("D2Q9")
D3Q19 = Lattice("D3Q19")


def get(name_or_dim):
    if name_or_dim in ("D2Q9", 2):
        return D2Q9
    if name_or_dim in ("D3Q19", 3):
        return D3Q19
    raise ValueError(name_or_dim)
