"""The Cartesian building blocks of Eqs. (10)-(13) as data (oracle).

TEST INFRASTRUCTURE ONLY (see the package header).

Each entry is (coefficient, k-monomial (px, py, pz), field name).  The field
B_ij = FT[F r_i r_j / r^2] (Eq. 11) and C_ijl = FT[F r_i^2 r_j r_l / r^4] (Eq. 13);
``field_monomial`` turns a name into the exponents (a, b, c) of r_x^a r_y^b r_z^c.

A_2 k^2 = sum of the A2_TERMS (Eq. 10), A_4 k^4 = sum of the A4_TERMS (Eq. 12),
written down term by term as the equations print them.

A_6 k^6 (l = 6) is not printed: Sec. 3 only states that higher orders decompose in
the same way.  A6_TERMS writes out the multinomial expansion of (k . r)^6 -- one
term per monomial k_x^a k_y^b k_z^c r_x^a r_y^b r_z^c, coefficient 6!/(a! b! c!),
field D_abc = FT[F r_x^a r_y^b r_z^c / r^6] -- the same construction that gives the
printed Eqs. (10) and (12) for n = 2 and 4.

Pinned by: tests/golden/eq10_eq12_terms.txt (the printed terms, transcribed
separately) and the identity (k.r)^n / (k r)^n = sum_terms coef k^p r^m / (k^n r^n)
checked on random unit vectors (tests/test_oracle_pins.py).
"""
from __future__ import annotations

from math import factorial

A2_TERMS = [
    (1, (2, 0, 0), "Bxx"),
    (1, (0, 2, 0), "Byy"),
    (1, (0, 0, 2), "Bzz"),
    (2, (1, 1, 0), "Bxy"),
    (2, (1, 0, 1), "Bxz"),
    (2, (0, 1, 1), "Byz"),
]

A4_TERMS = [
    (1, (4, 0, 0), "Cxxx"),
    (1, (0, 4, 0), "Cyyy"),
    (1, (0, 0, 4), "Czzz"),
    (4, (3, 1, 0), "Cxxy"),
    (4, (3, 0, 1), "Cxxz"),
    (4, (1, 3, 0), "Cyyx"),
    (4, (0, 3, 1), "Cyyz"),
    (4, (1, 0, 3), "Czzx"),
    (4, (0, 1, 3), "Czzy"),
    (6, (2, 2, 0), "Cxyy"),
    (6, (2, 0, 2), "Cxzz"),
    (6, (0, 2, 2), "Cyzz"),
    (12, (2, 1, 1), "Cxyz"),
    (12, (1, 2, 1), "Cyxz"),
    (12, (1, 1, 2), "Czxy"),
]

_AX = {"x": 0, "y": 1, "z": 2}


A6_TERMS = [(factorial(6) // (factorial(a) * factorial(b) * factorial(6 - a - b)), (a, b, 6 - a - b),
             f"D{a}{b}{6 - a - b}")
            for a in range(6, -1, -1) for b in range(6 - a, -1, -1)]


def field_monomial(name: str):
    """Exponents (a, b, c) of r_x^a r_y^b r_z^c in the numerator of a B, C or D field.

    B_ij -> r_i r_j ; C_ijl -> r_i^2 r_j r_l (Eq. 13) ; D_abc -> r_x^a r_y^b r_z^c.
    """
    if name[0] == "D":
        a, b, c = (int(v) for v in name[1:4])
        return (a, b, c), a + b + c
    e = [0, 0, 0]
    if name[0] == "B":
        i, j = name[1], name[2]
        e[_AX[i]] += 1
        e[_AX[j]] += 1
        return tuple(e), 2
    if name[0] == "C":
        i, j, l = name[1], name[2], name[3]
        e[_AX[i]] += 2
        e[_AX[j]] += 1
        e[_AX[l]] += 1
        return tuple(e), 4
    raise ValueError(name)
