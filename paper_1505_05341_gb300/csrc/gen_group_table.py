"""Generate group_table.inc: the k_y, k_z polynomial weights that fold the
transformed line-of-sight fields into powers of k_x.

Background (Sec. 3, Eqs. 9-13).  With hats r_hat = r / |r|,
  k^n A_n(k) = sum_{a+b+c=n} n!/(a! b! c!) k_x^a k_y^b k_z^c FT[F r_hat_x^a r_hat_y^b r_hat_z^c],
which for n = 2 and n = 4 is Eq. (10) and Eq. (12) term by term.  After the transforms
along y and z, k_y and k_z are known, so the terms with the same power p of k_x
can be summed: G_{n,p}(x; k_y, k_z), and k^n A_n = sum_p k_x^p FT_x[G_{n,p}].

The library transforms fewer than 22 fields: r_hat_z^2 = 1 - r_hat_x^2 - r_hat_y^2
turns every monomial with c >= 2 into ones with c <= 1 and lower degree, so the
fields actually transformed (the "basis") are
  0: F (for A_0), 1: F' = F with the node at r = 0 removed (that node has weight 0
  in every LOS field, so the identity above only holds for F'),
  degree 2, c <= 1 : (2,0,0) (1,1,0) (0,2,0) (1,0,1) (0,1,1),
  degree 4, c <= 1 : (4,0,0) (3,1,0) (2,2,0) (1,3,0) (0,4,0) (3,0,1) (2,1,1) (1,2,1) (0,3,1).
16 real fields = 8 complex transforms for l <= 4 (7 fields for l <= 2).  For l <= 6
the degree-6 monomials with c <= 1 add 13 fields (29 in all) and the groups
(6, 0..6) add 7 (16 in all).

Run:  python gen_group_table.py > group_table.inc
"""
from __future__ import annotations

import math
from collections import defaultdict
from fractions import Fraction

DEG2 = [(2, 0, 0), (1, 1, 0), (0, 2, 0), (1, 0, 1), (0, 1, 1)]
DEG4 = [(4, 0, 0), (3, 1, 0), (2, 2, 0), (1, 3, 0), (0, 4, 0),
        (3, 0, 1), (2, 1, 1), (1, 2, 1), (0, 3, 1)]
DEG6 = [(6 - b, b, 0) for b in range(7)] + [(5 - b, b, 1) for b in range(6)]


def basis(ell_max):
    """List of (a, b, c, degree) per basis index; index 0 = F, 1 = F'."""
    if ell_max == 0:
        return [(0, 0, 0, 0)]
    out = [(0, 0, 0, 0), (0, 0, 0, -1)]
    if ell_max >= 2:
        out += [m + (2,) for m in DEG2]
    if ell_max >= 4:
        out += [m + (4,) for m in DEG4]
    if ell_max >= 6:
        out += [m + (6,) for m in DEG6]
    return out


def reduce_term(a, b, c, n, ell_max):
    """x_hat^a y_hat^b z_hat^c (degree n = a+b+c >= 2, or F' for n = 0) as a
    combination {basis index: coefficient}."""
    bs = basis(ell_max)
    if n == 0:
        return {1: Fraction(1)}
    if c <= 1:
        return {bs.index((a, b, c, n)): Fraction(1)}
    out = defaultdict(Fraction)
    for sgn, (aa, bb, cc, nn) in ((1, (a, b, c - 2, n - 2)), (-1, (a + 2, b, c - 2, n)),
                                  (-1, (a, b + 2, c - 2, n))):
        for k, v in reduce_term(aa, bb, cc, nn, ell_max).items():
            out[k] += sgn * v
    return {k: v for k, v in out.items() if v != 0}


def groups(ell_max):
    """[(n, p)] in output order: A0, then (2,0..2), then (4,0..4)."""
    g = [(0, 0)]
    if ell_max >= 2:
        g += [(2, p) for p in range(3)]
    if ell_max >= 4:
        g += [(4, p) for p in range(5)]
    if ell_max >= 6:
        g += [(6, p) for p in range(7)]
    return g


def table(ell_max):
    """{(group, basis): {(b, c): coef}}: G_g = sum_basis poly(k_y, k_z) Psi_basis."""
    tab = defaultdict(lambda: defaultdict(Fraction))
    for gi, (n, p) in enumerate(groups(ell_max)):
        if n == 0:
            tab[(gi, 0)][(0, 0)] += 1
            continue
        for b in range(n - p + 1):
            c = n - p - b
            mult = math.factorial(n) // (math.factorial(p) * math.factorial(b) * math.factorial(c))
            for beta, coef in reduce_term(p, b, c, n, ell_max).items():
                tab[(gi, beta)][(b, c)] += mult * coef
    return {k: {m: v for m, v in poly.items() if v != 0} for k, poly in tab.items()}


def emit(ell_max):
    bs = basis(ell_max)
    gs = groups(ell_max)
    tab = table(ell_max)
    lines = []
    nb, ng = len(bs), len(gs)
    lines.append(f"// l_max = {ell_max}: {nb} basis fields -> {ng} k_x-power groups")
    lines.append(f"template <> struct GroupTable<{ell_max}> {{")
    lines.append(f"  static constexpr int NB = {nb};")
    lines.append(f"  static constexpr int NG = {ng};")
    lines.append("  // G_g(k_y, k_z) += sum_{LO <= beta < HI} poly_{g,beta}(k_y, k_z) Psi_beta, where psi(beta)")
    lines.append("  // returns Psi_beta; combine() zeroes G and adds every basis field.")
    lines.append("  template <int LO, int HI, class PsiAt>")
    lines.append("  __device__ static __forceinline__ void accumulate(PsiAt psi, float ky, float kz, float2 (&g)[NG]) {")
    npow = max(5, ell_max + 1)
    lines.append(f"    float kyp[{npow}], kzp[{npow}];")
    lines.append("    kyp[0] = 1.f; kzp[0] = 1.f;")
    lines.append("    #pragma unroll")
    lines.append(f"    for (int i = 1; i < {npow}; ++i) {{ kyp[i] = kyp[i - 1] * ky; kzp[i] = kzp[i - 1] * kz; }}")
    by_beta = {}
    for (gi, beta), poly in sorted(tab.items()):
        by_beta.setdefault(beta, []).append((gi, poly))
    for beta in sorted(by_beta):
        lines.append(f"    if constexpr (LO <= {beta} && {beta} < HI) {{ const float2 ps = psi({beta});")
        for gi, poly in by_beta[beta]:
            terms = []
            for (b, c), v in sorted(poly.items()):
                assert v.denominator == 1
                terms.append(f"({float(v.numerator)!r}f * kyp[{b}] * kzp[{c}])")
            lines.append(f"      {{ const float w = {' + '.join(terms)};")
            lines.append(f"        g[{gi}].x = fmaf(w, ps.x, g[{gi}].x); g[{gi}].y = fmaf(w, ps.y, g[{gi}].y); }}")
        lines.append("    }")
    lines.append("  }")
    lines.append("  template <class PsiAt>")
    lines.append("  __device__ static __forceinline__ void combine(PsiAt psi, float ky, float kz, float2 (&g)[NG]) {")
    for gi in range(ng):
        lines.append(f"    g[{gi}] = make_float2(0.f, 0.f);")
    lines.append(f"    accumulate<0, {nb}>(psi, ky, kz, g);")
    lines.append("  }")
    arr = ", ".join(f"{a}, {b}, {c}, {d}" for a, b, c, d in bs)
    lines.append("  // mono_c(beta, i): i = 0, 1, 2 exponents of r_hat_x, r_hat_y, r_hat_z; i = 3 degree.")
    lines.append("  __host__ __device__ static constexpr int mono_c(int beta, int i) {")
    lines.append(f"    constexpr int t[{4 * nb}] = {{{arr}}};")
    lines.append("    return t[4 * beta + i];")
    lines.append("  }")
    lines.append("  // Exponents (a, b, c) of r_hat_x^a r_hat_y^b r_hat_z^c and the degree of basis field")
    lines.append("  // beta; degree 0 = F itself, -1 = F with the node at r = 0 removed.")
    lines.append("  __device__ static __forceinline__ void mono(int beta, int& a, int& b, int& c, int& d) {")
    lines.append("    switch (beta) {")
    for i, (a, b, c, d) in enumerate(bs):
        lines.append(f"      case {i}: a = {a}; b = {b}; c = {c}; d = {d}; break;")
    lines.append("      default: a = 0; b = 0; c = 0; d = -2; break;")
    lines.append("    }")
    lines.append("  }")
    lines.append("};")
    return "\n".join(lines)


def main():
    print("// Generated by gen_group_table.py -- do not edit.")
    print("// Folds the y,z-transformed basis fields into powers of k_x (Eqs. 10 and 12).")
    print("template <int ELL> struct GroupTable;")
    for ell in (0, 2, 4, 6):
        print(emit(ell))


if __name__ == "__main__":
    main()
