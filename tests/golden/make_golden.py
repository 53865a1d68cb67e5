"""Writes tests/golden/omega_exact.json from the oracle's exact-rational routines.

Each case is a tiny graph with an exact Omega = (alpha L + I)^{-1} (Sec. 2,
forest matrix), its determinant det(I + alpha L) (= total weight of spanning
trees of G*, Kirchhoff / matrix-forest theorem, Sec. 2 and Prop. 1 proof) and
the exact farness rho(v) = n Omega_vv + tr Omega - 2 (Eq. 3).  The two exact
routes (Gauss-Jordan and forest enumeration) must agree before a case is
written.  Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys
from fractions import Fraction

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from oracle import exact  # noqa: E402

CASES = [
    # name, n, edges (u, v, w), alpha
    ("K2", 2, [(0, 1, "1")], "1"),
    ("P3_alpha_half", 3, [(0, 1, "1"), (1, 2, "1")], "1/2"),
    ("triangle_weighted", 3, [(0, 1, "2"), (1, 2, "1/2"), (0, 2, "3")], "1"),
    ("star4_alpha2", 4, [(0, 1, "1"), (0, 2, "1"), (0, 3, "1")], "2"),
    ("paw_weighted", 4, [(0, 1, "1"), (1, 2, "2"), (2, 0, "1"), (2, 3, "5/2")], "3/4"),
    ("two_components", 5, [(0, 1, "1"), (1, 2, "3"), (3, 4, "1/2")], "1"),
    ("isolated_plus_edge", 3, [(0, 1, "7/2")], "10"),
]


def main():
    out = []
    for name, n, edges, alpha in CASES:
        E = [(u, v, Fraction(w)) for u, v, w in edges]
        a = Fraction(alpha)
        om = exact.omega_gauss_jordan(n, E, a)
        om2, det = exact.omega_forests(n, E, a)
        assert om == om2, name
        tr = sum(om[i][i] for i in range(n))
        far = [n * om[i][i] + tr - 2 for i in range(n)]
        out.append({
            "name": name, "n": n, "alpha": alpha,
            "edges": [[u, v, w] for u, v, w in edges],
            "omega": [[str(x) for x in row] for row in om],
            "det_I_plus_alphaL": str(det),
            "farness_eq3": [str(x) for x in far],
            "cite": "Sec. 2 (forest matrix, matrix-forest theorem); Eq. 3 (farness)",
        })
    path = os.path.join(os.path.dirname(__file__), "omega_exact.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)
    write_group()


# Group forest farness (Sec. 5): exact rho(S) for every S of size 1 and 2,
# and the greedy sequence of Algorithm 3 taken on the exact values (the
# first vertex minimises rho({v}); each next one maximises the drop of rho).
GROUP_CASES = [
    ("paw_weighted", 4, [(0, 1, "1"), (1, 2, "2"), (2, 0, "1"), (2, 3, "5/2")], "3/4", 3),
    ("path5_weighted", 5, [(0, 1, "2"), (1, 2, "1"), (2, 3, "3"), (3, 4, "1/2")], "1", 3),
    ("kite_weighted", 5, [(0, 1, "1"), (0, 2, "2"), (1, 2, "3/2"), (1, 3, "1"), (2, 3, "3/8"), (3, 4, "4")],
     "2", 4),
]


def write_group():
    import itertools
    out = []
    for name, n, edges, alpha, k in GROUP_CASES:
        E = [(u, v, Fraction(w)) for u, v, w in edges]
        a = Fraction(alpha)
        rho = {}
        for r in (1, 2):
            for S in itertools.combinations(range(n), r):
                rho[S] = exact.group_farness(n, E, a, S)
        S = [min(range(n), key=lambda v: (rho[(v,)], v))]
        far = [rho[(S[0],)]]
        while len(S) < k:
            base = exact.group_farness(n, E, a, S)
            gains = {v: base - exact.group_farness(n, E, a, S + [v]) for v in range(n) if v not in S}
            best = max(gains.values())
            assert sum(1 for x in gains.values() if x == best) == 1, name  # no exact ties
            v = max(gains, key=lambda u: gains[u])
            S.append(v)
            far.append(exact.group_farness(n, E, a, S))
        out.append({
            "name": name, "n": n, "alpha": alpha, "k": k,
            "edges": [[u, v, w] for u, v, w in edges],
            "rho": {",".join(map(str, key)): str(val) for key, val in rho.items()},
            "greedy": S, "greedy_farness": [str(x) for x in far],
            "cite": "Sec. 5 (group forest farness, Algorithm 3)",
        })
    path = os.path.join(os.path.dirname(__file__), "group_exact.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
