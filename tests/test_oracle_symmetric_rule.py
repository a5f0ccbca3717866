"""The smaller symmetric volume rule (Grundmann-Moller, oracle/quadrature.symmetric_volume_rule)
pinned without reference to the library: exact monomial integrals to degree 2k+3 and not
beyond, weights summing to one, node counts C(k+5, 4), invariance of the node set under every
permutation of the barycentric coordinates; and the HDG pipeline of the oracle on it: the
condensed matrices equal the conical rule's whenever both rules integrate every integrand
exactly, the method is exact for u in P_k, and the observed orders are k + 1."""
from itertools import permutations
from math import comb, factorial

import numpy as np
import pytest

from oracle import hdg as ohdg
from oracle import quadrature
from oracle.geometry import ExpandedMesh
from workloads import boundary_faces, get_problem, kuhn_cube


def _mono(p, w, a, b, c):
    return float((w * p[:, 0] ** a * p[:, 1] ** b * p[:, 2] ** c).sum()) / 6.0


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_exactness_and_size(k):
    p, w, lam = quadrature.symmetric_volume_rule(k)
    assert len(w) == comb(k + 5, 4)
    assert abs(w.sum() - 1.0) < 1e-13
    assert np.all(lam > 0)  # interior nodes
    deg = 2 * k + 3
    worst = 0.0
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                exact = factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)
                worst = max(worst, abs(_mono(p, w, a, b, c) - exact) / exact)
    assert worst < 1e-12
    # not exact beyond its degree (some monomial of degree 2k+4 is missed)
    miss = max(abs(_mono(p, w, a, deg + 1 - a, 0) - factorial(a) * factorial(deg + 1 - a) / factorial(deg + 4))
               for a in range(deg + 2))
    assert miss > 1e-10


@pytest.mark.parametrize("k", [1, 2, 3])
def test_invariant_under_barycentric_permutations(k):
    p, w, lam = quadrature.symmetric_volume_rule(k)
    # the multiset of (node, weight) pairs (a node may occur on two levels, e.g. the centroid)
    ref = sorted(tuple(np.round(np.append(l, wt), 12)) for l, wt in zip(lam, w))
    for perm in permutations(range(4)):
        got = sorted(tuple(np.round(np.append(l[list(perm)], wt), 12)) for l, wt in zip(lam, w))
        assert got == ref


def test_condensed_blocks_equal_where_both_rules_are_exact():
    """kappa, c constant and tau = 1: every volume integrand is a polynomial of degree <= 2k,
    which both rules integrate exactly, so C^K and C_f^K (f linear) agree to rounding."""
    k = 2
    prob = get_problem("cube4_k1").at(s=2, k=k)
    c, e = kuhn_cube(2, 0.2, 1)
    d, n = boundary_faces(c, e, prob.classify)
    mesh = ExpandedMesh(c, e, d, n)
    out = {}
    for rule in ("conical", "symmetric"):
        tab = ohdg.Tables(k, rule)
        X, Y, Z = ohdg.volume_nodes(mesh, tab)
        blk = ohdg.local_blocks(mesh, tab, 2.0 + 0 * X, 0.5 + 0 * X, 1.0 + X - 2 * Y + Z)
        out[rule] = ohdg.local_solvers(blk)[:2]
    for a, b in zip(out["conical"], out["symmetric"]):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_exact_for_polynomial_solution():
    """u in P_k, kappa constant, c constant: the HDG solution is the projection of the exact
    one (q_h = q, u_h = u, u_hat = u), on the symmetric rule as on the conical one."""
    from workloads.problems import Problem
    k = 2
    u = lambda x, y, z: 1 + x - 2 * y * z + 0.5 * x * x  # noqa: E731
    q = lambda x, y, z: (-3 * (1 + x), 3 * 2 * z + 0 * x, 3 * 2 * y + 0 * x)  # noqa: E731  (kappa = 3)
    f = lambda x, y, z: -3 * 1.0 + 2 * u(x, y, z)  # noqa: E731  div q + c u with c = 2
    prob = Problem(name="poly", s=2, k=k, kappa=lambda x, y, z: 3 + 0 * x, c=lambda x, y, z: 2 + 0 * x, f=f,
                   uD=u, u=u, q=q, jitter=0.15, seed=2)
    r = ohdg.solve_problem(prob, rule="symmetric")
    e = ohdg.errors(r["mesh"], k, r["q"], r["u"], r["uhat"], r["ustar"], prob)
    assert max(e.values()) < 1e-11, e


@pytest.mark.parametrize("k", [1, 2])
def test_orders_on_symmetric_rule(k):
    """Observed orders k + 1 (s = 4 -> 8), and errors within 3 % of the conical rule's (the two
    discrete solutions differ by the quadrature error only)."""
    errs, conical = [], []
    for s in (4, 8):
        prob = get_problem("cube16_k3").at(s=s, k=k)
        r = ohdg.solve_problem(prob, rule="symmetric")
        errs.append(ohdg.errors(r["mesh"], k, r["q"], r["u"], r["uhat"], r["ustar"], prob))
        r0 = ohdg.solve_problem(prob)
        conical.append(ohdg.errors(r0["mesh"], k, r0["q"], r0["u"], r0["uhat"], r0["ustar"], prob))
    for key in ("e_q", "e_u", "e_uhat"):
        rate = np.log2(errs[0][key] / errs[1][key])
        assert rate > k + 1 - 0.2, (key, rate)
    for e, e0 in zip(errs, conical):
        for key in e0:
            assert abs(e[key] - e0[key]) <= 0.03 * e0[key], (key, e[key], e0[key])
