"""Quadrature rules (inputs): exactness against closed-form barycentric moments."""
from math import factorial

import numpy as np
import pytest

from paper_2605_14035_gb300.inputs import quadrature as Q


def bary_moment(exps, dim):
    """int_T prod lambda_i^k_i / |T| = dim! prod k_i! / (sum k + dim)!  (all dim+1 barycentrics)."""
    num = factorial(dim)
    for k in exps:
        num *= factorial(k)
    return num / factorial(sum(exps) + dim)


def all_bary_exps(dim, deg):
    out = []

    def rec(prefix, left, k):
        if k == dim + 1:
            out.append(tuple(prefix))
            return
        for a in range(left + 1):
            rec(prefix + [a], left - a, k + 1)

    rec([], deg, 0)
    return out


RULES = [
    (Q.gauss_interval(3), 1.0),
    (Q.gauss_interval(5), 1.0),
    (Q.tri_3pt_deg2(), 0.5),
    (Q.tri_7pt_deg5(), 0.5),
    (Q.tet_4pt_deg2(), 1.0 / 6.0),
    (Q.tet_14pt_deg5(), 1.0 / 6.0),
    (Q.tri_16pt_deg8(), 0.5),
    (Q.paper_rule(1), 1.0),
    (Q.paper_rule(3), 1.0 / 6.0),
    (Q.collapsed_gauss(2, 6), 0.5),
    (Q.collapsed_gauss(3, 5), 1.0 / 6.0),
]


@pytest.mark.parametrize("rule,vol", RULES, ids=[r.name for r, _ in RULES])
def test_barycentric_moments_exact(rule, vol):
    """All barycentric monomials up to the rule degree integrate exactly
    (a different basis from the x^a y^b monomials the rules were solved with)."""
    d = rule.dim
    lam = np.concatenate([1.0 - rule.xi.sum(1, keepdims=True), rule.xi], axis=1)
    worst = 0.0
    for ex in all_bary_exps(d, rule.degree):
        val = rule.w @ np.prod(lam ** np.array(ex)[None, :], axis=1)
        worst = max(worst, abs(val - vol * bary_moment(ex, d)))
    assert worst < 1e-15
    assert abs(rule.w.sum() - vol) < 1e-15


@pytest.mark.parametrize("rule", [Q.tri_7pt_deg5(), Q.tet_14pt_deg5()], ids=["tri7", "tet14"])
def test_not_exact_beyond_degree(rule):
    """A degree-5 rule cannot integrate every degree-6 monomial (sanity of the degree)."""
    d = rule.dim
    lam = np.concatenate([1.0 - rule.xi.sum(1, keepdims=True), rule.xi], axis=1)
    vol = 0.5 if d == 2 else 1 / 6
    errs = [abs(rule.w @ np.prod(lam ** np.array(ex)[None], axis=1) - vol * bary_moment(ex, d))
            for ex in all_bary_exps(d, 6) if sum(ex) == 6]
    assert max(errs) > 1e-8


def test_symmetric_rules_interior_positive():
    for r in (Q.tri_7pt_deg5(), Q.tet_14pt_deg5(), Q.tet_4pt_deg2(), Q.tri_3pt_deg2()):
        lam0 = 1 - r.xi.sum(1)
        assert np.all(r.xi > 0) and np.all(lam0 > 0) and np.all(r.w > 0)


def test_tri7_orbit_parameters_closed_form():
    """The symmetric 7-point degree-5 root has S21 parameters (6 -+ sqrt15)/21 and
    centroid weight 9/80 (Radon's rule): the solver reached the known root."""
    r = Q.tri_7pt_deg5()
    lam = np.concatenate([1.0 - r.xi.sum(1, keepdims=True), r.xi], axis=1)
    reps = set()
    for row in lam[1:]:
        for i in range(3):
            for j in range(i + 1, 3):
                if abs(row[i] - row[j]) < 1e-13:
                    reps.add(round(row[i], 12))
    s15 = 15 ** 0.5
    assert sorted(reps) == sorted([round((6 - s15) / 21, 12), round((6 + s15) / 21, 12)])
    assert abs(r.w[0] - 9 / 80) < 1e-14


def test_sixteen_point_rule_is_symmetric_and_interior():
    """The derived degree-8 rule: 16 points, positive weights, every point inside
    the triangle, and invariant under the permutations of the barycentrics."""
    r = Q.tri_16pt_deg8()
    assert r.w.size == 16 and r.degree == 8 and np.all(r.w > 0)
    lam = np.column_stack([1.0 - r.xi.sum(axis=1), r.xi])
    assert np.all(lam > 0)
    key = sorted(zip(np.round(np.sort(lam, axis=1), 12).tolist(), np.round(r.w, 14)))
    for perm in ([1, 0, 2], [2, 1, 0], [0, 2, 1]):
        lp = lam[:, perm]
        assert sorted(zip(np.round(np.sort(lp, axis=1), 12).tolist(), np.round(r.w, 14))) == key
