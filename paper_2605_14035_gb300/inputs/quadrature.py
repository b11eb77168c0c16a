"""Quadrature rules on the reference simplices (inputs to assembly, not part of it).

The assembly routines take the rule as an argument (Sec. 3.2.2, Eqs.
reference_quadrature_mass / reference_quadrature_stiffness: nodes xi_i and
weights w_i, i = 1..Q).  This module only *produces* rules; it holds none of the
assembly arithmetic.

Reference simplices (the paper's "span" of the unit vectors is read as their
convex hull):
  interval     [0, 1]                          |E^| = 1
  triangle     conv{(0,0), (1,0), (0,1)}        |E^| = 1/2
  tetrahedron  conv{0, e1, e2, e3}              |E^| = 1/6
Weights sum to |E^|.

Rules are *derived* here, never transcribed: the fully symmetric rules are the
solutions of their moment equations (all monomials up to the rule degree
integrated exactly), solved by Gauss-Newton from a coarse start; the Gauss and
collapsed (conical-product) rules come from the Legendre / Jacobi root
routines.  Exactness is verified when a rule is built.
"""
from __future__ import annotations

from dataclasses import dataclass
from functools import lru_cache
from math import factorial

import numpy as np

__all__ = [
    "Rule",
    "gauss_interval",
    "tri_3pt_deg2",
    "tri_7pt_deg5",
    "tet_14pt_deg5",
    "tet_4pt_deg2",
    "tri_16pt_deg8",
    "paper_rule",
    "collapsed_gauss",
    "monomial_exponents",
    "exact_monomial_integral",
    "default_rule",
]


@dataclass(frozen=True)
class Rule:
    """A quadrature rule on a reference simplex.

    xi: float64 [Q][dim] reference coordinates, w: float64 [Q] weights.
    degree: total polynomial degree integrated exactly.
    """

    dim: int
    xi: np.ndarray
    w: np.ndarray
    degree: int
    name: str

    @property
    def n_pts(self) -> int:
        return int(self.w.shape[0])


def monomial_exponents(dim: int, degree: int):
    """All exponent tuples alpha with |alpha| <= degree in `dim` variables."""
    out = []

    def rec(prefix, left, k):
        if k == dim:
            out.append(tuple(prefix))
            return
        for a in range(left + 1):
            rec(prefix + [a], left - a, k + 1)

    rec([], degree, 0)
    return out


def exact_monomial_integral(alpha) -> float:
    """Integral of prod x_i^alpha_i over the unit reference simplex of dim len(alpha).

    Closed form (Dirichlet integral): prod(alpha_i!) / (|alpha| + dim)!.
    """
    num = 1
    for a in alpha:
        num *= factorial(a)
    return num / factorial(sum(alpha) + len(alpha))


def _moment_residual(points: np.ndarray, weights: np.ndarray, exps) -> np.ndarray:
    res = np.empty(len(exps))
    for k, alpha in enumerate(exps):
        val = np.ones(points.shape[0])
        for i, a in enumerate(alpha):
            if a:
                val = val * points[:, i] ** a
        res[k] = weights @ val - exact_monomial_integral(alpha)
    return res


def _check_exact(rule: Rule, tol: float = 1e-14) -> None:
    exps = monomial_exponents(rule.dim, rule.degree)
    r = _moment_residual(rule.xi, rule.w, exps)
    if np.max(np.abs(r)) > tol:
        raise RuntimeError(f"rule {rule.name}: moment residual {np.max(np.abs(r)):.3e}")


def gauss_interval(n: int) -> Rule:
    """n-point Gauss-Legendre rule mapped to [0, 1]; degree 2n-1."""
    x, w = np.polynomial.legendre.leggauss(n)
    xi = ((x + 1.0) * 0.5).reshape(n, 1)
    rule = Rule(1, np.ascontiguousarray(xi), w * 0.5, 2 * n - 1, f"gauss{n}")
    _check_exact(rule)
    return rule


def tri_3pt_deg2() -> Rule:
    """Three interior points (1/6,1/6), (2/3,1/6), (1/6,2/3), weight 1/6 each.

    Degree 2: the S21 orbit at a = 1/6 with equal weights satisfies the three
    symmetric moment equations of degree <= 2 (checked below).
    """
    a = 1.0 / 6.0
    xi = np.array([[a, a], [1 - 2 * a, a], [a, 1 - 2 * a]])
    w = np.full(3, 1.0 / 6.0)
    rule = Rule(2, xi, w, 2, "tri3_deg2")
    _check_exact(rule)
    return rule


# --- symmetric-orbit constructions -------------------------------------------

def _tri_orbit_s21(a: float) -> np.ndarray:
    """Barycentric orbit (a, a, 1-2a) as reference (x, y) = (lambda2, lambda3)."""
    b = 1.0 - 2.0 * a
    lam = np.array([[a, a, b], [a, b, a], [b, a, a]])
    return lam[:, 1:]


def _tet_orbit_s31(a: float) -> np.ndarray:
    b = 1.0 - 3.0 * a
    lam = np.array([[b, a, a, a], [a, b, a, a], [a, a, b, a], [a, a, a, b]])
    return lam[:, 1:]


def _tet_orbit_s22(a: float) -> np.ndarray:
    b = 0.5 - a
    lam = np.array(
        [[a, a, b, b], [a, b, a, b], [a, b, b, a], [b, a, a, b], [b, a, b, a], [b, b, a, a]]
    )
    return lam[:, 1:]


def _gauss_newton(build, params0, exps, iters=200):
    """Solve the (consistent, overdetermined) moment equations for the orbit params."""
    p = np.array(params0, dtype=np.float64)
    for _ in range(iters):
        pts, wts = build(p)
        r = _moment_residual(pts, wts, exps)
        if np.max(np.abs(r)) < 1e-17:
            break
        jac = np.empty((len(exps), p.size))
        for j in range(p.size):
            h = 1e-7 * max(1.0, abs(p[j]))
            pp = p.copy()
            pm = p.copy()
            pp[j] += h
            pm[j] -= h
            jac[:, j] = (_moment_residual(*build(pp), exps) - _moment_residual(*build(pm), exps)) / (2 * h)
        step, *_ = np.linalg.lstsq(jac, -r, rcond=None)
        p = p + step
    return p


@lru_cache(maxsize=None)
def tri_7pt_deg5() -> Rule:
    """Fully symmetric 7-point degree-5 triangle rule: centroid + two S21 orbits.

    Unknowns (w0, a1, w1, a2, w2); equations: every monomial of degree <= 5.
    Solved by Gauss-Newton from a coarse start; the root found has all points
    interior and all weights positive (checked).
    """
    exps = monomial_exponents(2, 5)

    def build(p):
        w0, a1, w1, a2, w2 = p
        pts = np.vstack([[[1 / 3, 1 / 3]], _tri_orbit_s21(a1), _tri_orbit_s21(a2)])
        wts = np.concatenate([[w0], np.full(3, w1), np.full(3, w2)])
        return pts, wts

    p = _gauss_newton(build, [0.05, 0.1, 0.06, 0.45, 0.07], exps)
    pts, wts = build(p)
    rule = Rule(2, pts, wts, 5, "tri7_deg5")
    _check_exact(rule)
    _check_interior(rule)
    return rule


@lru_cache(maxsize=None)
def tet_14pt_deg5() -> Rule:
    """Fully symmetric 14-point degree-5 tetrahedron rule: two S31 orbits + one S22 orbit.

    Unknowns (a1, w1, a2, w2, b, w3); equations: every monomial of degree <= 5.
    The root reached from the start below has all 14 points interior and all
    weights positive (checked); it is the only such root found from a grid of
    starts (see tests).
    """
    exps = monomial_exponents(3, 5)

    def build(p):
        a1, w1, a2, w2, b, w3 = p
        pts = np.vstack([_tet_orbit_s31(a1), _tet_orbit_s31(a2), _tet_orbit_s22(b)])
        wts = np.concatenate([np.full(4, w1), np.full(4, w2), np.full(6, w3)])
        return pts, wts

    p = _gauss_newton(build, [0.1, 0.012, 0.3, 0.018, 0.05, 0.007], exps)
    pts, wts = build(p)
    rule = Rule(3, pts, wts, 5, "tet14_deg5")
    _check_exact(rule)
    _check_interior(rule)
    return rule


@lru_cache(maxsize=None)
def tet_4pt_deg2() -> Rule:
    """Symmetric 4-point degree-2 tetrahedron rule: one S31 orbit, weights 1/24."""
    exps = monomial_exponents(3, 2)

    def build(p):
        (a,) = p
        return _tet_orbit_s31(a), np.full(4, 1.0 / 24.0)

    p = _gauss_newton(build, [0.15], exps)
    pts, wts = build(p)
    rule = Rule(3, pts, wts, 2, "tet4_deg2")
    _check_exact(rule)
    _check_interior(rule)
    return rule


def _tri_orbit_s111(a: float, b: float) -> np.ndarray:
    """Barycentric orbit of (a, b, 1-a-b): its six permutations."""
    c = 1.0 - a - b
    lam = np.array([[a, b, c], [a, c, b], [b, a, c], [b, c, a], [c, a, b], [c, b, a]])
    return lam[:, 1:]


@lru_cache(maxsize=None)
def tri_16pt_deg8() -> Rule:
    """Fully symmetric 16-point degree-8 triangle rule (the size and degree the
    paper uses for P2 surfaces, Sec. 4.2): centroid + three S21 orbits + one
    S111 orbit.  Unknowns (w0, a1, w1, a2, w2, a3, w3, b1, b2, w4); equations:
    every monomial of degree <= 8.  Solved by Gauss-Newton from a few coarse
    starts; the first root with all points interior and positive weights is
    kept (checked, with exactness to 1e-14)."""
    exps = monomial_exponents(2, 8)

    def build(p):
        w0, a1, w1, a2, w2, a3, w3, b1, b2, w4 = p
        pts = np.vstack([[[1 / 3, 1 / 3]], _tri_orbit_s21(a1), _tri_orbit_s21(a2), _tri_orbit_s21(a3),
                         _tri_orbit_s111(b1, b2)])
        wts = np.concatenate([[w0], np.full(3, w1), np.full(3, w2), np.full(3, w3), np.full(6, w4)])
        return pts, wts

    starts = [[0.07, 0.45, 0.05, 0.17, 0.05, 0.05, 0.015, 0.26, 0.01, 0.014],
              [0.07, 0.46, 0.045, 0.17, 0.05, 0.06, 0.015, 0.30, 0.02, 0.01],
              [0.06, 0.44, 0.04, 0.2, 0.04, 0.05, 0.02, 0.25, 0.03, 0.012]]
    for st in starts:
        p = _gauss_newton(build, st, exps, iters=400)
        pts, wts = build(p)
        rule = Rule(2, pts, wts, 8, "tri16_deg8")
        try:
            _check_exact(rule)
            _check_interior(rule)
        except RuntimeError:
            continue
        return rule
    raise RuntimeError("no admissible 16-point degree-8 root from the starts")


def paper_rule(dim: int) -> Rule:
    """Rules of the sizes and degrees the paper names for P2 (Sec. 4.2: order
    10, 8 and 7 in one, two and three dimensions), derived here: 6-point Gauss
    (degree 11 >= 10) on the interval, the 16-point degree-8 symmetric triangle
    rule, and for the tetrahedron a degree-7 conical product rule (64 points;
    the paper's symmetric tet rule is not transcribed)."""
    if dim == 1:
        return gauss_interval(6)
    if dim == 2:
        return tri_16pt_deg8()
    if dim == 3:
        return collapsed_gauss(3, 4)
    raise ValueError(dim)


def _check_interior(rule: Rule) -> None:
    lam0 = 1.0 - rule.xi.sum(axis=1)
    if not (np.all(rule.xi > 0) and np.all(lam0 > 0) and np.all(rule.w > 0)):
        raise RuntimeError(f"rule {rule.name}: point outside the simplex or negative weight")


def collapsed_gauss(dim: int, n: int) -> Rule:
    """Conical-product (collapsed Gauss-Jacobi x Gauss-Legendre) rule, degree 2n-1.

    Triangle: x = u, y = v (1 - u) with Jacobian (1 - u), u ~ Gauss-Jacobi(0,1).
    Tetrahedron: x = u, y = v (1-u), z = t (1-u)(1-v), Jacobian (1-u)^2 (1-v).
    Used as a high-degree reference rule in tests (curved-element convergence).
    """
    from scipy.special import roots_jacobi

    def jac01(alpha):
        # Gauss-Jacobi nodes for weight (1-u)^alpha on [0, 1].
        x, w = roots_jacobi(n, alpha, 0.0)
        return (x + 1.0) * 0.5, w / 2.0 ** (alpha + 1)

    if dim == 1:
        return gauss_interval(n)
    ug, vg = jac01(dim - 1), None
    lg_x, lg_w = np.polynomial.legendre.leggauss(n)
    lg_x = (lg_x + 1) * 0.5
    lg_w = lg_w * 0.5
    if dim == 2:
        u, wu = ug
        U, V = np.meshgrid(u, lg_x, indexing="ij")
        W = np.outer(wu, lg_w)
        xi = np.stack([U.ravel(), (V * (1 - U)).ravel()], axis=1)
        rule = Rule(2, xi, W.ravel(), 2 * n - 1, f"collapsed_tri_{n}")
    elif dim == 3:
        u, wu = ug
        v, wv = jac01(1)
        U, V, T = np.meshgrid(u, v, lg_x, indexing="ij")
        W = wu[:, None, None] * wv[None, :, None] * lg_w[None, None, :]
        xi = np.stack([U.ravel(), (V * (1 - U)).ravel(), (T * (1 - U) * (1 - V)).ravel()], axis=1)
        rule = Rule(3, xi, W.ravel(), 2 * n - 1, f"collapsed_tet_{n}")
    else:
        raise ValueError(dim)
    _check_exact(rule, tol=1e-13)
    return rule


def default_rule(dim: int, order: int) -> Rule:
    """The rule each workload uses: P1 triangles 3-pt degree 2, P2 triangles 7-pt
    degree 5, tetrahedra 14-pt degree 5, curves 3-point Gauss (degree 5)."""
    if dim == 1:
        return gauss_interval(3)
    if dim == 2:
        return tri_3pt_deg2() if order == 1 else tri_7pt_deg5()
    if dim == 3:
        return tet_14pt_deg5()
    raise ValueError(dim)
