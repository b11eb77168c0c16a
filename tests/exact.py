"""Exact rational reference integrals on affine simplices (independent of the oracle).

Basis functions are written as polynomials in the barycentric coordinates
lambda_0..lambda_d with Fraction coefficients, and integrated with the
Dirichlet formula  int_T lambda^alpha = d! |T| alpha! / (|alpha| + d)!.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product
from math import factorial

import numpy as np

EDGES = {1: ((0, 1),), 2: ((0, 1), (1, 2), (2, 0)), 3: ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))}


def _mono(d, idx_pow):
    e = [0] * (d + 1)
    for i, p in idx_pow:
        e[i] += p
    return tuple(e)


def basis_polys(d, order):
    """List of {exponent tuple: Fraction}: Lagrange P1 / P2 in barycentrics."""
    out = []
    if order == 1:
        for a in range(d + 1):
            out.append({_mono(d, [(a, 1)]): Fraction(1)})
        return out
    for a in range(d + 1):
        out.append({_mono(d, [(a, 2)]): Fraction(2), _mono(d, [(a, 1)]): Fraction(-1)})
    for i, j in EDGES[d]:
        out.append({_mono(d, [(i, 1), (j, 1)]): Fraction(4)})
    return out


def pmul(p, q):
    r = {}
    for ea, ca in p.items():
        for eb, cb in q.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            r[e] = r.get(e, 0) + ca * cb
    return r


def pdiff(p, i):
    r = {}
    for e, c in p.items():
        if e[i]:
            ee = list(e)
            ee[i] -= 1
            r[tuple(ee)] = r.get(tuple(ee), 0) + c * e[i]
    return r


def pint(p, d):
    """int over T of p divided by |T|, exact."""
    tot = Fraction(0)
    for e, c in p.items():
        num = factorial(d)
        for k in e:
            num *= factorial(k)
        tot += c * Fraction(num, factorial(sum(e) + d))
    return tot


def exact_mass_ref(d, order):
    """Reference mass divided by |T| as Fractions [ref][ref]."""
    B = basis_polys(d, order)
    return [[pint(pmul(a, b), d) for b in B] for a in B]


def exact_mass_weighted_ref(d, order, weight_poly):
    B = basis_polys(d, order)
    return [[pint(pmul(pmul(a, b), weight_poly), d) for b in B] for a in B]


def grad_lambda(verts):
    """Constant gradients of the barycentric coordinates of an affine simplex
    embedded in R^n (tangential gradients for a lower-dimensional simplex)."""
    verts = np.asarray(verts, dtype=np.float64)
    E = (verts[1:] - verts[0]).T  # n x d
    dual = E @ np.linalg.inv(E.T @ E)  # n x d, columns = grad lambda_1..d
    g = np.zeros((verts.shape[0], verts.shape[1]))
    g[1:] = dual.T
    g[0] = -dual.sum(axis=1)
    return g


def simplex_measure(verts):
    verts = np.asarray(verts, dtype=np.float64)
    E = (verts[1:] - verts[0]).T
    d = E.shape[1]
    return np.sqrt(np.linalg.det(E.T @ E)) / factorial(d)


def exact_stiffness(verts, order):
    """Stiffness of an affine simplex: sum_ij (grad l_i . grad l_j) int d_i phi_a d_j phi_b."""
    d = len(verts) - 1
    B = basis_polys(d, order)
    g = grad_lambda(verts)
    T = simplex_measure(verts)
    ref = len(B)
    K = np.zeros((ref, ref))
    GG = g @ g.T
    dB = [[pdiff(p, i) for i in range(d + 1)] for p in B]
    for a, b in product(range(ref), range(ref)):
        acc = 0.0
        for i, j in product(range(d + 1), range(d + 1)):
            acc += GG[i, j] * float(pint(pmul(dB[a][i], dB[b][j]), d))
        K[a, b] = acc * T
    return K


def affine_nodes(verts, order):
    """Node coordinates of an affine P1/P2 simplex (corners, then straight edge midpoints)."""
    verts = np.asarray(verts, dtype=np.float64)
    if order == 1:
        return verts.copy()
    d = len(verts) - 1
    mids = [0.5 * (verts[i] + verts[j]) for i, j in EDGES[d]]
    return np.vstack([verts] + mids)
