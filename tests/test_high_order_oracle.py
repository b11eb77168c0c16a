"""Orders 3 and 4 (curves, triangles, tetrahedra) in the oracle, pinned independently
of its product formula: the Lagrange basis obtained by inverting the
Vandermonde matrix of the nodes (exact rationals), exact reference mass and
stiffness matrices, the Lagrange property, partition of unity and finite
differences of the gradients."""
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

import oracle
from paper_2605_14035_gb300.inputs import quadrature

sympy = pytest.importorskip("sympy")


TET_EDGES = [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
TET_FACES = [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]


def node_alphas(dim, p):
    """The documented node order: corners, then edge by edge ((0,1) for curves;
    (0,1), (1,2), (2,0) for triangles; those and (0,3), (1,3), (2,3) for tets)
    the nodes (p-k) e_i + k e_j, k = 1..p-1, then for triangles the interior
    nodes in increasing (alpha_1, alpha_2); for tets the face nodes face by face
    ((0,1,2), (0,1,3), (0,2,3), (1,2,3); on face (i,j,l) increasing (alpha_j,
    alpha_l)), then the interior nodes in increasing (alpha_1, alpha_2, alpha_3)."""
    al = []
    for i in range(dim + 1):
        a = [0] * (dim + 1)
        a[i] = p
        al.append(a)
    edges = [(0, 1)] if dim == 1 else ([(0, 1), (1, 2), (2, 0)] if dim == 2 else TET_EDGES)
    for i, j in edges:
        for k in range(1, p):
            a = [0] * (dim + 1)
            a[i], a[j] = p - k, k
            al.append(a)
    if dim == 2:
        for a1 in range(1, p):
            for a2 in range(1, p - a1):
                al.append([p - a1 - a2, a1, a2])
    if dim == 3:
        for i, j, l in TET_FACES:
            for aj in range(1, p):
                for al_ in range(1, p - aj):
                    a = [0] * 4
                    a[i], a[j], a[l] = p - aj - al_, aj, al_
                    al.append(a)
        for a1 in range(1, p):
            for a2 in range(1, p - a1):
                for a3 in range(1, p - a1 - a2):
                    al.append([p - a1 - a2 - a3, a1, a2, a3])
    return al


def ref_nodes(dim, p):
    """Reference coordinates (x, y) = (lambda_1, lambda_2) of the nodes, exact."""
    return [[Fraction(a[m + 1], p) for m in range(dim)] for a in node_alphas(dim, p)]


def vandermonde_basis(dim, p):
    """Lagrange basis as sympy polynomials from the Vandermonde inverse."""
    xs = sympy.symbols("x0:%d" % dim)
    monos = [m for m in product(range(p + 1), repeat=dim) if sum(m) <= p]
    nodes = ref_nodes(dim, p)
    V = sympy.Matrix([[sympy.prod([sympy.Rational(n[k].numerator, n[k].denominator) ** m[k] for k in range(dim)])
                       for m in monos] for n in nodes])
    C = V.inv()  # column a holds the coefficients of phi_a
    basis = [sum(C[r, a] * sympy.prod([xs[k] ** monos[r][k] for k in range(dim)]) for r in range(len(monos)))
             for a in range(len(nodes))]
    return xs, basis


def integrate_ref(expr, xs):
    """Exact integral over the reference interval / triangle / tetrahedron,
    monomial by monomial: int_0^1 x^a = 1/(a+1); over the triangle x^a y^b ->
    a! b! / (a+b+2)!; over the tetrahedron x^a y^b z^c -> a! b! c! / (a+b+c+3)!."""
    from math import factorial

    total = sympy.Rational(0)
    for mono, coef in sympy.Poly(sympy.expand(expr), *xs).terms():
        if len(xs) == 1:
            total += coef * sympy.Rational(1, mono[0] + 1)
        elif len(xs) == 2:
            a, b = mono
            total += coef * sympy.Rational(factorial(a) * factorial(b), factorial(a + b + 2))
        else:
            a, b, c = mono
            total += coef * sympy.Rational(factorial(a) * factorial(b) * factorial(c), factorial(a + b + c + 3))
    return total


@pytest.mark.parametrize("dim,p", [(1, 3), (1, 4), (2, 3), (2, 4), (3, 3), (3, 4)])
def test_lagrange_property_and_partition_of_unity(dim, p):
    nodes = np.array([[float(c) for c in n] for n in ref_nodes(dim, p)])
    phi, dphi = oracle.tabulate(dim, p, nodes)
    assert np.abs(phi - np.eye(len(nodes))).max() < 1e-13
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (20, dim))
    if dim >= 2:
        pts = pts[pts.sum(1) < 1]
    phi, dphi = oracle.tabulate(dim, p, pts)
    assert np.abs(phi.sum(1) - 1).max() < 1e-13
    assert np.abs(dphi.sum(1)).max() < 1e-12
    h = 1e-6
    for m in range(dim):
        e = np.zeros(dim)
        e[m] = h
        fd = (oracle.tabulate(dim, p, pts + e)[0] - oracle.tabulate(dim, p, pts - e)[0]) / (2 * h)
        assert np.abs(fd - dphi[:, :, m]).max() < 1e-7


@pytest.mark.parametrize("dim,p", [(1, 3), (1, 4), (2, 3), (2, 4), (3, 3), (3, 4)])
def test_reference_matrices_against_vandermonde_basis(dim, p):
    """Affine reference element (the identity map): oracle M and A against the
    exact integrals of the Vandermonde-built basis (curves, triangles: exact
    rational integration; tets: the basis evaluated at a degree-9 conical rule,
    itself checked exact on every monomial up to degree 9, which integrates the
    degree <= 8 products exactly)."""
    xs, basis = vandermonde_basis(dim, p)
    n = len(basis)
    grads = [[sympy.diff(f, x) for x in xs] for f in basis]
    if dim <= 2:
        Mx = np.array([[float(integrate_ref(basis[a] * basis[b], xs)) for b in range(n)] for a in range(n)])
        Ax = np.array([[float(integrate_ref(sum(grads[a][k] * grads[b][k] for k in range(dim)), xs))
                        for b in range(n)] for a in range(n)])
    else:
        exact = quadrature.collapsed_gauss(3, 5)
        pts = [exact.xi[:, k] for k in range(3)]
        ev = lambda f: np.broadcast_to(np.asarray(sympy.lambdify(xs, f, "numpy")(*pts), float), exact.w.shape)
        B = np.stack([ev(f) for f in basis])                                   # [n][Q]
        G = np.stack([np.stack([ev(g) for g in gr]) for gr in grads])          # [n][3][Q]
        Mx = (B * exact.w) @ B.T
        Ax = np.einsum("akq,bkq,q->ab", G, G, exact.w)
    rule = {1: quadrature.gauss_interval(6), 2: quadrature.tri_16pt_deg8(), 3: quadrature.collapsed_gauss(3, 5)}[dim]
    x = np.array([[float(c) for c in nd] for nd in ref_nodes(dim, p)])
    conn = np.arange(n, dtype=np.int32)[None, :]
    M, A, _ = oracle.local_matrices(x, conn, dim, p, rule.xi, rule.w)
    assert np.abs(M[0] - Mx).max() < 1e-14 * 100
    assert np.abs(A[0] - Ax).max() < 1e-12 * np.abs(Ax).max()


def _circle_p1(n):
    t = 2 * np.pi * np.arange(n) / n
    x = np.stack([np.cos(t), np.sin(t)], axis=1)
    conn = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1).astype(np.int32)
    return x, conn


@pytest.mark.parametrize("p,rate", [(3, 3.8), (4, 4.8)])
def test_sphere_and_circle_measures_converge(p, rate):
    """1^T M 1 -> 4 pi on the projected order-p icosphere and -> 2 pi on the
    projected order-p circle, at the rate of the geometric error O(h^{p+1})
    (observed: 4 for p = 3, 6 for p = 4 on the sphere); A.1 = 0."""
    from paper_2605_14035_gb300.inputs import meshes

    errs = []
    for lvl in (1, 2, 3):
        x, e = meshes.icosphere_high(lvl, p)
        r = quadrature.tri_16pt_deg8()
        rp, ci, M, A, _ = oracle.assemble(x, e, 2, p, r.xi, r.w)
        errs.append(abs(M.sum() - 4 * np.pi))
        rows = np.repeat(np.arange(x.shape[0]), np.diff(rp))
        assert np.abs(np.bincount(rows, A, x.shape[0])).max() < 1e-12
    assert np.log2(errs[1] / errs[2]) > rate
    cerrs = []
    for n in (16, 32, 64):
        x1, c1 = _circle_p1(n)
        x, e = meshes.to_order(x1, c1, p, project=lambda y: y / np.linalg.norm(y, axis=1, keepdims=True))
        r = quadrature.gauss_interval(6)
        _, _, M, _, _ = oracle.assemble(x, e, 1, p, r.xi, r.w)
        cerrs.append(abs(M.sum() - 2 * np.pi))
    assert np.log2(cerrs[1] / cerrs[2]) > rate


def test_order_lifting_shares_edge_nodes():
    """Generated order-p meshes: every edge node is shared by the two triangles
    meeting at the edge, and the closed surface has V + (p-1) E + (p-1)(p-2)/2 F nodes."""
    from paper_2605_14035_gb300.inputs import meshes

    for p in (3, 4):
        x, e = meshes.icosphere_high(1, p)
        F = e.shape[0]
        V, E = F // 2 + 2, 3 * F // 2
        assert x.shape[0] == V + (p - 1) * E + (p - 1) * (p - 2) // 2 * F
        counts = np.bincount(e[:, 3:3 + 3 * (p - 1)].ravel(), minlength=x.shape[0])
        assert set(np.unique(counts[V:V + (p - 1) * E])) == {2}


def test_edge_numbering_of_the_lifting_is_the_upper_csr_slots():
    """The GPU lifting numbers edges by the upper slots (i < j) of the order-1
    pattern in CSR order; on the CPU that is the lexicographic order of (low,
    high) vertex pairs the generator uses -- checked by rebuilding the generated
    edge-node numbers from the oracle's pattern."""
    from paper_2605_14035_gb300.inputs import meshes

    for x, e in (meshes.icosphere(2, 1), meshes.hex_disk(4, 1)):
        N = x.shape[0]
        rp, ci = oracle.pattern(e, N)
        upper = [(i, int(j)) for i in range(N) for j in ci[rp[i]:rp[i + 1]] if j > i]
        eid = {edge: k for k, edge in enumerate(upper)}
        for p in (3, 4):
            _, conn = meshes.to_order(x, e, p)
            for le, (a, b) in enumerate([(0, 1), (1, 2), (2, 0)]):
                i, j = e[:, a], e[:, b]
                lo, hi = np.minimum(i, j), np.maximum(i, j)
                ids = np.array([eid[(int(u), int(v))] for u, v in zip(lo, hi)])
                k1 = np.where(i < j, 1, p - 1)  # the node next to the edge's first corner
                assert np.array_equal(conn[:, 3 + le * (p - 1)], N + ids * (p - 1) + k1 - 1)


@pytest.mark.parametrize("case", ["sphere_p3", "circle_p4", "cube_p3"])
def test_adjoint_high_order_central_differences(case):
    """The oracle's adjoint at orders 3, 4 against central differences (h = 1e-6)
    of L = gM.M + gA.A + gC.MC restricted to the elements around the moved node."""
    import pins
    from cases import curved_cube
    from paper_2605_14035_gb300.inputs import meshes

    rng = np.random.default_rng(31)
    if case == "sphere_p3":
        (x, e), d, p, r = meshes.icosphere_high(0, 3), 2, 3, quadrature.tri_16pt_deg8()
    elif case == "circle_p4":
        t = np.linspace(0, 2 * np.pi, 9)[:-1]
        x1 = np.stack([np.cos(t), 0.8 * np.sin(t)], axis=1)
        e1 = np.stack([np.arange(8), (np.arange(8) + 1) % 8], axis=1).astype(np.int32)
        (x, e), d, p, r = meshes.to_order(x1, e1, 4), 1, 4, quadrature.gauss_interval(6)
    else:
        (x, e), d, p, r = curved_cube(1, 3, amp=0.01), 3, 3, quadrature.paper_rule(3)
    x = x + rng.normal(0, 0.003, size=x.shape)
    coef = 1.0 + rng.random((e.shape[0], r.n_pts))
    pat = oracle.pattern(e, x.shape[0])
    nnz = pat[1].size
    gM, gA, gC = rng.normal(size=(3, nnz))
    gx, gc = oracle.adjoint(x, e, d, p, r.xi, r.w, coef, pat, gM, gA, gC)
    h = 1e-6
    scale = np.abs(gx).max()
    for flat in rng.choice(x.size, 6, replace=False):
        k, i = divmod(int(flat), x.shape[1])
        elems = np.nonzero((e == k).any(axis=1))[0]
        xp, xm = x.copy(), x.copy()
        xp[k, i] += h
        xm[k, i] -= h
        fd = (pins.local_L(xp, e, d, p, r, coef, elems, gM, gA, gC, pat) -
              pins.local_L(xm, e, d, p, r, coef, elems, gM, gA, gC, pat)) / (2 * h)
        assert abs(fd - gx[k, i]) < 1e-6 * scale
    # MC is linear in the coefficient: a step in c_{e,q} moves L by exactly step * dL/dc_{e,q}
    for e0, q0 in ((0, 0), (e.shape[0] - 1, r.n_pts - 1)):
        cp, cm = coef.copy(), coef.copy()
        cp[e0, q0] += 0.5
        cm[e0, q0] -= 0.5
        dc = (pins.local_L(x, e, d, p, r, cp, [e0], gM, gA, gC, pat) -
              pins.local_L(x, e, d, p, r, cm, [e0], gM, gA, gC, pat))
        assert abs(dc - gc[e0, q0]) <= 1e-11 * np.abs(gc).max()
