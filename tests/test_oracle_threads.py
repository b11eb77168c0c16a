"""The all-core oracle assembly (the timed CPU baseline) against the
single-thread oracle: bit-identical results on every thread count, because
each slot's contributions are added in the same (element, a, b) order with the
same compensated sums.  Includes a mesh of more than one 65,536-element chunk
and meshes with repeated nodes in an element and unreferenced nodes."""
import numpy as np
import pytest

import oracle
from cases import build_cases, coef_field

CASES = build_cases()


def _check(x, e, d, p, xi, w, coef, n_nodes=None, threads=(1, 3, 8)):
    nn = x.shape[0] if n_nodes is None else n_nodes
    pat = oracle.pattern(e, nn)
    ref = oracle.assemble(x, e, d, p, xi, w, coef, pat=pat)
    for t in threads:
        got = oracle.assemble_threads(x, e, d, p, xi, w, coef, pat=pat, n_nodes=nn, threads=t)
        for k in (2, 3, 4):
            assert np.array_equal(got[k].view(np.int64), ref[k].view(np.int64)), (t, k)


@pytest.mark.parametrize("name", ["perturbed_sphere_p2", "cube_p2", "curve_p2", "disk_p1", "sphere_p3", "cube_p3"])
def test_threads_bit_identical(name):
    x, e, d, p, rule = CASES[name]
    coef = coef_field(oracle.eval_points(x, e, d, p, rule.xi))
    _check(x, e, d, p, rule.xi, rule.w, coef)


def test_threads_several_chunks():
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x, e = meshes.icosphere(6, 1)  # 81,920 elements: two chunks
    r = quadrature.tri_3pt_deg2()
    _check(x, e, 2, 1, r.xi, r.w, None, threads=(2, 8))


def test_threads_repeated_and_unreferenced_nodes():
    x, e, d, p, rule = CASES["disk_p1"]
    e = e.copy()
    e[5, 1] = e[5, 0]  # a repeated node in one element sums into one slot
    x2 = np.vstack([x, [[5.0, 5.0], [6.0, 6.0]]])  # two unreferenced nodes: empty rows
    _check(x2, e, d, p, rule.xi, rule.w, None)
