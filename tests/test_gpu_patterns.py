"""Pattern paths the small parity cases do not reach, against the oracle:
a node in more than 200 P2 triangles or 110 P2 tetrahedra (its row holds more
than 1024 raw column keys, so the block-wide segmented sort runs), and tile
blocks forced to 32-bit slot entries.  Patterns bit-exact; FP64 within 1e-12,
mixed within 1e-6 (diagonal-scaled); the entry width changes no bit."""
import numpy as np
import pytest
import torch

import oracle
from cases import coef_field, diag_scaled_error
from paper_2605_14035_gb300.inputs import quadrature

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lfem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14035_gb300 import lfem as m

    return m


def fan_triangles(k, surface):
    """k triangles around node 0 (a wavy disk when surface), lifted to P2."""
    t = 2 * np.pi * np.arange(k) / k
    r = 1.0 + 0.1 * np.cos(5 * t)
    ring = np.stack([r * np.cos(t), r * np.sin(t)], 1)
    v = np.vstack([[0.0, 0.0], ring])
    f = np.stack([np.zeros(k, int), 1 + np.arange(k), 1 + (np.arange(k) + 1) % k], 1).astype(np.int32)
    x, e = oracle.lift_order(v, f, 2)
    if surface:
        x = np.column_stack([x, 0.2 * np.sin(3 * x[:, 0]) * x[:, 1]])
    return x, e


def fan_tets(k):
    """k tetrahedra sharing the axis from node 0 to the apex, lifted to P2."""
    t = 2 * np.pi * np.arange(k) / k
    ring = np.stack([np.cos(t), np.sin(t), 0.05 * np.sin(7 * t)], 1)
    v = np.vstack([[0.0, 0.0, 0.0], ring, [0.0, 0.0, 1.0]])
    apex = k + 1
    f = np.stack([np.zeros(k, int), 1 + np.arange(k), 1 + (np.arange(k) + 1) % k, np.full(k, apex)], 1)
    return oracle.lift_order(v, f.astype(np.int32), 2)


CASES = {
    "fan_plane_p2": lambda: (*fan_triangles(210, False), 2, quadrature.tri_7pt_deg5()),
    "fan_surface_p2": lambda: (*fan_triangles(230, True), 2, quadrature.tri_7pt_deg5()),
    "fan_tets_p2": lambda: (*fan_tets(120), 3, quadrature.tet_14pt_deg5()),
}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_high_valence_rows(name, lfem):
    x, e, d, rule = CASES[name]()
    counts = np.bincount(e.ravel(), minlength=x.shape[0])
    assert counts.max() * e.shape[1] > 1024  # the block-wide sort's rows
    pat = lfem.Pattern(_dev(e), x.shape[0], d, 2)
    rp, ci = pat.csr()
    orp, oci = oracle.pattern(e, x.shape[0])
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)
    coef = coef_field(oracle.eval_points(x, e, d, 2, rule.xi))
    _, _, M, A, C = oracle.assemble(x, e, d, 2, rule.xi, rule.w, coef)
    for prec, tol in ((lfem.FP64, 1e-12), (lfem.MIXED, 1e-6)):
        cd = _dev(coef) if prec == lfem.FP64 else _dev(coef).float()
        out = lfem.assemble(pat, _dev(x), rule, cd, which=7, precision=prec)
        torch.cuda.synchronize()
        for k, ref in (("M", M), ("A", A), ("MC", C)):
            assert diag_scaled_error(out[k].double().cpu().numpy(), ref, orp, oci) <= tol, (name, prec, k)
    pat.sync_status()


@pytest.mark.parametrize("name", ["fan_surface_p2", "perturbed"])
def test_wide_entries_change_no_bit(name, lfem):
    if name == "perturbed":
        from cases import build_cases

        x, e, d, p, rule = build_cases()["perturbed_sphere_p2"]
    else:
        x, e, d, rule = CASES[name]()
    coef = coef_field(oracle.eval_points(x, e, d, 2, rule.xi))
    pat = lfem.Pattern(_dev(e), x.shape[0], d, 2)
    pat.retile(max(1024, pat.info()["max_row"]))
    ref = {prec: lfem.assemble(pat, _dev(x), rule, _dev(coef).to(dt), which=7, precision=prec)
           for prec, dt in ((lfem.FP64, torch.float64), (lfem.MIXED, torch.float32))}
    pat.debug_wide_entries(True)
    for prec, dt in ((lfem.FP64, torch.float64), (lfem.MIXED, torch.float32)):
        got = lfem.assemble(pat, _dev(x), rule, _dev(coef).to(dt), which=7, precision=prec)
        for k in ("M", "A", "MC"):
            assert torch.equal(got[k], ref[prec][k]), (prec, k)
    _, _, M, _, _ = oracle.assemble(x, e, d, 2, rule.xi, rule.w, coef)
    orp, oci = oracle.pattern(e, x.shape[0])
    assert diag_scaled_error(got["M"].double().cpu().numpy(), M, orp, oci) <= 1e-6
    pat.debug_wide_entries(False)
    pat.sync_status()
