"""CUDA path against the FP64 oracle, element by element, on the same seeded inputs.

Bars: patterns bit-exact; FP64 values within 1e-12 diagonal-scaled relative
error; mixed values within 1e-6 (the stated tolerances); bit-identical reruns
and tile-shape independence; adjoint within 1e-10 of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from cases import build_cases, coef_field, diag_scaled_error

pytestmark = pytest.mark.gpu

CASES = build_cases()
FP64_TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def lfem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14035_gb300 import lfem as m

    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def prepare(name, lfem, tile_slots=256):
    x, e, d, p, rule = CASES[name]
    pts = oracle.eval_points(x, e, d, p, rule.xi)
    coef = coef_field(pts)
    pat = lfem.Pattern(to_dev(e), x.shape[0], d, p)
    if tile_slots and not (d == 3 and p >= 3):  # order-3/4 tets have no row tiles
        pat.retile(tile_slots)
    return x, e, d, p, rule, coef, pat


@pytest.mark.parametrize("name", list(CASES))
def test_pattern_bit_exact(name, lfem):
    x, e, d, p, rule, coef, pat = prepare(name, lfem, tile_slots=0)
    rp, ci = pat.csr()
    orp, oci = oracle.pattern(e, x.shape[0])
    assert np.array_equal(rp.cpu().numpy(), orp)
    assert np.array_equal(ci.cpu().numpy(), oci)


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_values(name, lfem):
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    assert pat.info()["tiles"] > 2 or x.shape[0] < 50 or (d == 3 and p >= 3)
    orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
    out = lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=7, precision=lfem.FP64)
    torch.cuda.synchronize()
    for k, ref in (("M", M), ("A", A), ("MC", C)):
        err = diag_scaled_error(out[k].cpu().numpy(), ref, orp, oci)
        assert err <= FP64_TOL, (k, err)
    pat.sync_status()


@pytest.mark.parametrize("name", list(CASES))
def test_mixed_values(name, lfem):
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
    out = lfem.assemble(pat, to_dev(x), rule, to_dev(coef).float(), which=7, precision=lfem.MIXED)
    torch.cuda.synchronize()
    for k, ref in (("M", M), ("A", A), ("MC", C)):
        v = out[k].double().cpu().numpy()
        assert out[k].dtype == torch.float32
        err = diag_scaled_error(v, ref, orp, oci)
        assert err <= MIXED_TOL, (k, err)
    assert abs(out["M"].double().sum().item() - M.sum()) <= MIXED_TOL * abs(M.sum())


@pytest.mark.parametrize("name", ["perturbed_sphere_p2", "disk_p1", "curve_p2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_unaligned_buffers(name, prec, lfem):
    """Coordinates 8 bytes and outputs one value off a 16-byte boundary: node
    coordinates then arrive by per-node gathers instead of bulk copies and
    phase 2 stores value by value; the result is the aligned one, bit for bit,
    and within the tolerance of the oracle."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
    dt = torch.float64 if prec == 0 else torch.float32
    cd = to_dev(coef).to(dt)
    ref = lfem.assemble(pat, to_dev(x), rule, cd, which=7, precision=prec)
    flat = torch.zeros(x.size + 1, dtype=torch.float64, device="cuda")
    xu = flat[1:].view(x.shape)
    xu.copy_(to_dev(x))
    assert xu.data_ptr() % 16 == 8
    outs = {k: torch.full((pat.nnz + 1,), -1.0, dtype=dt, device="cuda")[1:] for k in ("M", "A", "MC")}
    got = lfem.assemble(pat, xu, rule, cd, which=7, precision=prec, out=outs)
    torch.cuda.synchronize()
    tol = FP64_TOL if prec == 0 else MIXED_TOL
    for k, r in (("M", M), ("A", A), ("MC", C)):
        assert torch.equal(got[k], ref[k]), k
        assert diag_scaled_error(got[k].double().cpu().numpy(), r, orp, oci) <= tol, k
    pat.sync_status()


@pytest.mark.parametrize("name", ["perturbed_sphere_p2", "cube_p2", "cube_p1", "cube_p3"])
def test_mixed_conditioning_threshold(name, lfem):
    """kappa_max = 1 sends every element (metric quality < 1) to the double
    recomputation, INFINITY sends none (no degenerate element here); both
    stay within the mixed tolerance."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
    xd, cd = to_dev(x), to_dev(coef).float()
    for kappa, n_fb in ((1.0, e.shape[0]), (float("inf"), 0)):
        pat.set_mixed_kappa(kappa)
        out = lfem.assemble(pat, xd, rule, cd, which=7, precision=lfem.MIXED)
        assert pat.fallback_count() == n_fb
        for k, ref in (("M", M), ("A", A), ("MC", C)):
            err = diag_scaled_error(out[k].double().cpu().numpy(), ref, orp, oci)
            assert err <= MIXED_TOL, (kappa, k, err)
    pat.sync_status()
    with pytest.raises(lfem.LfemError):
        pat.set_mixed_kappa(0.5)


@pytest.mark.parametrize("name", ["ellipsoid_p2", "cube_p2", "curve_p2", "disk_p1"])
@pytest.mark.parametrize("prec", [0, 1])
def test_deterministic_and_tile_independent(name, prec, lfem):
    """Bit-identical reruns and identical results for every tile capacity: each
    slot is summed in ascending element order whatever the tiling."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem, tile_slots=0)
    xd, cd = to_dev(x), to_dev(coef)
    if prec == 1:
        cd = cd.float()
    ref = lfem.assemble(pat, xd, rule, cd, which=7, precision=prec)
    again = lfem.assemble(pat, xd, rule, cd, which=7, precision=prec)
    for slots in (256, 512, 1024):
        pat.retile(slots)
        for chunk in (32, 96):
            pat.set_launch(chunk, 0)
            other = lfem.assemble(pat, xd, rule, cd, which=7, precision=prec)
            for k in ref:
                assert torch.equal(ref[k], other[k]), (k, slots, chunk)
    for k in ref:
        assert torch.equal(ref[k], again[k])


@pytest.mark.parametrize("name", ["cube_p3", "cube_p4"])
@pytest.mark.parametrize("prec", [0, 1])
def test_tet_high_deterministic_and_subsets(name, prec, lfem):
    """Order-3/4 tets: bit-identical reruns, and each matrix alone equals the
    same matrix assembled with the others."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    xd, cd = to_dev(x), to_dev(coef)
    if prec == 1:
        cd = cd.float()
    ref = lfem.assemble(pat, xd, rule, cd, which=7, precision=prec)
    again = lfem.assemble(pat, xd, rule, cd, which=7, precision=prec)
    for k in ref:
        assert torch.equal(ref[k], again[k])
    for which, k in ((1, "M"), (2, "A"), (4, "MC")):
        part = lfem.assemble(pat, xd, rule, cd, which=which, precision=prec)
        assert list(part) == [k] and torch.equal(part[k], ref[k])


@pytest.mark.parametrize("name", ["sphere_p1", "disk_p1", "cube_p1", "curve_p1"])
def test_p1_exact_reference_matrices(name, lfem):
    """No rule for order 1: the exact reference matrices (Sec. 4.2), against the
    closed-form oracle; LFEM_CMASS still needs a rule."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci, M, A = oracle.p1_exact(x, e, d)
    xd = to_dev(x)
    for prec, tol in ((lfem.FP64, FP64_TOL), (lfem.MIXED, MIXED_TOL)):
        out = lfem.assemble(pat, xd, None, which=3, precision=prec)
        for k, ref in (("M", M), ("A", A)):
            err = diag_scaled_error(out[k].double().cpu().numpy(), ref, orp, oci)
            assert err <= tol, (prec, k, err)
    pat.sync_status()
    with pytest.raises(lfem.LfemError):
        lfem.assemble(pat, xd, None, to_dev(coef), which=4)
    f = np.random.default_rng(3).standard_normal(x.shape[0])
    b = lfem.assemble_load(pat, xd, None, to_dev(f)).cpu().numpy()
    Md = np.zeros((x.shape[0], x.shape[0]))
    Md[np.repeat(np.arange(x.shape[0]), np.diff(orp)), oci] = M
    assert np.abs(b - Md @ f).max() <= 1e-12 * np.abs(Md @ f).max()


@pytest.mark.parametrize("which", [1, 2, 4, 3, 5, 6])
def test_subsets_of_matrices(which, lfem):
    x, e, d, p, rule, coef, pat = prepare("ellipsoid_p2", lfem)
    full = lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=7, precision=0)
    part = lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=which, precision=0)
    for k, bit in (("M", 1), ("A", 2), ("MC", 4)):
        if which & bit:
            assert torch.equal(full[k], part[k])
        else:
            assert k not in part


@pytest.mark.parametrize("name", ["ellipsoid_p2", "cube_p2", "curve_p2", "disk_p1", "space_curve_p2",
                                  "sphere_p3", "sphere_p4", "disk_p3", "circle_p4"])
def test_element_stages(name, lfem):
    x, e, d, p, rule, coef, pat = prepare(name, lfem, tile_slots=0)
    ed, xd = to_dev(e), to_dev(x)
    pts = lfem.eval_points(ed, d, p, xd, rule).cpu().numpy()
    assert np.abs(pts - oracle.eval_points(x, e, d, p, rule.xi)).max() < 1e-14 * max(1, np.abs(x).max())
    J, s, Gi = (t.cpu().numpy() for t in lfem.geometry(ed, d, p, xd, rule))
    oJ, os_, oGi = oracle.geometry(x, e, d, p, rule.xi)
    assert np.abs(J - oJ).max() <= 1e-13 * np.abs(oJ).max()
    assert np.abs(s - os_).max() <= 1e-13 * np.abs(os_).max()
    assert np.abs(Gi - oGi).max() <= 1e-11 * np.abs(oGi).max()
    Ml, Al, Cl = (t.cpu().numpy() for t in lfem.local(ed, d, p, xd, rule, to_dev(coef), which=7))
    oM, oA, oC = oracle.local_matrices(x, e, d, p, rule.xi, rule.w, coef)
    ref = e.shape[1]
    iu = np.triu_indices(ref)
    for got, want in ((Ml, oM), (Al, oA), (Cl, oC)):
        w = want[:, iu[0], iu[1]]
        assert np.abs(got - w).max() <= 1e-12 * np.abs(w).max()


def test_element_stages_reject_high_order_tets(lfem):
    """Order-3/4 tets keep their basis tables on the device: the stages say so."""
    x, e, d, p, rule, coef, pat = prepare("cube_p3", lfem, tile_slots=0)
    with pytest.raises(lfem.LfemError) as ei:
        lfem.eval_points(to_dev(e), d, p, to_dev(x), rule)
    assert ei.value.code == 3


@pytest.mark.parametrize("name", ["ellipsoid_p2", "cube_p2", "curve_p2", "disk_p2", "sphere_p1", "space_curve_p2"])
def test_adjoint_matches_oracle(name, lfem):
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci = oracle.pattern(e, x.shape[0])
    rng = np.random.default_rng(17)
    gM, gA, gC = rng.normal(size=(3, oci.size))
    gx, gc = lfem.assemble_adjoint(pat, to_dev(x), rule, to_dev(coef), to_dev(gM), to_dev(gA), to_dev(gC),
                                   want_coef_grad=True)
    ogx, ogc = oracle.adjoint(x, e, d, p, rule.xi, rule.w, coef, (orp, oci), gM, gA, gC)
    assert np.abs(gx.cpu().numpy() - ogx).max() <= 1e-10 * np.abs(ogx).max()
    assert np.abs(gc.cpu().numpy() - ogc).max() <= 1e-11 * np.abs(ogc).max()


@pytest.mark.parametrize("name", ["ellipsoid_p2", "cube_p2", "curve_p2", "disk_p2", "sphere_p1", "space_curve_p2"])
def test_mixed_adjoint_matches_oracle(name, lfem):
    """The mixed adjoint (FP32 geometry, double node sums, double recomputation of
    badly conditioned elements) within 1e-6 of the oracle, relative to max |g|."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci = oracle.pattern(e, x.shape[0])
    rng = np.random.default_rng(17)
    gM, gA, gC = rng.normal(size=(3, oci.size))
    gx, gc = lfem.assemble_adjoint(pat, to_dev(x), rule, to_dev(coef), to_dev(gM), to_dev(gA), to_dev(gC),
                                   want_coef_grad=True, precision=lfem.MIXED)
    ogx, ogc = oracle.adjoint(x, e, d, p, rule.xi, rule.w, coef, (orp, oci), gM, gA, gC)
    assert np.abs(gx.cpu().numpy() - ogx).max() <= 1e-6 * np.abs(ogx).max()
    assert np.abs(gc.cpu().numpy() - ogc).max() <= 1e-6 * np.abs(ogc).max()
    # kappa = 1: every element of dimension >= 2 is recomputed in double
    pat.set_mixed_kappa(1.0)
    gx1, _ = lfem.assemble_adjoint(pat, to_dev(x), rule, to_dev(coef), to_dev(gM), to_dev(gA), to_dev(gC),
                                   precision=lfem.MIXED)
    if d >= 2:
        assert pat.fallback_count() == e.shape[0]
        assert np.abs(gx1.cpu().numpy() - ogx).max() <= 1e-10 * np.abs(ogx).max()


@pytest.mark.parametrize("name", ["sphere_p3", "sphere_p4", "disk_p3", "circle_p4", "cube_p3", "cube_p4"])
def test_adjoint_high_orders_match_oracle(name, lfem):
    """Orders 3, 4 (warp per element, double): the node and coefficient gradients
    within 1e-10 of the oracle; the mixed request runs the same double path and
    counts every element as recomputed; reruns are bit-identical."""
    x, e, d, p, rule, coef, pat = prepare(name, lfem)
    orp, oci = oracle.pattern(e, x.shape[0])
    rng = np.random.default_rng(23)
    gM, gA, gC = rng.normal(size=(3, oci.size))
    args = (pat, to_dev(x), rule, to_dev(coef), to_dev(gM), to_dev(gA), to_dev(gC))
    gx, gc = lfem.assemble_adjoint(*args, want_coef_grad=True)
    ogx, ogc = oracle.adjoint(x, e, d, p, rule.xi, rule.w, coef, (orp, oci), gM, gA, gC)
    assert np.abs(gx.cpu().numpy() - ogx).max() <= 1e-10 * np.abs(ogx).max()
    assert np.abs(gc.cpu().numpy() - ogc).max() <= 1e-11 * np.abs(ogc).max()
    gx2, gc2 = lfem.assemble_adjoint(*args, want_coef_grad=True, precision=lfem.MIXED)
    assert pat.fallback_count() == e.shape[0]
    assert torch.equal(gx, gx2) and torch.equal(gc, gc2)
    # only the stiffness gradient, no coefficient
    gxa, _ = lfem.assemble_adjoint(pat, to_dev(x), rule, None, None, to_dev(gA), None)
    oga, _ = oracle.adjoint(x, e, d, p, rule.xi, rule.w, None, (orp, oci), None, gA, None)
    assert np.abs(gxa.cpu().numpy() - oga).max() <= 1e-10 * np.abs(oga).max()


def test_autograd_function(lfem):
    """AssembleFn backward against the oracle adjoint of L = u^T M u + v^T A v + w^T MC w."""
    x, e, d, p, rule, coef, pat = prepare("ellipsoid_p2", lfem)
    rng = np.random.default_rng(3)
    u, v, w = (to_dev(rng.normal(size=x.shape[0])) for _ in range(3))
    rp, ci = pat.csr()
    rows = torch.repeat_interleave(torch.arange(x.shape[0], device="cuda"), rp[1:] - rp[:-1])
    xt = to_dev(x).requires_grad_(True)
    ct = to_dev(coef).requires_grad_(True)
    M, A, MC = lfem.AssembleFn.apply(xt, ct, pat, rule)
    L = (M * u[rows] * u[ci]).sum() + (A * v[rows] * v[ci]).sum() + (MC * w[rows] * w[ci]).sum()
    L.backward()
    orp, oci = rp.cpu().numpy(), ci.cpu().numpy()
    rr = rows.cpu().numpy()
    un, vn, wn = u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy()
    ogx, ogc = oracle.adjoint(x, e, d, p, rule.xi, rule.w, coef, (orp, oci), un[rr] * un[oci], vn[rr] * vn[oci],
                              wn[rr] * wn[oci])
    assert np.abs(xt.grad.cpu().numpy() - ogx).max() <= 1e-10 * np.abs(ogx).max()
    assert np.abs(ct.grad.cpu().numpy() - ogc).max() <= 1e-10 * np.abs(ogc).max()


def test_bounded_wait_reports_timeout(lfem):
    """A wait that nothing completes (the first CTA skips its copy) gives up after
    its bound, the status word reports LFEM_E_TIMEOUT, and the context stays usable."""
    x, e, d, p, rule, coef, pat = prepare("ellipsoid_p2", lfem)
    ref = lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=7, precision=lfem.MIXED)
    pat.debug_starve_wait(True)
    lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=7, precision=lfem.MIXED)
    with pytest.raises(lfem.LfemError) as ei:
        pat.sync_status()
    assert ei.value.code == 8
    pat.debug_starve_wait(False)
    again = lfem.assemble(pat, to_dev(x), rule, to_dev(coef), which=7, precision=lfem.MIXED)
    pat.sync_status()
    for k in ref:
        assert torch.equal(ref[k], again[k])


def test_edge_cases(lfem):
    # empty mesh: every row empty
    pat = lfem.Pattern(torch.empty(0, 3, dtype=torch.int32, device="cuda"), 5, 2, 1)
    rp, ci = pat.csr()
    assert pat.nnz == 0 and rp.cpu().tolist() == [0] * 6
    out = lfem.assemble(pat, torch.zeros(5, 3, dtype=torch.float64, device="cuda"), CASES["sphere_p1"][4])
    assert out["M"].numel() == 0
    # one element, unused nodes, repeated node (degenerate -> status, M still finite)
    conn = np.array([[0, 2, 5]], dtype=np.int32)
    x = np.random.default_rng(0).normal(size=(7, 3))
    pat = lfem.Pattern(to_dev(conn), 7, 2, 1)
    rp, ci = pat.csr()
    orp, oci = oracle.pattern(conn, 7)
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(ci.cpu().numpy(), oci)
    rule = CASES["sphere_p1"][4]
    out = lfem.assemble(pat, to_dev(x), rule, which=3)
    _, _, M, A, _ = oracle.assemble(x, conn, 2, 1, rule.xi, rule.w)
    assert np.abs(out["M"].cpu().numpy() - M).max() < 1e-14 and np.abs(out["A"].cpu().numpy() - A).max() < 1e-12
    pat.sync_status()
    dup = np.array([[0, 2, 2]], dtype=np.int32)
    pat = lfem.Pattern(to_dev(dup), 7, 2, 1)
    assert np.array_equal(pat.csr()[1].cpu().numpy(), oracle.pattern(dup, 7)[1])
    out = lfem.assemble(pat, to_dev(x), rule, which=1)
    with pytest.raises(lfem.LfemError) as ei:
        pat.sync_status()
    assert ei.value.code == 7
    assert np.all(np.abs(out["M"].cpu().numpy()) < 1e-15)
    pat.sync_status()  # cleared
    out = lfem.assemble(pat, to_dev(x), rule, which=1, precision=lfem.MIXED)
    with pytest.raises(lfem.LfemError) as ei:
        pat.sync_status()
    assert ei.value.code == 7
    # index out of range is reported by the pattern build
    for bad in ([[0, 1, 7]], [[0, -1, 2]]):
        with pytest.raises(lfem.LfemError) as ei:
            lfem.Pattern(to_dev(np.array(bad, dtype=np.int32)), 7, 2, 1)
        assert ei.value.code == 2
    # invalid arguments
    with pytest.raises(lfem.LfemError) as ei:
        lfem.assemble(pat, to_dev(x[:, :1].copy()), rule, which=1)  # ambient 1 < dim 2
    assert ei.value.code == 3
    with pytest.raises(lfem.LfemError) as ei:
        lfem.assemble(pat, to_dev(x), rule, which=4)  # weighted mass without a coefficient
    assert ei.value.code == 1
    with pytest.raises(lfem.LfemError) as ei:
        lfem.Pattern(to_dev(conn), 7, 4, 1)
    assert ei.value.code == 3


def test_tet_high_edge_cases(lfem):
    """Order-3/4 tets: an empty mesh, a single reference element (against the
    oracle, both precisions), a flattened element (status LFEM_E_DEGENERATE in
    both precisions), node generation on one tet, and an empty order-1 mesh
    without a rule."""
    from paper_2605_14035_gb300.inputs import meshes

    rule = CASES["cube_p3"][4]
    for p in (3, 4):
        ref = (p + 1) * (p + 2) * (p + 3) // 6
        pat = lfem.Pattern(torch.empty(0, ref, dtype=torch.int32, device="cuda"), 5, 3, p)
        assert pat.nnz == 0
        xd = torch.zeros(5, 3, dtype=torch.float64, device="cuda")
        for prec in (lfem.FP64, lfem.MIXED):
            out = lfem.assemble(pat, xd, rule, which=3, precision=prec)
            assert out["M"].numel() == 0 and out["A"].numel() == 0
        assert torch.equal(lfem.assemble_load(pat, xd, rule, torch.ones(5, dtype=torch.float64, device="cuda")),
                           torch.zeros(5, dtype=torch.float64, device="cuda"))
        pat.sync_status()
        # one tet with its generated nodes, plus an unused node
        x1 = np.vstack([np.zeros(3), np.eye(3)]) * np.array([1.0, 0.8, 1.3]) + 0.1
        x, e = meshes.to_order(x1, np.array([[0, 1, 2, 3]], dtype=np.int32), p)
        x = np.vstack([x, [[5.0, 5.0, 5.0]]])
        pat = lfem.Pattern(to_dev(e), x.shape[0], 3, p)
        orp, oci, M, A, _ = oracle.assemble(x, e, 3, p, rule.xi, rule.w)
        assert np.array_equal(pat.csr()[1].cpu().numpy(), oci)
        for prec, tol in ((lfem.FP64, FP64_TOL), (lfem.MIXED, MIXED_TOL)):
            out = lfem.assemble(pat, to_dev(x), rule, which=3, precision=prec)
            for k, r in (("M", M), ("A", A)):
                assert diag_scaled_error(out[k].double().cpu().numpy(), r, orp, oci) <= tol, (p, prec, k)
        pat.sync_status()
        # every node on one plane: zero volume
        xf = x.copy()
        xf[:, 2] = 0.0
        for prec in (lfem.FP64, lfem.MIXED):
            lfem.assemble(pat, to_dev(xf), rule, which=1, precision=prec)
            with pytest.raises(lfem.LfemError) as ei:
                pat.sync_status()
            assert ei.value.code == 7
        # node generation on a single tet
        p1 = lfem.Pattern(to_dev(np.array([[0, 1, 2, 3]], dtype=np.int32)), 4, 3, 1)
        xg, eg = lfem.lift_order(p1, to_dev(x1), p)
        assert np.array_equal(eg.cpu().numpy(), e) and np.array_equal(xg.cpu().numpy(), x[:-1])
    pat = lfem.Pattern(torch.empty(0, 3, dtype=torch.int32, device="cuda"), 4, 2, 1)
    out = lfem.assemble(pat, torch.zeros(4, 3, dtype=torch.float64, device="cuda"), None, which=3)
    assert out["M"].numel() == 0
