"""Load vector (Sec. 2), the non-linear vectors of the mean curvature flow
system (Sec. 5.1) and one step of Dziuk's scheme on the GPU against the FP64
oracle, on the same seeded inputs."""
import numpy as np
import pytest
import torch

import oracle
from cases import build_cases

pytestmark = pytest.mark.gpu

CASES = build_cases()
TOL = 1e-12  # relative to max |reference|
SURFACES = ["sphere_p1", "ellipsoid_p2", "perturbed_sphere_p2", "cube_boundary_p2", "sphere_p2_gauss9"]


@pytest.fixture(scope="module")
def lfem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14035_gb300 import lfem as m

    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_load_vector(name, lfem):
    x, e, d, p, rule = CASES[name]
    f = np.random.default_rng(31).standard_normal(x.shape[0])
    ref = oracle.load(x, e, d, p, rule.xi, rule.w, f)
    pat = lfem.Pattern(dev(e), x.shape[0], d, p)
    b = lfem.assemble_load(pat, dev(x), rule, dev(f))
    again = lfem.assemble_load(pat, dev(x), rule, dev(f))
    got = b.cpu().numpy()
    assert np.abs(got - ref).max() <= TOL * np.abs(ref).max()
    assert torch.equal(b, again)


@pytest.mark.parametrize("name", SURFACES)
def test_mcf_nonlinear_vectors(name, lfem):
    x, e, d, p, rule = CASES[name]
    rng = np.random.default_rng(32)
    # a smooth field plus noise (any nodal field is a valid input; unit length is not required)
    nu = np.column_stack([np.sin(3 * x[:, 1]), np.cos(2 * x[:, 2]), x[:, 0] * x[:, 1]]) + 0.05 * rng.standard_normal(
        x.shape)
    u = np.column_stack([nu, rng.standard_normal(x.shape[0])])
    ref = oracle.kll(x, e, p, rule.xi, rule.w, u)
    pat = lfem.Pattern(dev(e), x.shape[0], d, p)
    out = lfem.assemble_mcf_nonlinear(pat, dev(x), rule, dev(u)).cpu().numpy()
    assert np.abs(out - ref).max() <= TOL * np.abs(ref).max()


def test_vectors_edge_cases(lfem):
    x, e, d, p, rule = CASES["curve_p2"]
    pat = lfem.Pattern(dev(e), x.shape[0], d, p)
    with pytest.raises(lfem.LfemError):
        lfem.assemble_mcf_nonlinear(pat, dev(x), rule, dev(np.zeros((x.shape[0], 4))))
    # an unreferenced node gets b = 0
    xs, es, ds, ps, rs = CASES["sphere_p1"]
    xs = np.vstack([xs, [[5.0, 5.0, 5.0]]])
    pat = lfem.Pattern(dev(es), xs.shape[0], ds, ps)
    b = lfem.assemble_load(pat, dev(xs), rs, dev(np.ones(xs.shape[0]))).cpu().numpy()
    assert b[-1] == 0.0
    assert abs(b[:-1].sum() - oracle.load(xs, es, ds, ps, rs.xi, rs.w, np.ones(xs.shape[0])).sum()) < 1e-12


@pytest.mark.parametrize("name", ["ellipsoid_p2", "perturbed_sphere_p2", "sphere_p1", "curve_p2", "cube_boundary_p2"])
def test_mcf_step(name, lfem):
    x, e, d, p, rule = CASES[name]
    tau = 1e-3
    ref = oracle.mcf_step(x, e, d, p, rule.xi, rule.w, tau)
    pat = lfem.Pattern(dev(e), x.shape[0], d, p)
    xd = dev(x)
    x1, it = lfem.mcf_step(pat, xd, rule, tau, rtol=1e-13, max_iter=5000)
    again, it2 = lfem.mcf_step(pat, xd, rule, tau, rtol=1e-13, max_iter=5000)
    assert it < 5000 and it == it2
    got = x1.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()
    assert torch.equal(x1, again)
    # in place
    xin = xd.clone()
    lfem.mcf_step(pat, xin, rule, tau, rtol=1e-13, max_iter=5000, out=xin)
    assert torch.equal(xin, x1)
    # on a side stream the 8-iteration blocks replay a captured graph: the same
    # kernels, so the same bits (first call captures, second replays)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):
            xs, its = lfem.mcf_step(pat, xd, rule, tau, rtol=1e-13, max_iter=5000, stream=stream)
            stream.synchronize()
            assert its == it and torch.equal(xs, x1)
        # a cap that is not a multiple of the check interval ends on direct launches
        xc, itc = lfem.mcf_step(pat, xd, rule, tau, rtol=1e-30, max_iter=13, stream=stream)
        stream.synchronize()
    xd13, itd = lfem.mcf_step(pat, xd, rule, tau, rtol=1e-30, max_iter=13)
    assert itc == itd == 13 and torch.equal(xc, xd13)


@pytest.mark.parametrize("kind,order", [("sphere", 3), ("sphere", 4), ("disk", 3), ("disk", 4), ("circle", 4),
                                        ("sphere", 2), ("cube", 2), ("cube", 3), ("cube", 4), ("cube_jit", 4)])
def test_lift_order_matches_the_cpu_generator(kind, order, lfem):
    """GPU node generation (P1 -> order p) against the oracle's node generation
    (oracle.lift_order, pinned to the documented barycentric positions and
    numbering): identical connectivity and identical coordinate bits."""
    from paper_2605_14035_gb300.inputs import meshes

    if kind == "sphere":
        x, e = meshes.icosphere(2, 1)
    elif kind == "disk":
        x, e = meshes.hex_disk(5, 1)
    elif kind == "cube":
        x, e = meshes.kuhn_cube_p2(3, order=1)
    elif kind == "cube_jit":
        x, e = meshes.kuhn_cube_p2(4, jitter=0.2, seed=meshes.BASE_SEED + 21, order=1)
    else:
        t = 2 * np.pi * np.arange(30) / 30
        x = np.stack([np.cos(t), np.sin(t)], axis=1)
        e = np.stack([np.arange(30), (np.arange(30) + 1) % 30], axis=1).astype(np.int32)
    xr, er = oracle.lift_order(x, e, order)
    pat = lfem.Pattern(dev(e), x.shape[0], e.shape[1] - 1, 1)
    xg, eg = lfem.lift_order(pat, dev(x), order)
    assert np.array_equal(eg.cpu().numpy(), er)
    assert np.array_equal(xg.cpu().numpy(), xr)
