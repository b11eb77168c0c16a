"""Batched assembly (one persistent launch over many meshes of different element
types) and its CUDA-graph replay, against single-mesh assembly and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from cases import build_cases, coef_field, diag_scaled_error

pytestmark = pytest.mark.gpu

NAMES = ["curve_p1", "curve_p2", "disk_p1", "disk_p2", "sphere_p1", "ellipsoid_p2", "half_disk_p2"]
HIGH = ["sphere_p3", "disk_p3", "circle_p4", "sphere_p4"]


@pytest.fixture(scope="module")
def lfem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_14035_gb300 import lfem as m

    return m


def make_batch(lfem, which=7, tile_slots=512, names=NAMES):
    cases = build_cases()
    meshes, meta = [], []
    for name in names:
        x, e, d, p, rule = cases[name]
        coef = coef_field(oracle.eval_points(x, e, d, p, rule.xi))
        pat = lfem.Pattern(torch.from_numpy(e).cuda(), x.shape[0], d, p)
        pat.retile(tile_slots)
        meshes.append({"pattern": pat, "coords": torch.from_numpy(x).cuda(), "rule": rule,
                       "coef": torch.from_numpy(coef).float().cuda()})
        meta.append((x, e, d, p, rule, coef))
    return lfem.Batch(meshes, which=which), meshes, meta


def test_batch_matches_single_mesh_and_oracle(lfem):
    batch, meshes, meta = make_batch(lfem)
    assert batch.info()["work_items"] > len(NAMES)
    batch.assemble()
    batch.sync_status()
    for i, m in enumerate(meshes):
        single = lfem.assemble(m["pattern"], m["coords"], m["rule"], m["coef"], which=7, precision=lfem.MIXED)
        got = batch.outputs(i)
        for k in ("M", "A", "MC"):
            assert torch.equal(got[k], single[k]), (NAMES[i], k)
        x, e, d, p, rule, coef = meta[i]
        orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
        for k, ref in (("M", M), ("A", A), ("MC", C)):
            assert diag_scaled_error(got[k].double().cpu().numpy(), ref, orp, oci) <= 1e-6, (NAMES[i], k)


def test_batch_graph_replay_follows_coordinates(lfem):
    batch, meshes, meta = make_batch(lfem, which=3)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.graph_launch(stream)
        stream.synchronize()
        first = [{k: v.clone() for k, v in batch.outputs(i).items()} for i in range(len(meshes))]
        # move every node, replay the captured graph, compare with fresh single-mesh assemblies
        for m in meshes:
            m["coords"].mul_(1.25)
        batch.graph_launch(stream)
        stream.synchronize()
    batch.sync_status(stream)
    for i, m in enumerate(meshes):
        fresh = lfem.assemble(m["pattern"], m["coords"], m["rule"], which=3, precision=lfem.MIXED)
        got = batch.outputs(i)
        for k in ("M", "A"):
            assert torch.equal(got[k], fresh[k]), (NAMES[i], k)
            assert not torch.equal(got[k], first[i][k])


def test_batch_with_orders_3_and_4(lfem):
    """Order-3/4 items beside the persistent launch: bit-identical to their single
    assembly, within 1e-6 of the oracle, and followed by the graph replay."""
    names = ["disk_p2"] + HIGH + ["curve_p1"]
    batch, meshes, meta = make_batch(lfem, which=7, names=names)
    batch.assemble()
    batch.sync_status()
    assert batch.info()["elements_computed"] >= sum(m[1].shape[0] for m in meta)
    for i, m in enumerate(meshes):
        single = lfem.assemble(m["pattern"], m["coords"], m["rule"], m["coef"], which=7, precision=lfem.MIXED)
        x, e, d, p, rule, coef = meta[i]
        orp, oci, M, A, C = oracle.assemble(x, e, d, p, rule.xi, rule.w, coef)
        for k, ref in (("M", M), ("A", A), ("MC", C)):
            got = batch.outputs(i)[k]
            assert torch.equal(got, single[k]), (names[i], k)
            assert diag_scaled_error(got.double().cpu().numpy(), ref, orp, oci) <= 1e-6, (names[i], k)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        batch.graph_launch(stream)
        for m in meshes:
            m["coords"].mul_(0.75)
        batch.graph_launch(stream)
        stream.synchronize()
    batch.sync_status(stream)
    for i, m in enumerate(meshes):
        fresh = lfem.assemble(m["pattern"], m["coords"], m["rule"], m["coef"], which=7, precision=lfem.MIXED)
        for k in ("M", "A", "MC"):
            assert torch.equal(batch.outputs(i)[k], fresh[k]), (names[i], k)


def test_batch_rejects_tets(lfem):
    cases = build_cases()
    x, e, d, p, rule = cases["cube_p2"]
    pat = lfem.Pattern(torch.from_numpy(e).cuda(), x.shape[0], d, p)
    with pytest.raises(lfem.LfemError) as ei:
        lfem.Batch([{"pattern": pat, "coords": torch.from_numpy(x).cuda(), "rule": rule}], which=1)
    assert ei.value.code == 3


def test_batch_autotune_per_family_and_cache(lfem, tmp_path):
    """lfem_batch_autotune picks a capacity per element family (dim, order) from
    its candidates, leaves every pattern at it, writes the cache and reads it
    back; the batch made afterwards still matches single-mesh assembly bit for
    bit."""
    _, meshes, meta = make_batch(lfem, which=3)
    spec = [{k: m[k] for k in ("pattern", "coords", "rule")} for m in meshes]
    cache = str(tmp_path / "batch_tune.txt")
    best = lfem.batch_autotune(spec, which=3, cache_path=cache)
    cand = {1024, 1536, 2048, 2304, 2560, 3072}
    assert all(v in cand for v in best)  # every family is present in this batch
    for name, (x, e, d, p, rule, coef) in zip(NAMES, meta):
        want = best[2 * (d - 1) + (p - 1)]
        info = meshes[NAMES.index(name)]["pattern"].info()
        assert info["tile_slots"] == max(want, info["max_row"]), name
    text = open(cache).read().split()
    assert text[1:] == [str(v) for v in best] and text[0].startswith("batch_w3")
    # a second call reads the cache: the same answer
    assert lfem.batch_autotune(spec, which=3, cache_path=cache) == best
    batch = lfem.Batch(spec, which=3)
    batch.assemble()
    batch.sync_status()
    for i, m in enumerate(meshes):
        single = lfem.assemble(m["pattern"], m["coords"], m["rule"], which=3, precision=lfem.MIXED)
        for k in ("M", "A"):
            assert torch.equal(batch.outputs(i)[k], single[k]), (NAMES[i], k)
