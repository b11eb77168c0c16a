"""Further workloads of bench.py (--workload c1 | c3 | c4 | c5 | c2q16 | p4).

c1  P1 icosphere, 5 refinements (20,480 triangles): FP64 mass + stiffness,
    3-point rule; launch-bound, so also the same assembly replayed from a CUDA
    graph (one-mesh batch, mixed precision).
c3  P2 Kuhn cube 64^3 (1,572,864 ten-node tets, jittered) mass + stiffness with
    the 14-point rule, plus the boundary surface mass on its 49,152 P2
    triangles; FP64 and mixed.
c4  512 meshes of uneven size (P2 curves, P1/P2 disks, P2 spheres; about 77 M
    elements), mass + stiffness, mixed precision, one persistent launch per
    batch replayed from a CUDA graph, tile capacity picked by timing; against
    the plain FP64 path mesh by mesh.
c5  evolving P2 ellipsoid (327,680 triangles): 100 steps of reassembly of M(x),
    A(x) (graph replay) with nodes moved along the discrete normal flow, then
    the adjoint of L = u^T M u + v^T A v through the autograd function; on the
    final surface also the load vector, the flow's non-linear vectors and one
    step of Dziuk's scheme (FP64 assembly + hand-written PCG), each against the
    oracle.
c2q16  the C2 surface with the 16-point degree-8 rule (the rule size the paper
    uses for P2), mass + stiffness through the general element path.
p4  order 4 on the sphere: the level-6 P1 icosphere lifted to order 4 on the GPU,
    projected, mass + stiffness with the 16-point rule.
Each prints one JSON line.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

import bench


def _line(args, workload, value, unit, ms, extra):
    d = {"metric": "elements/s", "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": extra.pop("dtype", "f32+f64"), "data": "synthetic",
         "config": {"workload": workload, **extra.pop("config", {})}}
    d.update(extra)
    print(json.dumps(d), flush=True)


def _timer(torch, flush):
    def timed(fn, steps, warmup, stream=None):
        st = stream or torch.cuda.current_stream()
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            if flush is not None:
                flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            ms.append((a, b))
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ms) / steps

    return timed


def run_c1(args):
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x, e = meshes.icosphere(5, 1)
    rule = quadrature.tri_3pt_deg2()
    xd, ed = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda()
    pat = lfem.Pattern(ed, x.shape[0], 2, 1)
    timed = _timer(torch, None)
    out = {k: torch.empty(pat.nnz, dtype=torch.float64, device="cuda") for k in ("M", "A")}
    ms64 = timed(lambda: lfem.assemble(pat, xd, rule, which=3, precision=lfem.FP64, out=out), args.steps * 10, 10)
    batch = lfem.Batch([{"pattern": pat, "coords": xd, "rule": rule}], which=3)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ms_graph = timed(lambda: batch.graph_launch(s), args.steps * 10, 10, stream=s)
    batch.sync_status(s)
    area = float(out["M"].sum())
    _line(args, "p1_icosphere_r5_M_A", x.shape[0] and e.shape[0] / (ms64 * 1e-3), "elements/s", ms64,
          {"dtype": "f64", "config": {"elements": int(e.shape[0]), "nnz_per_matrix": pat.nnz, "l2": "resident"},
           "mixed_graph": {"value": e.shape[0] / (ms_graph * 1e-3), "ms_per_step": ms_graph},
           "area_minus_4pi": area - 4 * np.pi})


def run_c3(args):
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x, e = meshes.kuhn_cube_p2(64)
    b = meshes.boundary_faces_p2(e)
    r_tet, r_tri = quadrature.tet_14pt_deg5(), quadrature.tri_7pt_deg5()
    xd, ed, bd = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(b).cuda()
    pt = lfem.Pattern(ed, x.shape[0], 3, 2)
    pb = lfem.Pattern(bd, x.shape[0], 2, 2)
    flush = torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    timed = _timer(torch, flush)
    res = {}
    for prec, dt, name in ((lfem.MIXED, torch.float32, "mixed"), (lfem.FP64, torch.float64, "fp64")):
        ot = {k: torch.empty(pt.nnz, dtype=dt, device="cuda") for k in ("M", "A")}
        ob = {"M": torch.empty(pb.nnz, dtype=dt, device="cuda")}

        def step():
            lfem.assemble(pt, xd, r_tet, which=3, precision=prec, out=ot)
            lfem.assemble(pb, xd, r_tri, which=1, precision=prec, out=ob)

        ms = timed(step, args.steps, args.warmup)
        res[name] = {"ms_per_step": ms, "value": (e.shape[0] + b.shape[0]) / (ms * 1e-3),
                     "volume": float(ot["M"].double().sum()), "boundary_area": float(ob["M"].double().sum()),
                     "fp64_fallback_tets": pt.fallback_count() if prec == lfem.MIXED else 0}
        pt.sync_status()
    alg = e.shape[0] * 40 + x.shape[0] * 24 + 2 * pt.nnz * 4 + b.shape[0] * 24 + pb.nnz * 4
    peak, kind = bench.measured_peaks()
    ach = alg / (res["mixed"]["ms_per_step"] * 1e-3) / 1e9
    tflops = e.shape[0] * TET_P2_FLOPS / (res["mixed"]["ms_per_step"] * 1e-3) / 1e12
    _line(args, "p2_kuhn_cube_64_tets_M_A_plus_boundary_M", res["mixed"]["value"], "elements/s",
          res["mixed"]["ms_per_step"],
          {"config": {"tets": int(e.shape[0]), "boundary_triangles": int(b.shape[0]), "nnz_tets": pt.nnz,
                      "l2": "flushed between steps"},
           "fp64": res["fp64"], "mixed": res["mixed"],
           # tets are bound by FP32 arithmetic: about 6.1k multiply-adds + 0.8k multiplies per P2 tet
           # (M + A, 14 points; counted from the element code) against the FP32 pipe peak
           "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": tflops / FP32_PEAK_TFLOPS, "traffic": None, "flops_per_tet": TET_P2_FLOPS,
                        "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"},
           "roofline_hbm": {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                            "algorithmic_bytes": alg, "peak_kind": kind}})


FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
TET_P2_FLOPS = 12950


def _gen_batch(n_meshes, scale):
    """Generate the batch in a spawn process pool (no GPU is touched before)."""
    import multiprocessing as mp

    from paper_2605_14035_gb300.inputs import meshes

    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.starmap(meshes.batch_item, [(i, n_meshes, scale) for i in range(n_meshes)])


def measure_batch(args):
    """The 512-mesh batch (curves, planar disks, spheres; mixed precision, M + A):
    generated in a spawn pool, patterns built, tile capacities tuned per element
    family by the library (lfem_batch_autotune), then one persistent launch per
    step replayed as a CUDA graph, against the plain FP64 path mesh by mesh."""
    t0 = time.time()
    items = _gen_batch(args.batch_meshes, args.batch_scale)
    t_gen = time.time() - t0
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import quadrature

    rules = {1: quadrature.gauss_interval(3), (2, 1): quadrature.tri_3pt_deg2(), (2, 2): quadrature.tri_7pt_deg5()}
    torch.cuda.synchronize()
    t0 = time.time()
    mesh_list = []
    n_el = 0
    alg = 0
    for fam, x, e, d, p in items:
        xd, ed = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda()
        pat = lfem.Pattern(ed, x.shape[0], d, p)
        rule = rules[1] if d == 1 else rules[(d, p)]
        mesh_list.append({"pattern": pat, "coords": xd, "rule": rule})
        n_el += e.shape[0]
        alg += e.nbytes + x.nbytes + 2 * pat.nnz * 4
    torch.cuda.synchronize()
    t_pat = time.time() - t0
    del items
    s = torch.cuda.Stream()
    timed = _timer(torch, torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda"))
    t0 = time.time()
    if args.no_autotune:
        for m in mesh_list:
            m["pattern"].retile(2304)
        slots = (2304, 2304, 2304, 2304)
    else:
        slots = lfem.batch_autotune(mesh_list, which=3)
    t_tune = time.time() - t0
    batch = lfem.Batch(mesh_list, which=3)
    with torch.cuda.stream(s):
        ms = timed(lambda: batch.graph_launch(s), args.steps, args.warmup, stream=s)
        # one more step, untimed and by direct launches, inside an NVTX range: the
        # launches an ncu capture of the batch's DRAM traffic selects
        torch.cuda.nvtx.range_push("batch_step")
        batch.assemble(s)
        torch.cuda.nvtx.range_pop()
    batch.sync_status(s)
    binfo = batch.info()
    del batch
    # plain FP64 path, mesh by mesh (same matrices; its double local matrices
    # need smaller tiles: a 2048-slot tile of a P1 disk holds ~1,100 elements)
    for m in mesh_list:
        m["pattern"].retile(1024)
    outs = [{k: torch.empty(m["pattern"].nnz, dtype=torch.float64, device="cuda") for k in ("M", "A")}
            for m in mesh_list]

    def fp64_all():
        for m, o in zip(mesh_list, outs):
            lfem.assemble(m["pattern"], m["coords"], m["rule"], which=3, precision=lfem.FP64, out=o)

    ms64 = timed(fp64_all, max(2, args.steps // 4), 1)
    del outs, mesh_list
    torch.cuda.empty_cache()
    peak, kind = bench.measured_peaks()
    ach = alg / (ms * 1e-3) / 1e9
    traffic = bench.measured_traffic(bench.BATCH_KERNEL, "batch_512_meshes_M_A_tiles" + "-".join(str(v) for v in slots),
                                     bench.BATCH_SOURCES)
    return {"workload": "batch_512_meshes_M_A", "value": n_el / (ms * 1e-3), "unit": "elements/s",
            "ms_per_step": ms, "meshes": args.batch_meshes, "elements": int(n_el),
            "tile_slots": {"curves_p1": slots[0], "curves_p2": slots[1], "triangles_p1": slots[2],
                           "triangles_p2": slots[3]}, "work_items": binfo["work_items"],
            "l2": "flushed between steps", "generation_s": round(t_gen, 1), "pattern_build_s": round(t_pat, 1),
            "tuning_s": round(t_tune, 1),
            "fp64_plain_per_mesh": {"value": n_el / (ms64 * 1e-3), "ms_per_step": ms64},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "traffic": traffic, "traffic_unit": "DRAM bytes per step (ncu, every launch of one step)",
                         "algorithmic_bytes": int(alg), "peak_kind": kind}}


def run_c4(args):
    r = measure_batch(args)
    _line(args, r["workload"], r["value"], "elements/s", r["ms_per_step"],
          {"config": {k: r[k] for k in ("meshes", "elements", "tile_slots", "work_items", "l2", "generation_s",
                                         "pattern_build_s", "tuning_s")},
           "fp64_plain_per_mesh": r["fp64_plain_per_mesh"], "roofline": r["roofline"]})


def run_c5(args):
    import torch

    import oracle
    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x, e = meshes.ellipsoid(7)
    rule = quadrature.tri_7pt_deg5()
    N = x.shape[0]
    xd, ed = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda()
    pat = lfem.Pattern(ed, N, 2, 2)
    rp, ci = pat.csr()
    crow = rp
    col = ci.long()
    tau, steps = 1e-6, 100
    s = torch.cuda.Stream()
    batch = lfem.Batch([{"pattern": pat, "coords": xd, "rule": rule}], which=3)
    ev = []
    with torch.cuda.stream(s):
        for k in range(steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            batch.graph_launch(s)
            b.record(s)
            ev.append((a, b))
            out = batch.outputs(0)
            A = torch.sparse_csr_tensor(crow, col, out["A"].double(), size=(N, N))
            Mabs = torch.sparse_csr_tensor(crow, col, out["M"].double().abs(), size=(N, N))
            Dm = Mabs @ torch.ones(N, dtype=torch.float64, device="cuda")
            xd.sub_(tau * (A @ xd) / Dm[:, None])
    torch.cuda.synchronize()
    batch.sync_status(s)
    ms_step = sum(a.elapsed_time(b) for a, b in ev[5:]) / (steps - 5)
    o32 = {k: torch.empty(pat.nnz, dtype=torch.float32, device="cuda") for k in ("M", "A")}
    lfem.assemble(pat, xd, rule, which=3, precision=lfem.MIXED, out=o32)
    fallback = pat.fallback_count()
    # plain FP64 reassembly of the final surface for comparison
    timed = _timer(torch, None)
    o64 = {k: torch.empty(pat.nnz, dtype=torch.float64, device="cuda") for k in ("M", "A")}
    ms64 = timed(lambda: lfem.assemble(pat, xd, rule, which=3, precision=lfem.FP64, out=o64), 20, 3)
    # adjoint of L = u^T M u + v^T A v through the autograd function
    rng = np.random.default_rng(20260519)
    u = torch.from_numpy(rng.normal(size=N)).cuda()
    v = torch.from_numpy(rng.normal(size=N)).cuda()
    rows = torch.repeat_interleave(torch.arange(N, device="cuda"), rp[1:] - rp[:-1])
    xt = xd.clone().requires_grad_(True)

    def fwd_bwd(precision=lfem.FP64):
        xt.grad = None
        M, A, _ = lfem.AssembleFn.apply(xt, None, pat, rule, precision)
        L = (M.double() * u[rows] * u[col]).sum() + (A.double() * v[rows] * v[col]).sum()
        L.backward()
        return L

    ms_adj_mixed = timed(lambda: fwd_bwd(lfem.MIXED), 10, 2)
    fwd_bwd(lfem.MIXED)
    torch.cuda.synchronize()
    g_mixed = xt.grad.cpu().numpy().copy()
    ms_adj = timed(fwd_bwd, 10, 2)
    L = fwd_bwd()
    torch.cuda.synchronize()
    xh = xt.detach().cpu().numpy()
    un, vn, rr, cn = u.cpu().numpy(), v.cpu().numpy(), rows.cpu().numpy(), ci.cpu().numpy()
    t0 = time.perf_counter()
    ogx, _ = oracle.adjoint(xh, e, 2, 2, rule.xi, rule.w, None, (rp.cpu().numpy(), cn), un[rr] * un[cn],
                            vn[rr] * vn[cn], None)
    t_orc = time.perf_counter() - t0
    gerr = float(np.abs(xt.grad.cpu().numpy() - ogx).max() / np.abs(ogx).max())
    gerr_mixed = float(np.abs(g_mixed - ogx).max() / np.abs(ogx).max())
    # the right-hand sides of the flow on the final surface (Sec. 5.1): load
    # vector of the nodal mean curvature field and the non-linear vectors,
    # FP64, against the oracle
    H = torch.from_numpy(rng.normal(size=N)).cuda()
    nrm = xd / xd.norm(dim=1, keepdim=True)
    uf = torch.cat([nrm, H[:, None]], dim=1).contiguous()
    ms_load = timed(lambda: lfem.assemble_load(pat, xd, rule, H), 20, 3)
    ms_nl = timed(lambda: lfem.assemble_mcf_nonlinear(pat, xd, rule, uf), 20, 3)
    nl = lfem.assemble_mcf_nonlinear(pat, xd, rule, uf).cpu().numpy()
    onl = oracle.kll(xh, e, 2, rule.xi, rule.w, uf.cpu().numpy())
    nl_err = float(np.abs(nl - onl).max() / np.abs(onl).max())
    # one step of Dziuk's scheme on the final surface: FP64 assembly + PCG on the GPU,
    # against the oracle's direct solve
    # (on a side stream: the solver's 8-iteration blocks replay a captured graph)
    xs = xd.clone()
    ms_st = torch.cuda.Stream()
    ms_st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(ms_st):
        x1, cg_it = lfem.mcf_step(pat, xs, rule, 1e-4, rtol=1e-12, max_iter=5000, stream=ms_st)
        t_mcf = []
        for _ in range(3):
            a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(ms_st)
            lfem.mcf_step(pat, xs, rule, 1e-4, rtol=1e-12, max_iter=5000, out=x1, stream=ms_st)
            b0.record(ms_st)
            ms_st.synchronize()
            t_mcf.append(a0.elapsed_time(b0))
    torch.cuda.current_stream().wait_stream(ms_st)
    ox1 = oracle.mcf_step(xh, e, 2, 2, rule.xi, rule.w, 1e-4)
    mcf_err = float(np.abs(x1.cpu().numpy() - ox1).max() / np.abs(ox1).max())
    _line(args, "evolving_ellipsoid_r7_100_steps_plus_adjoint", e.shape[0] / (ms_step * 1e-3), "elements/s",
          ms_step,
          {"config": {"elements": int(e.shape[0]), "steps": steps, "tau": tau, "precision": "mixed, graph replay"},
           "fp64_assembly_ms": ms64, "adjoint_fwd_bwd_ms": ms_adj, "fp64_fallback_elements_final": fallback,
           "adjoint_vs_oracle_max_rel": gerr, "oracle_adjoint_s": t_orc, "L": float(L),
           "adjoint_mixed_fwd_bwd_ms": ms_adj_mixed, "adjoint_mixed_vs_oracle_max_rel": gerr_mixed,
           "load_vector_ms": ms_load, "mcf_nonlinear_ms": ms_nl, "mcf_nonlinear_vs_oracle_max_rel": nl_err,
           "dziuk_step_ms": min(t_mcf), "dziuk_step_cg_iterations": cg_it, "dziuk_step_vs_oracle_max_rel": mcf_err})


def run_c2q16(args):
    """The C2 surface with the rule size the paper uses for P2 triangles (16 points,
    degree 8): the general element path (any rule) in mixed precision and FP64."""
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import quadrature

    x, e, _ = bench.make_inputs(args.level)
    rule = quadrature.paper_rule(2)
    xd, ed = torch.from_numpy(x).cuda(), torch.from_numpy(e).cuda()
    pat = lfem.Pattern(ed, x.shape[0], 2, 2)
    flush = torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    timed = _timer(torch, flush)
    res = {}
    for prec, dt, name in ((lfem.MIXED, torch.float32, "mixed"), (lfem.FP64, torch.float64, "fp64")):
        if not args.no_autotune:
            lfem.autotune(pat, xd, rule, which=3, precision=prec)
        out = {k: torch.empty(pat.nnz, dtype=dt, device="cuda") for k in ("M", "A")}
        ms = timed(lambda: lfem.assemble(pat, xd, rule, which=3, precision=prec, out=out), args.steps, args.warmup)
        res[name] = {"ms_per_step": ms, "value": e.shape[0] / (ms * 1e-3), "tile_slots": pat.info()["tile_slots"],
                     "M_sum": float(out["M"].double().sum())}
        if prec == lfem.MIXED:
            res[name]["fp64_fallback_elements"] = pat.fallback_count()
        pat.sync_status()
    alg = e.shape[0] * 24 + x.shape[0] * 24 + 2 * pat.nnz * 4
    peak, kind = bench.measured_peaks()
    ach = alg / (res["mixed"]["ms_per_step"] * 1e-3) / 1e9
    _line(args, "p2_perturbed_sphere_r8_M_A_rule16_deg8", res["mixed"]["value"], "elements/s",
          res["mixed"]["ms_per_step"],
          {"config": {"elements": int(e.shape[0]), "quadrature": "tri 16-point degree 8 (general path)",
                      "l2": "flushed between steps"},
           "fp64": res["fp64"], "mixed": res["mixed"],
           "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": None, "algorithmic_bytes": alg, "peak_kind": kind}})


def run_p4(args):
    """Order 4 on the sphere: the P1 icosphere (level 6) lifted to order 4 on the GPU
    (lfem_lift_order), nodes projected to S^2, then M + A with the 16-point rule."""
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x1, e1 = meshes.icosphere(6, 1)
    xd1, ed1 = torch.from_numpy(x1).cuda(), torch.from_numpy(e1).cuda()
    p1 = lfem.Pattern(ed1, x1.shape[0], 2, 1)
    t_lift = []
    for _ in range(3):
        a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        xp, ep = lfem.lift_order(p1, xd1, 4)
        b0.record()
        torch.cuda.synchronize()
        t_lift.append(a0.elapsed_time(b0))
    xp = xp / xp.norm(dim=1, keepdim=True)
    rule = quadrature.tri_16pt_deg8()
    pat = lfem.Pattern(ep, xp.shape[0], 2, 4)
    flush = torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    timed = _timer(torch, flush)
    res = {}
    for prec, dt, name in ((lfem.MIXED, torch.float32, "mixed"), (lfem.FP64, torch.float64, "fp64")):
        out = {k: torch.empty(pat.nnz, dtype=dt, device="cuda") for k in ("M", "A")}
        ms = timed(lambda: lfem.assemble(pat, xp, rule, which=3, precision=prec, out=out), args.steps, args.warmup)
        res[name] = {"ms_per_step": ms, "value": ep.shape[0] / (ms * 1e-3),
                     "area_minus_4pi": float(out["M"].double().sum()) - 4 * np.pi}
        pat.sync_status()
    _line(args, "p4_icosphere_r6_M_A_rule16", res["mixed"]["value"], "elements/s", res["mixed"]["ms_per_step"],
          {"config": {"elements": int(ep.shape[0]), "nodes": int(xp.shape[0]), "nnz_per_matrix": pat.nnz,
                      "quadrature": "tri 16-point degree 8", "l2": "flushed between steps"},
           "fp64": res["fp64"], "mixed": res["mixed"], "lift_order_ms": min(t_lift)})


def run_tet34(args):
    """Orders 3 and 4 on tetrahedra: the P1 Kuhn cube (16^3 cells, 24576 tets)
    lifted on the GPU (lfem_lift_order), then M + A with the 64-point degree-7
    conical rule, FP64 and mixed.  Affine elements: sum M = 1 and A 1 = 0 are
    checked on the results."""
    import torch

    from paper_2605_14035_gb300 import lfem
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x1, e1 = meshes.kuhn_cube_p2(16, order=1)
    xd1, ed1 = torch.from_numpy(x1).cuda(), torch.from_numpy(e1).cuda()
    p1 = lfem.Pattern(ed1, x1.shape[0], 3, 1)
    rule = quadrature.paper_rule(3)
    flush = torch.empty(bench.L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    timed = _timer(torch, flush)
    res = {}
    for order in (3, 4):
        t_lift = []
        for _ in range(3):
            a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record()
            xp, ep = lfem.lift_order(p1, xd1, order)
            b0.record()
            torch.cuda.synchronize()
            t_lift.append(a0.elapsed_time(b0))
        pat = lfem.Pattern(ep, xp.shape[0], 3, order)
        rp, ci = pat.csr()
        rows = torch.repeat_interleave(torch.arange(xp.shape[0], device="cuda"), rp[1:] - rp[:-1])
        r = {"elements": int(ep.shape[0]), "nodes": int(xp.shape[0]), "nnz_per_matrix": pat.nnz,
             "lift_order_ms": min(t_lift)}
        for prec, dt, name in ((lfem.MIXED, torch.float32, "mixed"), (lfem.FP64, torch.float64, "fp64")):
            out = {k: torch.empty(pat.nnz, dtype=dt, device="cuda") for k in ("M", "A")}
            ms = timed(lambda: lfem.assemble(pat, xp, rule, which=3, precision=prec, out=out), args.steps,
                       args.warmup)
            rowsum = torch.zeros(xp.shape[0], dtype=torch.float64, device="cuda")
            rowsum.index_add_(0, rows, out["A"].double())
            r[name] = {"ms_per_step": ms, "value": ep.shape[0] / (ms * 1e-3),
                       "volume_minus_1": float(out["M"].double().sum()) - 1.0,
                       "max_abs_A_rowsum": float(rowsum.abs().max())}
            if name == "mixed":
                r["fallback_elements_mixed"] = pat.fallback_count()
            pat.sync_status()
        res[f"p{order}"] = r
    _line(args, "tet_p4_kuhn16_M_A_rule64", res["p4"]["mixed"]["value"], "elements/s",
          res["p4"]["mixed"]["ms_per_step"],
          {"config": {"cells": "16^3 Kuhn cube", "quadrature": "tet 64-point degree 7", "l2": "flushed between steps"},
           "p3": res["p3"], "p4": res["p4"]})


def run(args):
    return {"c1": run_c1, "c3": run_c3, "c4": run_c4, "c5": run_c5, "c2q16": run_c2q16, "p4": run_p4,
            "tet34": run_tet34}[args.workload](args)
