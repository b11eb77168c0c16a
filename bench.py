"""Throughput of isoparametric P2 surface assembly on one GB300 (or N replicas).

Workload (default): P2 perturbed sphere r(theta, phi) = 1 + 0.2 sin(3 theta) cos(2 phi),
icosphere refined 8 times (1,310,720 six-node triangles, 2,621,442 nodes,
nnz 30,146,562 per matrix), mass + stiffness + coefficient-weighted mass
(c = 1 + x^2 + y z at the physical quadrature points) with the 7-point
degree-5 rule.  A step is one assembly of the three CSR matrices.

  value      elements/s of the mixed path (float geometry and local matrices,
             double fallback on ill-conditioned elements, compensated sums)
  fp64       elements/s of the plain FP64 path on the same inputs
  e2e        the same step through the public API with host buffers: pinned
             coordinates and coefficient copied in, the three matrices copied out
  roofline   k_assemble_pipe (mixed) algorithmic bytes / launch time vs the
             measured HBM copy bandwidth; traffic = DRAM bytes per launch from
             the committed ncu capture while the kernel's sources match it

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
# FP64 path: algorithmic flops per P2 surface element with the 7-point rule
# (M + A + MC; counted per quadrature point: Jacobian 36, metric 18, normal
# and its norm 16, w s G^-1 and metric quality 12, mass-type products 96,
# stiffness gradients 48 and products 84 -> 310; x 7 points, + 33 for the
# corner edge vectors and edge-node deviations of the element)
FP64_FLOPS_PER_ELEMENT = 7 * 310 + 33
FP64_PEAK_GFLOPS = 1250.0  # nominal dense FP64 of one GB300
WORKLOAD = "p2_perturbed_sphere_r8_M_A_MC"
KERNEL = "k_assemble_pipe<float,u16,EType<2,3,2,fast>>"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lfem", choices=["lfem", "reference"])
    ap.add_argument("--level", type=int, default=8, help="icosphere refinement level")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-elems", type=int, default=0, help="elements in the oracle sample (0 = auto)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "c2q16", "p4", "tet34"],
                    help="c2 (default): P2 perturbed sphere; c1 P1 sphere; c3 P2 tets + boundary; "
                         "c4 512-mesh batch; c5 evolving ellipsoid + adjoint")
    ap.add_argument("--batch-meshes", type=int, default=512)
    ap.add_argument("--batch-scale", type=float, default=1.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tile-slots", type=int, default=0, help="fixed tile capacity (implies no autotuning)")
    ap.add_argument("--no-batch", action="store_true", help="leave the 512-mesh batch out of the default line")
    return ap.parse_args()


def make_inputs(level):
    from paper_2605_14035_gb300.inputs import meshes, quadrature

    x, e = meshes.icosphere(level, 2)
    x = meshes.radial_perturbation(x, 0.2)
    return x, e, quadrature.tri_7pt_deg5()


def coef_from_points(pts):
    return 1.0 + pts[..., 0] ** 2 + pts[..., 1] * pts[..., 2]


class ClockSampler:
    """SM clock, power and clock-event reasons of one GPU, read through NVML
    (read-only queries) every millisecond while running, so that even a
    millisecond-long timed region gets samples; `mark(t0, t1)` restricts the
    summary to the samples taken between two host times.  Falls back to
    nvidia-smi at 200 ms when NVML cannot be loaded."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.rows = []
        self.window = None
        self.nvml = None

    def _nvml_open(self):
        import ctypes

        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(h)) != 0:
            return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        mx = ctypes.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx))
        return lib, h, reasons, mx.value

    def _loop(self):
        import ctypes

        lib, h, reasons, mx = self.nvml
        clk, pw, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self.stop:
            ok = lib.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(clk)) == 0
            lib.nvmlDeviceGetPowerUsage(h, ctypes.byref(pw))
            reasons(h, ctypes.byref(rs))
            if ok:
                act = [n for n, b in self.BITS.items() if rs.value & b]
                self.rows.append((time.perf_counter(), float(clk.value), float(mx), pw.value / 1000.0, act))
            time.sleep(0.001)

    def __enter__(self):
        import threading

        try:
            self.nvml = self._nvml_open()
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.stop = False
            self.thread = threading.Thread(target=self._loop, daemon=True)
            self.thread.start()
            return self
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.nvml is not None:
            self.stop = True
            self.thread.join(timeout=5)
            try:
                self.nvml[0].nvmlShutdown()
            except (AttributeError, OSError):
                pass
            return
        out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (out or "").strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                act = [names[i] for i, v in enumerate(f[5:9]) if v.lower() == "active"]
                self.rows.append((None, float(f[1]), float(f[2]), float(f[3]), act))
            except ValueError:
                continue

    def summary(self):
        rows = self.rows
        if self.window is not None and rows and rows[0][0] is not None:
            inside = [r for r in rows if self.window[0] <= r[0] <= self.window[1]]
            rows = inside or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        reasons = sorted({a for r in rows for a in r[4]})
        return {"sm_mhz": statistics.median(r[1] for r in rows), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": reasons, "samples": len(rows), "power_w_max": max(r[3] for r in rows),
                "source": "nvml 1 ms" if self.nvml is not None else "nvidia-smi 200 ms"}


def dist_init(backend):
    """One process per GPU (torchrun env); replicas: no collective on the data path,
    only the barrier and the max over ranks of the timed region."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return None, 1, 0, 0
    import torch
    import torch.distributed as dist

    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend)
    return dist, world, rank, local


def rank_barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(ms, dist, device):
    """Timed-region length of the job: the slowest rank's."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, steps, tot_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / (tot_ms * 1e-3)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Sources that define the timed kernel; a DRAM traffic figure taken with ncu is
# reported only while these files are byte-identical to the captured build.
KERNEL_SOURCES = ("assemble_pipe.cuh", "assemble_fast.cuh", "assemble_impl.cuh", "lfem_internal.cuh", "dispatch.cuh",
                  "assemble_d2.cu", "lfem_api.cu", "pattern.cu")


# the batch: one launch per element family (curve kernels live in assemble_d1.cu)
BATCH_KERNEL = "k_assemble_pipe (batch: one launch per element family)"
BATCH_SOURCES = KERNEL_SOURCES + ("assemble_d1.cu", "batch.cu")


def kernel_source_hash(sources=KERNEL_SOURCES):
    import hashlib

    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2605_14035_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(kernel, workload, sources=KERNEL_SOURCES):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch (per step for the
    batch) from the committed ncu summary, or None when the kernel sources
    changed since the capture."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        entries = json.load(f)["entries"]
    src = kernel_source_hash(sources)
    for en in entries:
        if en["kernel"] == kernel and en["workload"] == workload and en["source_sha256"] == src:
            return float(en["dram_bytes_per_launch"])
    return None


def oracle_sample(x, e, rule, n_elem, threads=1, keep=False):
    """Time the oracle on the first n_elem elements (pattern of that sub-mesh
    built beforehand): the single-thread assembly (threads = 1) or the
    all-core one (threads = 0: every thread OpenMP offers; bit-identical
    results).  Returns the seconds, and with keep the oracle's
    (row_ptr, col_idx, M, A, MC)."""
    import oracle

    sub = np.ascontiguousarray(e[:n_elem])
    pts = oracle.eval_points(x, sub, 2, 2, rule.xi)
    coef = coef_from_points(pts)
    pat = oracle.pattern(sub, x.shape[0])
    t0 = time.perf_counter()
    if threads == 1:
        res = oracle.assemble(x, sub, 2, 2, rule.xi, rule.w, coef, pat=pat)
    else:
        res = oracle.assemble_threads(x, sub, 2, 2, rule.xi, rule.w, coef, pat=pat, threads=threads)
    dt = time.perf_counter() - t0
    return (dt, res) if keep else dt


def host_description():
    """Core count and CPU model of the host the oracle runs on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def diag_scaled(v, ref, rows, cols, n):
    """max |v - ref| / sqrt(|ref_ii ref_jj|) over all entries (the tolerance metric)."""
    d = np.zeros(n)
    isd = rows == cols
    d[rows[isd]] = np.abs(ref[isd])
    den = np.sqrt(d[rows] * d[cols])
    return float((np.abs(v - ref) / den).max())


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, run on every host core
    (its all-core assembly, bit-identical to the single-thread one), one
    assembly of the whole workload mesh per step (pattern and coefficients
    prepared once, outside the timed steps)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    x, e, rule = make_inputs(args.level)
    n = min(args.cpu_sample_elems or e.shape[0], e.shape[0])
    sub = np.ascontiguousarray(e[:n])
    coef = coef_from_points(oracle.eval_points(x, sub, 2, 2, rule.xi))
    pat = oracle.pattern(sub, x.shape[0])
    threads = oracle.max_threads()

    def step():
        oracle.assemble_threads(x, sub, 2, 2, rule.xi, rule.w, coef, pat=pat)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = n * args.steps / tot
    line = {
        "impl": "reference", "metric": "elements/s", "value": value, "unit": "elements/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": int(e.shape[0]), "sample_elements_per_step": n},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": threads, "kind": "oracle",
                         "sample": f"{'all' if n == e.shape[0] else f'first {n}'} elements of the workload per step, "
                                   f"M+A+MC, FP64, {threads} threads", "host": host_description()},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        import bench_extra

        return bench_extra.run(args)

    import torch

    from paper_2605_14035_gb300 import lfem

    dist, world, rank, local = dist_init("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    x, e, rule = make_inputs(args.level)
    nE, N = e.shape[0], x.shape[0]
    xd = torch.from_numpy(x).to(dev)
    ed = torch.from_numpy(e).to(dev)
    # the pattern (CSR, incidence maps and row tiles) is built once per topology: timed on its own
    torch.cuda.synchronize()
    t_pat = time.perf_counter()
    pat = lfem.Pattern(ed, N, 2, 2)
    torch.cuda.synchronize()
    pattern_ms = 1e3 * (time.perf_counter() - t_pat)
    pts = lfem.eval_points(ed, 2, 2, xd, rule)
    coef64 = coef_from_points(pts).contiguous()
    coef32 = coef64.float()
    del pts
    nnz = pat.nnz
    tuned = None
    t_tune = time.perf_counter()
    if args.tile_slots:
        pat.retile(args.tile_slots)
    elif not args.no_autotune:
        tuned = lfem.autotune(pat, xd, rule, coef32, which=7, precision=lfem.MIXED)
    torch.cuda.synchronize()
    tune_ms = 1e3 * (time.perf_counter() - t_tune)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        rank_barrier(dist)

    def timed(fn, steps, warmup, clk=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        t_host0 = time.perf_counter()
        evs = []
        for _ in range(steps):
            flush.fill_(1.0)  # untimed: evict L2 between steps
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if clk is not None:
            clk.mark(t_host0, time.perf_counter())
        barrier()
        ms = [a.elapsed_time(b) for a, b in evs]
        return max_over_ranks(sum(ms), dist, dev), ms

    out_mixed = {k: torch.empty(nnz, dtype=torch.float32, device=dev) for k in ("M", "A", "MC")}
    out_fp64 = {k: torch.empty(nnz, dtype=torch.float64, device=dev) for k in ("M", "A", "MC")}

    def step_mixed():
        lfem.assemble(pat, xd, rule, coef32, which=7, precision=lfem.MIXED, out=out_mixed)

    def step_fp64():
        lfem.assemble(pat, xd, rule, coef64, which=7, precision=lfem.FP64, out=out_fp64)

    sm_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        try:
            sm_index = int(vis.split(",")[local])
        except ValueError:
            pass
    with ClockSampler(sm_index) as clk:
        tot_ms, per = timed(step_mixed, args.steps, args.warmup, clk)
    clocks = clk.summary()
    fallback = pat.fallback_count()
    pat.sync_status()
    value = job_value(world, nE, args.steps, tot_ms)

    res = {}
    if not args.skip_fp64:
        tot64, per64 = timed(step_fp64, max(3, args.steps // 4), max(1, args.warmup // 2))
        k64 = max(3, args.steps // 4)
        ms64 = tot64 / k64
        gflops = FP64_FLOPS_PER_ELEMENT * nE / (ms64 * 1e-3) / 1e9
        res["fp64"] = {"value": world * nE * k64 / (tot64 * 1e-3), "unit": "elements/s", "ms_per_step": ms64,
                       "roofline": {"bound": "fp64 alu", "achieved": gflops, "peak": FP64_PEAK_GFLOPS,
                                    "unit": "GFLOP/s", "frac": gflops / FP64_PEAK_GFLOPS,
                                    "flops_per_element": FP64_FLOPS_PER_ELEMENT,
                                    "peak_kind": "nominal GB300 FP64 (no measured FP64 peak)"}}
        # accuracy of the mixed path against the FP64 path on every entry (diagonal-scaled)
        rp, ci = pat.csr()
        rows = torch.repeat_interleave(torch.arange(N, device=dev), rp[1:] - rp[:-1])
        isd = rows == ci.long()
        errs = {}
        for k in ("M", "A", "MC"):
            ref = out_fp64[k]
            diag = torch.zeros(N, dtype=torch.float64, device=dev)
            diag[rows[isd]] = ref[isd].abs()
            den = torch.sqrt(diag[rows] * diag[ci.long()])
            errs[k] = float(((out_mixed[k].double() - ref).abs() / den).max().item())
        errs["sum_M"] = abs(float(out_mixed["M"].double().sum()) - float(out_fp64["M"].sum())) / float(out_fp64["M"].sum())
        res["mixed_vs_fp64_err"] = errs
        del rows, isd

    # end to end through the public API with host buffers
    x_h = torch.from_numpy(x).pin_memory()
    c_h = coef32.cpu().pin_memory()
    outs_h = {k: torch.empty(nnz, dtype=torch.float32).pin_memory() for k in ("M", "A", "MC")}
    xd2 = torch.empty_like(xd)
    cd2 = torch.empty_like(coef32)

    def step_e2e():
        xd2.copy_(x_h, non_blocking=True)
        cd2.copy_(c_h, non_blocking=True)
        lfem.assemble(pat, xd2, rule, cd2, which=7, precision=lfem.MIXED, out=out_mixed)
        for k in outs_h:
            outs_h[k].copy_(out_mixed[k], non_blocking=True)

    k_e2e = max(3, args.steps // 4)
    tot_e2e, _ = timed(step_e2e, k_e2e, 2)
    h2d = x.nbytes + coef32.numel() * 4
    d2h = 3 * nnz * 4

    # the same steps as a stream of jobs: two device buffer sets, uploads on one
    # stream, assembly on the current one, downloads on a third, so step k+1's
    # upload runs while step k's results come back (every step still moves all
    # of its inputs and outputs; assemblies stay serialised on the pattern)
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    xin = [xd2, torch.empty_like(xd)]
    cin = [cd2, torch.empty_like(coef32)]
    outd = [out_mixed, {k: torch.empty(nnz, dtype=torch.float32, device=dev) for k in ("M", "A", "MC")}]
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_comp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    for ev in ev_comp + ev_out:
        ev.record(stream)

    def step_e2e_pipelined(i):
        j = i % 2
        s_in.wait_event(ev_comp[j])  # the previous kernel on buffer j has read its inputs
        with torch.cuda.stream(s_in):
            xin[j].copy_(x_h, non_blocking=True)
            cin[j].copy_(c_h, non_blocking=True)
        ev_in[j].record(s_in)
        stream.wait_event(ev_in[j])
        stream.wait_event(ev_out[j])  # buffer j's previous results are on the host
        lfem.assemble(pat, xin[j], rule, cin[j], which=7, precision=lfem.MIXED, out=outd[j], stream=stream)
        ev_comp[j].record(stream)
        s_out.wait_event(ev_comp[j])
        with torch.cuda.stream(s_out):
            for k in outs_h:
                outs_h[k].copy_(outd[j][k], non_blocking=True)
        ev_out[j].record(s_out)

    def run_pipelined(n):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for i in range(n):
            step_e2e_pipelined(i)
        stream.wait_event(ev_out[(n - 1) % 2])
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    run_pipelined(3)  # warm-up
    barrier()
    tot_pipe = max_over_ranks(run_pipelined(k_e2e), dist, dev)

    # roofline of k_assemble_tiles (mixed): algorithmic bytes = unique inputs + outputs
    alg_bytes = nE * 6 * 4 + N * 3 * 8 + nE * rule.n_pts * 4 + 3 * nnz * 4
    launch_ms = tot_ms / args.steps
    peak, peak_kind = measured_peaks()
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    info = pat.info()
    traffic = measured_traffic(KERNEL, f"{WORKLOAD}_tile{info['tile_slots']}")

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        n_s = args.cpu_sample_elems or nE
        # the oracle's values for the parity keys (all cores, bit-identical to one thread)
        _, ores = oracle_sample(x, e, rule, n_s, threads=0, keep=True)
        dt_one = oracle_sample(x, e, rule, min(n_s, 400000), threads=1)
        n_one = min(n_s, 400000)
        # the all-core timing in a process of its own (no torch runtime beside it): the reference arm
        cpu = None
        try:
            r = subprocess.run([sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", "3",
                                "--warmup", "1", "--level", str(args.level)] +
                               (["--cpu-sample-elems", str(n_s)] if args.cpu_sample_elems else []),
                               capture_output=True, text=True, timeout=600,
                               env={k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE")})
            ref_line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
            cpu = dict(ref_line["cpu_baseline"])
            cpu["sample"] += f"; {ref_line['ms_per_step']:.0f} ms per assembly, after one warm-up, in a separate process"
        except (subprocess.SubprocessError, OSError, ValueError, IndexError, KeyError) as ex:
            cpu = {"value": None, "unit": "elements/s", "kind": "oracle", "error": str(ex)[:200]}
        cpu["single_thread"] = {"value": n_one / dt_one, "unit": "elements/s", "cores": 1,
                                "sample": f"first {n_one} elements, {dt_one:.2f} s, in the benchmark process"}
        if n_s == nE:
            # the benchmarked configuration against the oracle, entry by entry
            orp, oci, oM, oA, oC = ores
            rp, ci = pat.csr()
            rp_h, ci_h = rp.cpu().numpy(), ci.cpu().numpy()
            pattern_equal = bool(np.array_equal(rp_h, orp) and np.array_equal(ci_h, oci))
            rows = np.repeat(np.arange(N), np.diff(orp))
            cols = oci.astype(np.int64)
            parity = {"pattern_equal": pattern_equal, "tolerance": {"fp64": 1e-12, "mixed": 1e-6},
                      "metric": "max |v - v*| / sqrt(|v*_ii v*_jj|) over every entry, v* = FP64 oracle"}
            if pattern_equal:
                parity["mixed_vs_oracle"] = {k: diag_scaled(out_mixed[k].double().cpu().numpy(), r, rows, cols, N)
                                             for k, r in (("M", oM), ("A", oA), ("MC", oC))}
                if not args.skip_fp64:
                    parity["fp64_vs_oracle"] = {k: diag_scaled(out_fp64[k].cpu().numpy(), r, rows, cols, N)
                                                for k, r in (("M", oM), ("A", oA), ("MC", oC))}
                parity["ok"] = all(v <= 1e-6 for v in parity["mixed_vs_oracle"].values()) and all(
                    v <= 1e-12 for v in parity.get("fp64_vs_oracle", {}).values())
            del rows, cols, ores

    # the 512-mesh batch (mixed, M + A, tile capacities tuned by the library)
    batch = None
    if not args.no_batch:
        import bench_extra

        del out_fp64, out_mixed, outd, xin, cin, flush
        torch.cuda.empty_cache()
        batch = bench_extra.measure_batch(args)

    line = {
        "metric": "elements/s", "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "elements": nE, "nodes": N, "nnz_per_matrix": nnz, "matrices": "M,A,MC",
                   "precision": "mixed", "quadrature": "tri 7-point degree 5", "l2": "flushed between steps",
                   "tile_slots": info["tile_slots"], "autotuned": tuned is not None, "tiles": info["tiles"],
                   "recompute": info["recompute"],
                   "fp64_fallback_elements": fallback, "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_unit": "DRAM bytes per launch (ncu)",
                     "kernel": KERNEL, "algorithmic_bytes": alg_bytes,
                     "peak_kind": peak_kind},
        "cpu_baseline": cpu,
        "e2e": {"value": world * nE * k_e2e / (tot_pipe * 1e-3), "unit": "elements/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": tot_pipe / k_e2e,
                "mode": "pipelined: step k+1's upload overlaps step k's download (two device buffer sets)",
                "serial": {"value": world * nE * k_e2e / (tot_e2e * 1e-3), "ms_per_step": tot_e2e / k_e2e}},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "pattern_build_ms": pattern_ms,
        "tile_tuning_ms": tune_ms,
        "parity": parity,
        "batch": batch,
        **res,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
