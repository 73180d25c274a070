#!/usr/bin/env python3
"""Benchmark of MGR-preconditioned FGMRES on GB300.

Headline workload: the large heterogeneous two-phase poromechanics Jacobian,
256x256x96 unit cells (31,803,171 unknowns: 19,220,259 displacement + 2 x
6,291,456 cell dofs, 1.56e9 non-zeros), high-contrast permeability channels
(1e3 in a 1e-3 background) and alternating stiff/soft layers (E 1e4 / 10,
nu 0.3), seeded synthetic inputs; mixed precision (MGR_MIXED: FP32
preconditioner, FP64 FGMRES).  One step = one pass of the whole hot path on
the resident Jacobian: mgr_setup (device hierarchy: W_p, S_1 with N_max
dropping, S_2, both AMG hierarchies) + fgmres_solve to a 1e-8 true relative
residual + mgr_destroy.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  value = unknowns solved per second over all ranks
(setup + solve), timed with CUDA events on the solve stream, barrier and
synchronize on both sides, max over ranks.  Several GPUs run independent
replicas (a single system's solve has no partition without halo exchange).
Extra keys: the FP64 preconditioner on the same system (mixed-vs-FP64
speedup), end to end from host buffers, the 128x128x64 and 64x64x32 two-phase
workloads with their errors against the oracle, operator variants, the
64-system ensemble.  The reference arm times the CPU oracle (oracle/) on a
bounded sample of the headline recipe.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MGR-FGMRES solve s & dofs/s to rel-res 1e-8; V-cycle HBM GB/s; mixed vs FP64"
HEADLINE = dict(nx=256, ny=256, nz=96, seed=0)
HEADLINE_NAME = ("two-phase poromechanics Jacobian, 256x256x96 cells, permeability channels "
                 "1e3 in 1e-3, stiff/soft layers E 1e4/10, MGR_MIXED, displacement AMG with one "
                 "level of aggressive coarsening")
# the solver configuration of the paper's Sec. 6 for the displacement AMG (one
# level of aggressive coarsening) on top of the library defaults
HEADLINE_OPTS = dict(agg_levels=[1, 0, 0])
# the same recipe at 1/512 of the cells: the bounded CPU sample of the oracle
SAMPLE = dict(nx=32, ny=32, nz=12, seed=0)
MEDIUM = dict(nx=128, ny=128, nz=64, seed=0, sigma=2.0, E_sigma=1.5)
MEDIUM_NAME = "two_phase_128x128x64"
SMALL = dict(nx=64, ny=64, nz=32, seed=0, sigma=2.0)
MAX_ITER = 4000
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vcycles", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line only: skip the FP64, e2e, other workloads, variants "
                         "and ensemble legs")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the 64-system batched ensemble extra measurement")
    ap.add_argument("--ensemble-size", type=int, default=64)
    ap.add_argument("--profile", action="store_true",
                    help="short run for ncu: one headline setup and --profile-iters FGMRES "
                         "iterations after a warm-up on the 64x64x32 workload; prints a "
                         "partial line")
    ap.add_argument("--profile-iters", type=int, default=30)
    ap.add_argument("--profile-workload", choices=["headline", "headline_vcycle", "small", "medium",
                                                   "krylov"],
                    default="headline")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def dist_max(x, world):
    """Max of a per-rank number over all ranks (identity for one rank); the
    reduction buffer lives where the process group's backend wants it."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_max):
    """Whole-job throughput: the units every rank processed in one step,
    over the slowest rank's step time."""
    return units_per_rank * world / (ms_max * 1e-3)


# --------------------------------------------------------------------------- clocks
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def smi_device_id(device):
    """The identifier nvidia-smi -i needs for a torch device: its UUID (or PCI
    bus id), not the process-local index, which under CUDA_VISIBLE_DEVICES can
    name another GPU of the machine."""
    import torch
    props = torch.cuda.get_device_properties(device)
    uuid = getattr(props, "uuid", None)
    if uuid is not None:
        u = str(uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    bus = getattr(props, "pci_bus_id", None)
    if bus is not None:
        return "%08X:%02X:%02X.0" % (getattr(props, "pci_domain_id", 0), bus,
                                     getattr(props, "pci_device_id", 0))
    return str(device)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    def __init__(self, smi_id):
        self.idx = smi_id
        self.proc = None
        self.path = None
        self.out = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.idx), "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        time.sleep(0.2)
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
        if self.out:
            self.out.close()
            self.out = None

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                     hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return dict(sm_mhz=statistics.median(r["sm"] for r in rows),
                    sm_max_mhz=max(r["smax"] for r in rows), samples=len(rows),
                    reasons=sorted(reasons))


# --------------------------------------------------------------------------- roofline
def vcycle_bytes(mgr, h, slot, value_bytes):
    """Algorithmic DRAM bytes of one V-cycle of AMG slot `slot`: every matrix
    read once per use (row pointers 8 B, column index 4 B -- or a 2-byte
    pattern id per row where the operator has shared row patterns, and in
    FP32 a slice offset per 32 rows instead of row pointers -- value),
    every vector read or written once per kernel (see the design notes)."""
    vb = value_bytes
    nlev = mgr.mgr_amg_levels(h, slot)
    total = 0
    dims = []
    for k in range(nlev):
        a = mgr.mgr_get_csr_dims(h, mgr.Q_AMG_A, slot, k)
        dims.append(a)
    for k in range(nlev - 1):
        n, _, nnzA = dims[k]
        nc = dims[k + 1][0]
        _, _, nnzP = mgr.mgr_get_csr_dims(h, mgr.Q_AMG_P, slot, k)
        _, _, nnzR = mgr.mgr_get_csr_dims(h, mgr.Q_AMG_R, slot, k)
        if mgr.mgr_row_patterns(h, slot, k) > 0:
            # shared row patterns: a 2-byte pattern id per row instead of a
            # column index per non-zero (the pattern table stays in cache);
            # the FP32 values sliced by 32 rows: a slice offset per 32 rows
            # instead of a row pointer per row (the zero padding, < 1% here,
            # is not counted)
            rows = (n // 32 + 1) * 8 if vb == 4 else (n + 1) * 8
            A = rows + 2 * n + nnzA * vb
        else:
            A = (n + 1) * 8 + nnzA * (4 + vb)
        total += 3 * n * vb                                   # t = dinv .* b
        total += A + 3 * n * vb                               # r = b - A t
        total += (nc + 1) * 8 + nnzR * (4 + vb) + n * vb + nc * vb   # b_c = R r
        total += (n + 1) * 8 + nnzP * (4 + vb) + nc * vb + 2 * n * vb  # t += P x_c
        total += A + 4 * n * vb                               # x = t + dinv (b - A t)
    nco = dims[-1][0]
    total += nco * nco * vb + 2 * nco * vb                    # dense coarsest inverse
    return total


VCYCLE_END = b"// ---- end of the AMG V-cycle: kernels and launch rules above this line ----"


def source_hash():
    """Hash of the source that defines the V-cycle's kernels and launch rules:
    csrc/apply.cu up to its end-of-V-cycle marker."""
    h = hashlib.sha256()
    f = os.path.join(ROOT, "paper_1904_05960_gb300", "csrc", "apply.cu")
    with open(f, "rb") as fh:
        src = fh.read()
    cut = src.find(VCYCLE_END)
    h.update(b"apply.cu")
    h.update(src if cut < 0 else src[:cut])
    return h.hexdigest()[:16]


def profiled_traffic(tag, algorithmic):
    """DRAM bytes per V-cycle from the committed ncu summary
    profiles/vcycle_uu_traffic_<tag>.txt if it was taken on the current kernel
    sources, scaled to `algorithmic` bytes when the capture was on a smaller
    case (traffic ~ proportional to the bytes the V-cycle must move); else
    None.  Returns (bytes, note)."""
    path = os.path.join(PROFILES, f"vcycle_uu_traffic_{tag}.txt")
    if not os.path.exists(path):
        return None, None
    kv = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != source_hash():
        return None, "stale capture (kernel source changed)"
    try:
        t = float(kv["dram_bytes_per_vcycle"])
        alg = float(kv["algorithmic_bytes_per_vcycle"])
    except (KeyError, ValueError):
        return None, None
    if abs(alg - algorithmic) <= 1e-6 * algorithmic:
        return t, f"ncu capture of this V-cycle ({kv.get('workload', '?')})"
    return t * algorithmic / alg, (f"scaled from the ncu capture of {kv.get('workload', '?')} "
                                   f"(traffic/algorithmic {t / alg:.3f})")


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- arms
def sample_problem():
    from paper_1904_05960_gb300 import synth
    return synth.channels(**SAMPLE)


def sample_text(p, iters):
    return (f"bounded CPU sample: the headline recipe at {SAMPLE['nx']}x{SAMPLE['ny']}x{SAMPLE['nz']} "
            f"cells ({p.n:,} unknowns, {iters} oracle iterations), one oracle setup + FGMRES "
            "solve per step; value = sample unknowns / step seconds")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    p = sample_problem()
    times = []
    iters = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = oracle.Oracle(p, **HEADLINE_OPTS)
        r = o.fgmres(p.rhs, maxit=MAX_ITER)
        dt = time.perf_counter() - t0
        del o
        if i >= args.warmup:
            times.append(dt)
        iters = r["iters"]
    ms = 1e3 * sum(times) / len(times)
    value = p.n / (ms * 1e-3)
    line = dict(metric=METRIC, value=value, unit="dofs/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=HEADLINE_NAME, parallelism=f"replicas x{world}",
                            sample=sample_text(p, iters)),
                cpu_baseline=dict(value=value, unit="dofs/s", cores=1, kind="oracle",
                                  sample=sample_text(p, iters)),
                e2e=dict(value=value, unit="dofs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


class Timer:
    """CUDA events on one stream around a region."""

    def __init__(self, torch, stream):
        self.torch, self.stream = torch, stream
        self.e0 = torch.cuda.Event(enable_timing=True)
        self.e1 = torch.cuda.Event(enable_timing=True)

    def start(self):
        self.e0.record(self.stream)

    def stop(self):
        self.e1.record(self.stream)
        self.torch.cuda.synchronize()
        return self.e0.elapsed_time(self.e1)


def graph_ms(torch, stream, fn, reps):
    """Average time of fn() replayed from a CUDA graph (the way the solve runs
    the preconditioner's kernels)."""
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        fn(side)
    torch.cuda.synchronize()
    tm = Timer(torch, stream)
    with torch.cuda.stream(stream):
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        tm.start()
        for _ in range(reps):
            g.replay()
        ms = tm.stop() / reps
    del g
    return ms


def run_ours(args):
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1904_05960_gb300 import mgr, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def reduce_max(x):
        return dist_max(x, world)

    stream = torch.cuda.current_stream()
    tm = Timer(torch, stream)
    fo = mgr.fgmres_options_default(restart=50, max_iter=MAX_ITER, rtol=1e-8)
    peak, peak_kind = measured_peak()
    extras = not (args.no_extras or args.profile)

    def solve_step(A, b, x, prec, **kw):
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=prec, **kw), stream)
        r = mgr.fgmres_solve(h, A, b, x, fo, stream)
        mgr.mgr_destroy(h)
        if not r["converged"]:
            raise RuntimeError(f"FGMRES did not converge: {r}")
        return r

    # ---- the 64x64x32 workload first: it also brings every FP64 and FP32
    # kernel of the library into the process before the headline is timed
    small = None
    ps = synth.two_phase(**SMALL)
    As = mgr.DeviceMatrix(ps)
    bs = torch.from_numpy(ps.rhs).cuda()
    xs = torch.zeros_like(bs)
    if args.profile and args.profile_workload == "krylov":
        # FGMRES iterations inside an NVTX range "solve" on the 96x96x48
        # two-phase workload (2.27M unknowns: modified Gram-Schmidt; 115M
        # non-zeros: the sliced Jacobian copy), small enough for full ncu
        # captures of the Krylov kernels
        pk = synth.two_phase(96, 96, 48, seed=0, sigma=2.0)
        Ak = mgr.DeviceMatrix(pk)
        bk = torch.from_numpy(pk.rhs).cuda()
        xk = torch.zeros_like(bk)
        solve_step(Ak, bk, xk, mgr.MGR_MIXED, **HEADLINE_OPTS)
        hk = mgr.mgr_setup(Ak, mgr.mgr_options_default(True, precision=mgr.MGR_MIXED,
                                                       **HEADLINE_OPTS), stream)
        xk.zero_()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("solve")
        rk = mgr.fgmres_solve(hk, Ak, bk, xk, mgr.fgmres_options_default(max_iter=args.profile_iters),
                              stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        mgr.mgr_destroy(hk)
        if rank == 0:
            print(json.dumps(dict(profile=True, workload="krylov", unknowns=pk.n, nnz=pk.nnz,
                                  iters=rk["iters"])), flush=True)
        return
    if args.profile and args.profile_workload in ("small", "medium"):
        pp = ps if args.profile_workload == "small" else synth.two_phase(**MEDIUM)
        Ap = As if pp is ps else mgr.DeviceMatrix(pp)
        bp = torch.from_numpy(pp.rhs).cuda()
        xp = torch.zeros_like(bp)
        solve_step(Ap, bp, xp, mgr.MGR_MIXED, **HEADLINE_OPTS)
        torch.cuda.synchronize()
        h = mgr.mgr_setup(Ap, mgr.mgr_options_default(True, precision=mgr.MGR_MIXED,
                                                      **HEADLINE_OPTS), stream)
        nu = pp.meta["n_u"]
        vin = torch.randn(nu, dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vin)
        mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("vcycle")
        for _ in range(args.vcycles):
            mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps(dict(profile=True, workload=args.profile_workload, vcycles=args.vcycles,
                                  vcycle_algorithmic_bytes=vcycle_bytes(mgr, h, 0, 4))), flush=True)
        mgr.mgr_destroy(h)
        return
    if args.profile:
        # bring the FP32 kernels into the process before the profiled launches
        solve_step(As, bs, xs, mgr.MGR_MIXED, **HEADLINE_OPTS)
        torch.cuda.synchronize()
    res_small = {}
    for prec in (() if args.profile else (mgr.MGR_FP64, mgr.MGR_MIXED)):
        solve_step(As, bs, xs, prec)
        tm.start()
        for _ in range(3):
            r = solve_step(As, bs, xs, prec)
        res_small[prec] = (tm.stop() / 3, r, xs.cpu().numpy().copy())
    vc_small = {}
    for prec, vb in (() if args.profile else ((mgr.MGR_FP64, 8), (mgr.MGR_MIXED, 4))):
        h = mgr.mgr_setup(As, mgr.mgr_options_default(True, precision=prec), stream)
        vin = torch.randn(ps.meta["n_u"], dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vin)
        ms_v = graph_ms(torch, stream, lambda st: mgr.mgr_vcycle(h, 0, vin, vx, st), 50)
        byts = vcycle_bytes(mgr, h, 0, vb)
        vc_small[prec] = dict(ms=ms_v, bytes=byts, frac=byts / (ms_v * 1e-3) / 1e9 / peak)
        mgr.mgr_destroy(h)
    if not args.profile:
        small = dict(workload="two-phase 64x64x32 cells, lognormal k sigma 2", unknowns=ps.n,
                     nnz=ps.nnz)
        for prec, key in ((mgr.MGR_FP64, "fp64"), (mgr.MGR_MIXED, "mixed")):
            ms, r, _ = res_small[prec]
            small[key] = dict(ms_per_step=ms, value=job_value(ps.n, world, ms), iters=r["iters"],
                              setup_s=r["setup_s"], solve_s=r["solve_s"],
                              vcycle_uu_ms=vc_small[prec]["ms"],
                              vcycle_uu_frac=vc_small[prec]["frac"])
        small["speedup_mixed_vs_fp64"] = res_small[mgr.MGR_FP64][0] / res_small[mgr.MGR_MIXED][0]

    # ---- headline workload
    t0 = time.perf_counter()
    p = synth.channels(**HEADLINE)
    gen_s = time.perf_counter() - t0
    A = mgr.DeviceMatrix(p)
    b = torch.from_numpy(p.rhs).cuda()
    x = torch.zeros_like(b)
    if args.profile and args.profile_workload == "headline_vcycle":
        # the FP32 A_uu V-cycle alone on the headline hierarchy, inside an NVTX
        # range "vcycle" (for DRAM-traffic counters of its kernels)
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=mgr.MGR_MIXED,
                                                     **HEADLINE_OPTS), stream)
        vin = torch.randn(p.meta["n_u"], dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vin)
        mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("vcycle")
        for _ in range(args.vcycles):
            mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps(dict(profile=True, workload="headline_vcycle", vcycles=args.vcycles,
                                  vcycle_algorithmic_bytes=vcycle_bytes(mgr, h, 0, 4))), flush=True)
        mgr.mgr_destroy(h)
        return
    if args.profile:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("headline")
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=mgr.MGR_MIXED,
                                                     **HEADLINE_OPTS), stream)
        r = mgr.fgmres_solve(h, A, b, x, mgr.fgmres_options_default(max_iter=args.profile_iters),
                             stream)
        mgr.mgr_destroy(h)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps(dict(profile=True, workload="headline", iters=r["iters"],
                                  solve_s=r["solve_s"], setup_s=r["setup_s"])), flush=True)
        return

    for _ in range(args.warmup):
        solve_step(A, b, x, mgr.MGR_MIXED, **HEADLINE_OPTS)
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(smi_device_id(local))
    sampler.__enter__()
    l0 = mgr.mgr_launch_count()
    tm.start()
    info = None
    for _ in range(args.steps):
        info = solve_step(A, b, x, mgr.MGR_MIXED, **HEADLINE_OPTS)
    ms_local = tm.stop() / args.steps
    barrier()
    launches = mgr.mgr_launch_count() - l0
    sampler.__exit__()
    clocks = sampler.summary()
    ms = reduce_max(ms_local)
    x_mixed = x.cpu().numpy().copy()

    # roofline: the A_uu V-cycle (F-relaxation of the first reduction) in
    # FP32, graph-replayed, on the headline hierarchy; the pressure V-cycle
    # and the FP64 Jacobian product beside it
    h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=mgr.MGR_MIXED, **HEADLINE_OPTS),
                      stream)
    kernels = {}
    for slot, name in ((0, "vcycle_uu_fp32"), (2, "vcycle_pressure_fp32")):
        nA = mgr.mgr_get_csr_dims(h, mgr.Q_AMG_A, slot, 0)[0]
        vin = torch.randn(nA, dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vin)
        ms_v = graph_ms(torch, stream, lambda st: mgr.mgr_vcycle(h, slot, vin, vx, st), args.vcycles)
        byts = vcycle_bytes(mgr, h, slot, 4)
        kernels[name] = dict(ms=ms_v, algorithmic_bytes=byts, gbs=byts / (ms_v * 1e-3) / 1e9,
                             frac=byts / (ms_v * 1e-3) / 1e9 / peak)
        del vin, vx
    used, reserved = mgr.mgr_memory_usage()
    # the FP64 Jacobian product as the solve forms it (over the sliced copy
    # of A the solve makes: one thread per row, one multiply-add per
    # non-zero), the plain CSR product beside it, and the per-solve copy
    y = torch.empty_like(b)
    xin = torch.randn_like(b)
    tm.start()
    sliced = mgr.mgr_jacobian_product(h, A, xin, y, refresh=True)
    ms_copy = tm.stop()
    csr_bytes = (p.n + 1) * 8 + p.nnz * 12 + 2 * p.n * 8
    sell_bytes = (p.n // 32 + 1) * 8 + (p.n + 1) * 8 + p.nnz * 12 + 2 * p.n * 8
    for name, fn, byts in (
            ("jacobian_spmv_fp64", lambda: mgr.mgr_jacobian_product(h, A, xin, y, refresh=False),
             sell_bytes if sliced else csr_bytes),
            ("jacobian_spmv_fp64_csr", lambda: mgr.mgr_spmv(A, xin, y), csr_bytes)):
        fn()
        tm.start()
        for _ in range(args.vcycles):
            fn()
        ms_az = tm.stop() / args.vcycles
        kernels[name] = dict(ms=ms_az, algorithmic_bytes=byts, gbs=byts / (ms_az * 1e-3) / 1e9,
                             frac=byts / (ms_az * 1e-3) / 1e9 / peak,
                             fp64_fma_floor_ms=p.nnz / 0.625e12 * 1e3)
    kernels["jacobian_spmv_fp64"].update(sliced_copy=bool(sliced), copy_ms_per_solve=ms_copy,
                                         fp64_floor_note="nnz multiply-adds at GB300's nominal "
                                                         "1.25 TFLOP/s FP64")
    mgr.mgr_destroy(h)
    del y, xin
    dom = kernels["vcycle_uu_fp32"]
    traffic, traffic_note = profiled_traffic("fp32", dom["algorithmic_bytes"])

    line = dict(
        metric=METRIC, value=job_value(p.n, world, ms), unit="dofs/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32/f64",
        data="synthetic",
        config=dict(workload=HEADLINE_NAME, unknowns=p.n, nnz=p.nnz,
                    parallelism=f"replicas x{world}",
                    step="mgr_setup + fgmres_solve (m=50, rtol 1e-8 true residual) + mgr_destroy",
                    l2="inputs larger than L2 (CSR of A: %.1f GB)" % (p.nnz * 12 / 1e9),
                    iters=info["iters"], restarts=info["restarts"], setup_s=info["setup_s"],
                    solve_s=info["solve_s"], rel_res_true=info["relres"],
                    options="library defaults (Sec. 5.3 scheme) with agg_levels = [1, 0, 0]",
                    device_pool_gb=used / 1e9, generation_s=gen_s),
        roofline=dict(bound="hbm", kernel="AMG V-cycle on A_uu (F-relaxation of the first "
                      "reduction), FP32, on the headline hierarchy",
                      achieved=dom["gbs"], peak=peak, unit="GB/s", frac=dom["frac"],
                      peak_kind=peak_kind, traffic=traffic, traffic_note=traffic_note,
                      algorithmic_bytes=dom["algorithmic_bytes"], ms=dom["ms"],
                      timing="CUDA-graph replay of mgr_vcycle, CUDA events"),
        kernels=kernels, clocks=clocks, gpu_launches=launches)

    if extras:
        # same step with the FP64 preconditioner (the plain form)
        xd = torch.zeros_like(b)
        tm.start()
        rd = solve_step(A, b, xd, mgr.MGR_FP64, **HEADLINE_OPTS)
        ms_fp64 = reduce_max(tm.stop())
        x_fp64 = xd.cpu().numpy().copy()
        del xd
        line["mixed_vs_fp64"] = dict(fp64_ms_per_step=ms_fp64, speedup=ms_fp64 / ms,
                                     fp64_iters=rd["iters"], fp64_setup_s=rd["setup_s"],
                                     fp64_solve_s=rd["solve_s"],
                                     rel_diff_mixed_vs_fp64=float(
                                         np.linalg.norm(x_mixed - x_fp64) / np.linalg.norm(x_fp64)))
        # end to end through the public API from pinned host buffers: one
        # mgr_solve_host call copies the matrix and rhs in, runs setup + FGMRES
        # + teardown and copies x out.  The main steps above already ran every
        # kernel and filled the library's memory pool; one more warm-up here.
        del A
        torch.cuda.empty_cache()
        Ah = mgr.HostMatrix(p, pin=True)
        bh = torch.from_numpy(p.rhs).pin_memory()
        xh = torch.empty(p.n, dtype=torch.float64).pin_memory()
        h2d = Ah.nbytes + bh.numel() * bh.element_size()
        d2h = xh.numel() * xh.element_size()
        om = mgr.mgr_options_default(True, precision=mgr.MGR_MIXED, **HEADLINE_OPTS)
        r = mgr.mgr_solve_host(Ah, bh, xh, om, fo, stream)
        barrier()
        torch.cuda.synchronize()
        tm.start()
        r = mgr.mgr_solve_host(Ah, bh, xh, om, fo, stream)
        ms_e2e = reduce_max(tm.stop())
        if not r["converged"]:
            raise RuntimeError(f"FGMRES did not converge: {r}")
        line["e2e"] = dict(value=job_value(p.n, world, ms_e2e), unit="dofs/s",
                           h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h, ms_per_step=ms_e2e,
                           steps=1, warmup=1, api="mgr_solve_host")
        del Ah, bh, xh
    else:
        del A
    del b, x
    torch.cuda.empty_cache()
    mgr.mgr_trim_memory(0)

    if extras:
        # the 128x128x64 two-phase workload (5.34M unknowns)
        pm = synth.two_phase(**MEDIUM)
        Am = mgr.DeviceMatrix(pm)
        bm = torch.from_numpy(pm.rhs).cuda()
        xm = torch.zeros_like(bm)
        med = dict(workload="two-phase 128x128x64 cells, lognormal k sigma 2, lognormal E sigma 1.5",
                   unknowns=pm.n, nnz=pm.nnz)
        sols = {}
        for prec, key, reps in ((mgr.MGR_MIXED, "mixed", 2), (mgr.MGR_FP64, "fp64", 1)):
            solve_step(Am, bm, xm, prec)
            tm.start()
            for _ in range(reps):
                r = solve_step(Am, bm, xm, prec)
            msm = reduce_max(tm.stop() / reps)
            sols[key] = xm.cpu().numpy().copy()
            med[key] = dict(ms_per_step=msm, value=job_value(pm.n, world, msm), iters=r["iters"],
                            setup_s=r["setup_s"], solve_s=r["solve_s"], rel_res_true=r["relres"])
        med["speedup_mixed_vs_fp64"] = med["fp64"]["ms_per_step"] / med["mixed"]["ms_per_step"]
        line["two_phase_128x128x64"] = med
        del Am, bm, xm
        torch.cuda.empty_cache()
        line["two_phase_64x64x32"] = small

        # operator and smoother variants (Sec. 5.1 options, multicolour block
        # Gauss-Seidel, one sweep of ILU(1) as the level-2 global smoother as in
        # Sec. 6, aggressive coarsening of A_uu, BF16 smoother diagonals): the
        # same step on the 64x64x32 workload
        variants = {}
        for vname, prec, vkw in (("jacobi_restriction", mgr.MGR_FP64, dict(restrict_jacobi=[1, 1])),
                                 ("mgr_post", mgr.MGR_FP64, dict(frelax_post=[1, 1])),
                                 ("point_block_dff", mgr.MGR_FP64, dict(dff_block=[1, 1])),
                                 ("block_gauss_seidel", mgr.MGR_FP64, dict(global_smoother=[0, 1])),
                                 ("aggressive_uu_amg", mgr.MGR_FP64, dict(agg_levels=[1, 0, 0])),
                                 ("ilu1_smoother", mgr.MGR_FP64,
                                  dict(global_smoother=[0, 2], global_sweeps=[0, 1],
                                       ilu_solve_sweeps=3)),
                                 ("bf16_diagonals_mixed", mgr.MGR_MIXED, dict(diag_bf16=1)),
                                 ("f16_values_mixed", mgr.MGR_MIXED, dict(values_f16=1))):
            solve_step(As, bs, xs, prec, **vkw)
            tm.start()
            for _ in range(3):
                rv = solve_step(As, bs, xs, prec, **vkw)
            msv = tm.stop() / 3
            variants[vname] = dict(ms_per_step=msv, iters=rv["iters"], setup_s=rv["setup_s"],
                                   solve_s=rv["solve_s"], relres=rv["relres"],
                                   precision="mixed" if prec == mgr.MGR_MIXED else "fp64")
        line["variants_64x64x32"] = variants
        if not args.no_ensemble:
            line["ensemble"] = run_ensemble(args, mgr, stream, world)

    # errors against the oracle (the oracle is run or read here, outside every
    # timed region) and the CPU baseline
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        from oracle import fingerprint
        errs = {}
        # headline: the true residual of the GPU solution recomputed with the
        # oracle's own sparse product (plain serial C), and the whole method
        # against the oracle on the bounded sample of the same recipe
        t0 = time.perf_counter()
        ax = oracle.csr_spmv(p.row_ptr, p.col, p.val, x_mixed)
        errs["headline_rel_res_by_oracle_spmv"] = float(
            np.linalg.norm(p.rhs - ax) / np.linalg.norm(p.rhs))
        errs["headline_oracle_spmv_s"] = time.perf_counter() - t0
        del ax
        psm = sample_problem()
        t0 = time.perf_counter()
        o = oracle.Oracle(psm, **HEADLINE_OPTS)
        ro = o.fgmres(psm.rhs, maxit=MAX_ITER)
        dt = time.perf_counter() - t0
        del o
        line["cpu_baseline"] = dict(value=psm.n / dt, unit="dofs/s", cores=1, kind="oracle",
                                    sample=sample_text(psm, ro["iters"]), seconds=dt,
                                    iters=ro["iters"])
        Asm = mgr.DeviceMatrix(psm)
        bsm = torch.from_numpy(psm.rhs).cuda()
        xsm = torch.zeros_like(bsm)
        for prec, key in ((mgr.MGR_MIXED, "sample_mixed"), (mgr.MGR_FP64, "sample_fp64")):
            r = solve_step(Asm, bsm, xsm, prec, **HEADLINE_OPTS)
            xg = xsm.cpu().numpy()
            errs[key] = dict(rel_err=float(np.linalg.norm(xg - ro["x"]) / np.linalg.norm(ro["x"])),
                             iters=r["iters"], oracle_iters=ro["iters"])
        if extras:
            fp = fingerprint.load(MEDIUM_NAME)
            errs[MEDIUM_NAME] = {k: fingerprint.compare(v, fp) for k, v in sols.items()}
            t0 = time.perf_counter()
            xo = oracle.Oracle(ps).fgmres(ps.rhs)["x"]
            errs["two_phase_64x64x32"] = {
                k: float(np.linalg.norm(res_small[prec][2] - xo) / np.linalg.norm(xo))
                for prec, k in ((mgr.MGR_FP64, "fp64"), (mgr.MGR_MIXED, "mixed"))}
            errs["two_phase_64x64x32_oracle_s"] = time.perf_counter() - t0
        line["error_vs_oracle"] = errs
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ensemble(args, mgr, stream, world):
    """The ensemble workload: 64 independent two-phase Jacobians (cubic sides
    16-48, sigma in [1, 3], dt in [0.1, 10]), MGR_MIXED preconditioner with
    FP64 FGMRES.  One step = mgr_setup_batched + fgmres_solve_batched +
    mgr_destroy_batched; compared with the same systems solved one after
    another through mgr_setup / fgmres_solve / mgr_destroy on one stream."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    import torch
    from paper_1904_05960_gb300 import synth
    count = args.ensemble_size
    As, bs = [], []
    t0 = time.perf_counter()
    # the generator is numpy; build members in spawned processes (this process
    # already holds a CUDA context) and upload each as it arrives
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        for pm in ex.map(synth.ensemble_member, range(count)):
            As.append(mgr.DeviceMatrix(pm))
            bs.append(torch.from_numpy(pm.rhs).cuda())
    gen_s = time.perf_counter() - t0
    unknowns = sum(A.n for A in As)
    nnz = sum(A.nnz for A in As)
    opts = mgr.mgr_options_default(True, precision=mgr.MGR_MIXED)
    fo = mgr.fgmres_options_default()
    xs = [torch.zeros_like(b) for b in bs]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    em = torch.cuda.Event(enable_timing=True)

    def batched(workers):
        bh = mgr.mgr_setup_batched(As, opts, workers, stream)
        em.record(stream)
        info = mgr.mgr_batch_info(bh)
        st, infos = mgr.fgmres_solve_batched(bh, As, bs, xs, fo, stream)
        mgr.mgr_destroy_batched(bh)
        return info, st, infos

    tune, _, _ = batched(0)                 # warm-up; the autotuner picks the schedule
    batched(-1 if tune["workers"] > 0 else 8)   # warm-up of the other schedule
    torch.cuda.synchronize()
    schedules, results = {}, {}
    name = lambda wk: "lockstep" if wk < 0 else f"{wk}_workers"
    other = -1 if tune["workers"] > 0 else 8
    for wk in (tune["workers"], other):
        e0.record(stream)
        _, st_w, infos_w = batched(wk)
        e1.record(stream)
        torch.cuda.synchronize()
        schedules[name(wk)] = dict(s=e0.elapsed_time(e1) * 1e-3, setup_s=e0.elapsed_time(em) * 1e-3)
        results[name(wk)] = (st_w, infos_w, [x.clone() for x in xs])
    st, infos, xb = results[name(tune["workers"])]
    schedules[name(other)]["bitwise_equal_to_tuned"] = all(
        torch.equal(a, c) for a, c in zip(results[name(other)][2], xb))
    first = "lockstep" if tune["workers"] < 0 else f"{tune['workers']}_workers"
    batched_s = schedules[first]["s"]
    setup_part = schedules[first]["setup_s"]

    torch.cuda.synchronize()
    e0.record(stream)
    seq_iters = []
    for A, b, x in zip(As, bs, xs):
        h = mgr.mgr_setup(A, opts, stream)
        r = mgr.fgmres_solve(h, A, b, x, fo, stream)
        mgr.mgr_destroy(h)
        seq_iters.append(r["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    seq_s = e0.elapsed_time(e1) * 1e-3
    same = all(torch.equal(a, b) for a, b in zip(xb, xs))
    iters = [i["iters"] for i in infos]
    out = dict(
        workload=f"{count} two-phase Jacobians, cubic sides 16-48 cells, sigma U[1,3], "
                 "dt logU[0.1,10]; MGR_MIXED preconditioner, FP64 FGMRES",
        systems=count, unknowns=unknowns, nnz=nnz,
        value=unknowns * world / batched_s, unit="dofs/s",
        batched_s=batched_s, sequential_s=seq_s, speedup_vs_sequential=seq_s / batched_s,
        batched_setup_s=setup_part, batched_solve_and_destroy_s=batched_s - setup_part,
        step="mgr_setup_batched + fgmres_solve_batched + mgr_destroy_batched",
        schedule=first, schedules=schedules, autotune_round_ms=tune["tune_ms"],
        iters_min=min(iters), iters_max=max(iters), iters_total=sum(iters),
        all_converged=all(i["converged"] for i in infos) and st == mgr.MGR_SUCCESS,
        max_rel_res_true=max(i["relres"] for i in infos),
        iters_equal_to_single=iters == seq_iters, bitwise_equal_to_single=same,
        generation_s=gen_s)
    del As, bs, xs, xb
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
