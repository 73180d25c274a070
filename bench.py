#!/usr/bin/env python3
"""Benchmark of MGR-preconditioned FGMRES on GB300.

Workload: the two-phase poromechanics Jacobian on 64x64x32 unit cells
(680,419 unknowns: 418,275 displacement + 2 x 131,072 cell dofs), FP64 plain
MGR, seeded synthetic inputs.  One step = one pass of the whole hot path on a
fresh Jacobian: mgr_setup (device hierarchy: W_p, S_1 with N_max dropping,
S_2, both AMG hierarchies) + fgmres_solve to a 1e-8 true relative residual +
mgr_destroy.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  value = unknowns solved per second over all ranks
(setup + solve), timed with CUDA events on the solve stream, barrier and
synchronize on both sides, max over ranks.  Several GPUs run independent
replicas (a single system's solve has no partition without halo exchange).
The reference arm times the CPU oracle (oracle/) on a bounded sample of the
same workload family.
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
WORKLOAD = dict(nx=64, ny=64, nz=32, seed=0, sigma=2.0)
SAMPLE = dict(nx=32, ny=32, nz=16, seed=0, sigma=2.0)
WORKLOAD_NAME = "two-phase poromechanics Jacobian, 64x64x32 cells, FP64 plain MGR"
# the mixed-precision large case (128x128x64 cells, lognormal E): extra keys
LARGE = dict(nx=128, ny=128, nz=64, seed=0, sigma=2.0, E_sigma=1.5)
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "vcycle_uu_traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--vcycles", type=int, default=50)
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 128x128x64 mixed-precision extra measurement")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the 64-system batched ensemble extra measurement")
    ap.add_argument("--ensemble-size", type=int, default=64)
    ap.add_argument("--profile", action="store_true",
                    help="short run for ncu: FP64 steps and V-cycles only, no clock "
                         "sampling, no mixed/e2e/oracle legs; prints a partial line")
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
    read once per use (row pointers 8 B, column index 4 B, value), every
    vector read or written once per kernel (see the design notes)."""
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
        A = (n + 1) * 8 + nnzA * (4 + vb)
        total += 3 * n * vb                                   # t = dinv .* b
        total += A + 3 * n * vb                               # r = b - A t
        total += (nc + 1) * 8 + nnzR * (4 + vb) + n * vb + nc * vb   # b_c = R r
        total += (n + 1) * 8 + nnzP * (4 + vb) + nc * vb + 2 * n * vb  # t += P x_c
        total += A + 4 * n * vb                               # x = t + dinv (b - A t)
    nco = dims[-1][0]
    total += nco * nco * vb + 2 * nco * vb                    # dense coarsest inverse
    return total


def source_hash():
    """Hash of the source that defines the V-cycle's kernels (csrc/apply.cu)."""
    h = hashlib.sha256()
    f = os.path.join(ROOT, "paper_1904_05960_gb300", "csrc", "apply.cu")
    with open(f, "rb") as fh:
        h.update(b"apply.cu")
        h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per V-cycle from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    kv = {}
    with open(PROFILE_TRAFFIC) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_vcycle"])
    except (KeyError, ValueError):
        return None


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- arms
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1904_05960_gb300 import synth
    p = synth.two_phase(**SAMPLE)
    times = []
    iters = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o = oracle.Oracle(p)
        r = o.fgmres(p.rhs)
        dt = time.perf_counter() - t0
        del o
        if i >= args.warmup:
            times.append(dt)
        iters = r["iters"]
    ms = 1e3 * sum(times) / len(times)
    value = p.n / (ms * 1e-3)
    sample = (f"two-phase {SAMPLE['nx']}x{SAMPLE['ny']}x{SAMPLE['nz']} cells ({p.n:,} unknowns), "
              "same recipe as the 64x64x32 workload; one oracle setup + FGMRES solve per step")
    line = dict(metric=METRIC, value=value, unit="dofs/s", n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD_NAME, parallelism=f"replicas x{world}",
                            sample=f"bounded CPU sample: {p.n:,} unknowns, {iters} iterations; "
                                   "value scaled to dofs/s of the sample"),
                cpu_baseline=dict(value=value, unit="dofs/s", cores=1, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit="dofs/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


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

    p = synth.two_phase(**WORKLOAD)
    stream = torch.cuda.current_stream()
    A = mgr.DeviceMatrix(p)
    b = torch.from_numpy(p.rhs).cuda()
    x = torch.zeros_like(b)
    fo = mgr.fgmres_options_default(restart=50, max_iter=1000, rtol=1e-8)

    def step(prec, xout):
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=prec), stream)
        r = mgr.fgmres_solve(h, A, b, xout, fo, stream)
        mgr.mgr_destroy(h)
        if not r["converged"]:
            raise RuntimeError(f"FGMRES did not converge: {r}")
        return r

    def timed(prec, steps, warmup, clocks=False):
        for _ in range(warmup):
            step(prec, x)
        barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(smi_device_id(local)) if clocks else None
        if sampler:
            sampler.__enter__()
        l0 = mgr.mgr_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = None
        for _ in range(steps):
            info = step(prec, x)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        launches = mgr.mgr_launch_count() - l0
        if sampler:
            sampler.__exit__()
        ms = reduce_max(e0.elapsed_time(e1) / steps)
        return ms, info, launches, (sampler.summary() if sampler else None)

    ms64, info64, launches, clocks = timed(mgr.MGR_FP64, args.steps, args.warmup,
                                           clocks=not args.profile)
    x64 = x.cpu().numpy().copy()
    if args.profile:
        peak, _ = measured_peak()
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True), stream)
        vin = torch.randn(p.meta["n_u"], dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vin)
        mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("vcycle_uu_fp64")
        for _ in range(args.vcycles):
            mgr.mgr_vcycle(h, 0, vin, vx, stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        byts = vcycle_bytes(mgr, h, 0, 8)
        mgr.mgr_destroy(h)
        if rank == 0:
            print(json.dumps(dict(profile=True, ms_per_step=ms64, iters=info64["iters"],
                                  gpu_launches=launches, vcycle_algorithmic_bytes=byts,
                                  vcycles=args.vcycles)), flush=True)
        return
    ms32, info32, _, _ = timed(mgr.MGR_MIXED, args.steps, args.warmup)
    x32 = x.cpu().numpy().copy()

    # end to end through the public API with host buffers (pinned): one
    # mgr_solve_host call copies the matrix and rhs in, runs setup + FGMRES +
    # teardown and copies x out
    Ah = mgr.HostMatrix(p, pin=True)
    bh = torch.from_numpy(p.rhs).pin_memory()
    xh = torch.empty(p.n, dtype=torch.float64).pin_memory()
    h2d = Ah.nbytes + bh.numel() * bh.element_size()
    d2h = xh.numel() * xh.element_size()
    o64 = mgr.mgr_options_default(True)

    def e2e_step():
        r = mgr.mgr_solve_host(Ah, bh, xh, o64, fo, stream)
        if not r["converged"]:
            raise RuntimeError(f"FGMRES did not converge: {r}")

    for _ in range(args.warmup):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = reduce_max(e0.elapsed_time(e1) / args.steps)

    # V-cycle of the displacement AMG (F-relaxation of the first reduction)
    peak, peak_kind = measured_peak()
    vc = {}
    for prec, vb in ((mgr.MGR_FP64, 8), (mgr.MGR_MIXED, 4)):
        h = mgr.mgr_setup(A, mgr.mgr_options_default(True, precision=prec), stream)
        nu = p.meta["n_u"]
        vb_in = torch.randn(nu, dtype=torch.float64, device="cuda")
        vx = torch.empty_like(vb_in)
        for _ in range(5):
            mgr.mgr_vcycle(h, 0, vb_in, vx, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.vcycles):
            mgr.mgr_vcycle(h, 0, vb_in, vx, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_eager = e0.elapsed_time(e1) / args.vcycles
        # timed the way the solve runs it: the V-cycle's launches replayed from
        # a CUDA graph (the preconditioner application is one captured graph)
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side):
            mgr.mgr_vcycle(h, 0, vb_in, vx, side)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            for _ in range(5):
                g.replay()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push(f"vcycle_uu_{'fp64' if vb == 8 else 'fp32'}")
            e0.record(stream)
            for _ in range(args.vcycles):
                g.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        ms_v = e0.elapsed_time(e1) / args.vcycles
        del g
        # the mixed entry point's FP64<->FP32 casts are inside the measured call
        # but not in the algorithmic bytes
        byts = vcycle_bytes(mgr, h, 0, vb)
        vc[prec] = dict(ms=ms_v, ms_eager=ms_eager, bytes=byts, gbs=byts / (ms_v * 1e-3) / 1e9)
        mgr.mgr_destroy(h)

    large = None
    if not args.no_large:
        pl = synth.two_phase(**LARGE)
        Al = mgr.DeviceMatrix(pl)
        bl = torch.from_numpy(pl.rhs).cuda()
        xl = torch.zeros_like(bl)
        res = {}
        for prec in (mgr.MGR_MIXED, mgr.MGR_FP64):
            def lstep():
                hh = mgr.mgr_setup(Al, mgr.mgr_options_default(True, precision=prec), stream)
                rr = mgr.fgmres_solve(hh, Al, bl, xl, fo, stream)
                mgr.mgr_destroy(hh)
                return rr
            lstep()
            barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            reps = 2
            for _ in range(reps):
                rr = lstep()
            e1.record(stream)
            torch.cuda.synchronize()
            res[prec] = (reduce_max(e0.elapsed_time(e1) / reps), rr)
        msm, rm = res[mgr.MGR_MIXED]
        msd, rd = res[mgr.MGR_FP64]
        large = dict(workload="two-phase 128x128x64 cells, lognormal E (sigma 1.5), MGR_MIXED",
                     unknowns=pl.n, nnz=pl.nnz, value=job_value(pl.n, world, msm), unit="dofs/s",
                     ms_per_step=msm, iters=rm["iters"], rel_res_true=rm["relres"],
                     setup_s=rm["setup_s"], solve_s=rm["solve_s"], fp64_ms_per_step=msd,
                     fp64_iters=rd["iters"], speedup_mixed_vs_fp64=msd / msm)
        del Al, bl, xl

    # operator and smoother variants (Sec. 5.1 options, multicolour block
    # Gauss-Seidel, one sweep of ILU(1) as the level-2 global smoother as in
    # Sec. 6): the same FP64 step on the same workload
    variants = {}
    for vname, vkw in (("jacobi_restriction", dict(restrict_jacobi=[1, 1])),
                       ("mgr_post", dict(frelax_post=[1, 1])),
                       ("point_block_dff", dict(dff_block=[1, 1])),
                       ("block_gauss_seidel", dict(global_smoother=[0, 1])),
                       ("aggressive_uu_amg", dict(agg_levels=[1, 0, 0])),
                       ("ilu1_smoother", dict(global_smoother=[0, 2], global_sweeps=[0, 1],
                                              ilu_solve_sweeps=3))):
        vo = mgr.mgr_options_default(True, **vkw)

        def vstep():
            hh = mgr.mgr_setup(A, vo, stream)
            rr = mgr.fgmres_solve(hh, A, b, x, fo, stream)
            mgr.mgr_destroy(hh)
            return rr
        vstep()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            rv = vstep()
        e1.record(stream)
        torch.cuda.synchronize()
        msv = e0.elapsed_time(e1) / 3
        variants[vname] = dict(ms_per_step=msv, iters=rv["iters"], setup_s=rv["setup_s"],
                               solve_s=rv["solve_s"], converged=rv["converged"],
                               relres=rv["relres"])

    ensemble = None
    if not args.no_ensemble:
        ensemble = run_ensemble(args, mgr, stream, world)

    n = p.n
    value = job_value(n, world, ms64)
    line = dict(
        metric=METRIC, value=value, unit="dofs/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=ms64, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=WORKLOAD_NAME,
                    unknowns=n, nnz=p.nnz, parallelism=f"replicas x{world}",
                    step="mgr_setup + fgmres_solve (m=50, rtol 1e-8 true residual) + mgr_destroy",
                    l2="inputs larger than L2 (CSR of A: %.0f MB)" % (p.nnz * 12 / 1e6),
                    iters=info64["iters"], setup_s=info64["setup_s"],
                    solve_s=info64["solve_s"]),
        roofline=dict(bound="hbm", kernel="AMG V-cycle on A_uu (F-relaxation of level 0), FP64",
                      achieved=vc[mgr.MGR_FP64]["gbs"], peak=peak, unit="GB/s",
                      frac=vc[mgr.MGR_FP64]["gbs"] / peak, peak_kind=peak_kind,
                      traffic=profiled_traffic(), algorithmic_bytes=vc[mgr.MGR_FP64]["bytes"],
                      ms=vc[mgr.MGR_FP64]["ms"], timing="CUDA-graph replay of mgr_vcycle",
                      ms_eager_launches=vc[mgr.MGR_FP64]["ms_eager"]),
        mixed=dict(value=job_value(n, world, ms32), ms_per_step=ms32,
                   speedup_vs_fp64=ms64 / ms32, iters=info32["iters"],
                   setup_s=info32["setup_s"], solve_s=info32["solve_s"],
                   vcycle_gbs=vc[mgr.MGR_MIXED]["gbs"],
                   vcycle_frac=vc[mgr.MGR_MIXED]["gbs"] / peak),
        e2e=dict(value=job_value(n, world, ms_e2e), unit="dofs/s", h2d_bytes_per_step=h2d,
                 d2h_bytes_per_step=d2h, ms_per_step=ms_e2e),
        clocks=clocks,
        gpu_launches=launches,
    )
    if large:
        line["large_mixed"] = large
    if ensemble:
        line["ensemble"] = ensemble
    if variants:
        line["variants"] = variants
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        o = oracle.Oracle(p)
        r = o.fgmres(p.rhs)
        dt = time.perf_counter() - t0
        xo = r["x"]
        nrm = np.linalg.norm(xo)
        line["cpu_baseline"] = dict(
            value=n / dt, unit="dofs/s", cores=1, kind="oracle",
            sample="one full oracle setup + FGMRES solve of this 64x64x32 workload",
            seconds=dt, iters=r["iters"])
        line["error_vs_oracle"] = dict(fp64=float(np.linalg.norm(x64 - xo) / nrm),
                                       mixed=float(np.linalg.norm(x32 - xo) / nrm))
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

    tune, _, _ = batched(0)                 # warm-up; the autotuner picks the workers
    torch.cuda.synchronize()
    e0.record(stream)
    _, st, infos = batched(tune["workers"])
    e1.record(stream)
    torch.cuda.synchronize()
    batched_s = e0.elapsed_time(e1) * 1e-3
    setup_part = e0.elapsed_time(em) * 1e-3
    xb = [x.clone() for x in xs]

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
        workers=tune["workers"], autotune_round_ms=tune["tune_ms"],
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
