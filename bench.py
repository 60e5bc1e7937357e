"""Benchmark of the DWF multigrid hot path on GB300.

Metric: D_hop HBM GB/s (the algorithmic bytes of every hopping-term launch of
the step divided by the step's time), with the mixed-precision red-black CGNR
solve to a true residual of 1e-8 (Sec. 5.1 of arXiv:2103.05034) as the step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--no-cpu-baseline] [--mg-compare]

One step = one rbcg_solve (FP32 inner CG, FP64 reliable updates, FP64 true
residual) of D_DW x = b from x = 0 on the 16^3x32, Ls = 16 smeared-random
workload, inputs resident in HBM.  The L2 is flushed (a 512 MB write) before
every timed step; each step is timed with CUDA events on the launching stream.

N > 1 (torchrun): every rank solves its own source on its own GPU (replicas,
weak scaling; the path has no exchange step on one GPU per problem); value =
all ranks' bytes / max-over-ranks time.

--impl reference: the FP64 numpy oracle timed on the host cores on a bounded
sample of the same workload (one full-lattice D_hop per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "D_hop HBM GB/s (% of peak); MG vs FP64 RB-CG time to 1e-8 residual, same GPU"
UNIT = "GB/s"


# ---------------------------------------------------------------------- helpers
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(*rel):
    h = hashlib.sha256()
    for r in rel:
        h.update(open(os.path.join(ROOT, r), "rb").read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_key, shash):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p)).get(kernel_key)
    except Exception:
        return None
    if not d or d.get("source_hash") != shash:
        return None
    return d.get("dram_bytes_per_launch")


def build_workload(name, rank):
    """Links and (for host-sized lattices) the Gaussian source of a workload.
    Paper-size lattices (over 2^30 5D sites' worth of host memory) get no host
    source: their inputs are drawn on the device."""
    w = synth.WORKLOADS[name]
    L, Ls = w["L"], w["Ls"]
    U = synth.workload_gauge(name)
    b = None
    if int(np.prod(L)) * Ls <= (1 << 27):
        b = synth.gaussian_spinor(L, Ls, synth.SEED_SOURCE + rank)
    return w, U, b


# ---------------------------------------------------------------------- CPU oracle legs
def oracle_dhop_sample(w, U, b):
    """One full-lattice FP64 oracle D_hop; returns (seconds, algorithmic bytes)."""
    from oracle import dwf
    L, Ls = w["L"], w["Ls"]
    t0 = time.perf_counter()
    dwf.dhop(U, b)
    dt = time.perf_counter() - t0
    V5 = int(np.prod(L)) * Ls
    nbytes = V5 * (24 * 16) + int(np.prod(L)) * 8 * 9 * 16  # FP64 spinors in+out, 8 links per site
    return dt, nbytes


def cpu_baseline_leg(w, U, b):
    dt, nbytes = oracle_dhop_sample(w, U, b)
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full-lattice FP64 numpy D_hop at {'x'.join(map(str, w['L']))}x{w['Ls']} "
                      f"({dt:.1f} s, single-threaded numpy)",
            "seconds": dt}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w, U, b = build_workload(args.workload, 0)
    for _ in range(args.warmup):
        oracle_dhop_sample(w, U, b)
    times, nbytes = [], 0
    for _ in range(args.steps):
        dt, nb = oracle_dhop_sample(w, U, b)
        times.append(dt)
        nbytes += nb
    tot = sum(times)
    val = nbytes / tot / 1e9
    sample = f"one full-lattice FP64 numpy D_hop at {'x'.join(map(str, w['L']))}x{w['Ls']} per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "oracle": "numpy FP64",
                                             "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- MG vs FP64 RB-CG
# HDCR parameters for the 16^3x32, Ls=16 workload: 4^4 x Ls blocks, 16 + 16
# basis vectors from the paper's recursive Chebyshev filter (m = 500,
# Delta = 100, lambda_lo = 0.05, Tables 1 and 12), coarse CG to 0.02, pGCR(32).
# The smoother interval is lowered to [0.05, lambda_max] with order 32: on the
# smeared-random stand-in fields the Shamir bulk modes reach H^2 ~ 0.04, below
# the paper's [0.5, 60] (with that interval the solve stalls near 1e-4).
MG_PARAMS = dict(block=(4, 4, 4, 4), nbasis=32, subspace="recursive", filter_order=500, delta=100,
                 lambda_lo=0.05, smooth=(0.05, None, 32), coarse_tol=0.02, coarse_maxiter=5000,
                 nkrylov=32, maxiter=300)


def mg_vs_fp64(ctx, w, b, bd, tol):
    """Time to a true residual of `tol` on the same GPU and source: plain FP64
    red-black CG against HDCR setup + solve (mixed precision).  One run each,
    outside the timed steps; CUDA-event and host-clock times agree because
    both calls synchronise."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import F32, F64, SOLVE_F64, SUBSPACE_BATCH, SUBSPACE_RECURSIVE

    L, Ls, mf = w["L"], w["Ls"], w["mf"]
    out = {}
    x = torch.zeros_like(bd)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ops.rbcg_solve(ctx, x, bd, mf, tol, 100000, SOLVE_F64)
    out["fp64_rbcg_s"] = time.perf_counter() - t0
    out["fp64_rbcg_iterations"] = st["iterations"]
    out["fp64_rbcg_true_residual"] = st["true_residual"]
    from paper_2103_05034_gb300 import layout
    p = dict(MG_PARAMS)
    nb = p["nbasis"]
    recursive = p["subspace"] == "recursive"
    neta = 1 if recursive else nb  # the recursive basis grows from one Gaussian
    t0 = time.perf_counter()
    v0 = torch.from_numpy(layout.complex_to_real(layout.to_full(synth.gaussian_spinor(L, Ls, 77), L), F64)).cuda()
    eta = torch.cat([torch.from_numpy(layout.complex_to_real(
        layout.to_full(synth.gaussian_spinor(L, Ls, synth.SEED_BASIS + i), L), F64).reshape(-1))
        for i in range(neta)]).cuda()
    torch.cuda.synchronize()
    t_in = time.perf_counter() - t0  # host-side input generation, not counted
    t0 = time.perf_counter()
    # lambda_max of D^dag D bounds the filter and smoother intervals (power
    # method in FP32, 100 iterations, 10 % margin: the Rayleigh quotient
    # approaches the top of the spectrum from below)
    lmax = ops.dwf_power_max(ctx, v0, mf, 100, F32) * 1.10
    prm = ops.mg_params(p["block"], nb, mf, subspace_mode=SUBSPACE_RECURSIVE if recursive else SUBSPACE_BATCH,
                        lambda_lo=p["lambda_lo"], lambda_max=lmax, filter_order=p["filter_order"],
                        delta=p["delta"], smooth=(p["smooth"][0], lmax, p["smooth"][2]),
                        coarse_tol=p["coarse_tol"],
                        coarse_maxiter=p["coarse_maxiter"], nkrylov=p["nkrylov"], maxiter=p["maxiter"])
    G = ops.MG(ctx, prm, eta)
    torch.cuda.synchronize()
    out["mg_setup_s"] = time.perf_counter() - t0
    x.zero_()
    t0 = time.perf_counter()
    sm = ops.mg_solve(G, x, bd, tol)
    out["mg_solve_s"] = time.perf_counter() - t0
    out["mg_outer_iterations"] = sm["iterations"]
    out["mg_coarse_iterations"] = sm["coarse_iterations"]
    out["mg_fine_matmuls"] = sm["fine_matmuls"]
    out["mg_true_residual"] = sm["true_residual"]
    out["mg_subspace_s"] = sm["setup_seconds"]
    out["mg_coarse_op_s"] = sm["coarse_op_seconds"]
    out["mg_total_s"] = out["mg_setup_s"] + out["mg_solve_s"]
    out["speedup_fp64_over_mg"] = out["fp64_rbcg_s"] / out["mg_total_s"]
    out["lambda_max"] = lmax
    out["params"] = {k: v for k, v in p.items()}
    out["input_generation_s_not_counted"] = t_in
    G.close()
    return out


# ---------------------------------------------------------------------- GPU leg
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2103_05034_gb300 import layout, ops
    from paper_2103_05034_gb300._lib import F32, F64, SOLVE_MIXED_F32

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w, U, b = build_workload(args.workload, rank)
    L, Ls, M5, mf = w["L"], w["Ls"], w["M5"], w["mf"]
    ctx = ops.Context(L, Ls, M5, U)
    hop_variant, hop_tuned_ms = ops.dwf_autotune(ctx, F32, 20)  # setup, not timed
    bfull = layout.complex_to_real(layout.to_full(b, L), F64)
    bd = torch.from_numpy(bfull).to(dev)
    xd = torch.zeros_like(bd)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def solve(x, bb):
        return ops.rbcg_solve(ctx, x, bb, mf, args.tol, 100000, SOLVE_MIXED_F32)

    for _ in range(args.warmup):
        xd.zero_()
        solve(xd, bd)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    stats = []
    ops.dwf_reset_counters(ctx)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        st = solve(xd, bd)
        ev[k][1].record(stream)
        stats.append(st)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    launches, hop_bytes = ops.dwf_counters(ctx)
    t_dev = sum(a.elapsed_time(bq) for a, bq in ev) / 1e3
    t_max = t_dev
    tot_bytes = hop_bytes
    if world > 1:
        tt = torch.tensor([t_dev, hop_bytes], dtype=torch.float64, device=dev)
        tmax = tt.clone()
        dist.all_reduce(tmax[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[1:], op=dist.ReduceOp.SUM)
        t_max, tot_bytes = float(tmax[0]), float(tt[1])
    value = tot_bytes / t_max / 1e9

    # ---- dominant kernel: the FP32 hopping term, timed alone with an L2 flush before each launch
    inp = ctx.new_half(F32)
    inp.copy_(torch.from_numpy(layout.complex_to_real(layout.to_half(b, L, 1), F32).reshape(-1)).to(dev))
    out = torch.zeros_like(inp)
    hop_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(20)]
    for _ in range(3):
        ops.dwf_dhop(ctx, out, inp, 0)
    for k, (e0, e1) in enumerate(hop_ev):
        flush.fill_(float(k))
        e0.record(stream)
        ops.dwf_dhop(ctx, out, inp, 0)
        e1.record(stream)
    torch.cuda.synchronize()
    hop_ms = float(np.mean([a.elapsed_time(bq) for a, bq in hop_ev]))
    Vh = ctx.Vh
    hop_alg_bytes = Vh * (Ls * 24 * 8 + 72 * 8)
    peaks, peak_kind = measured_peaks()
    achieved = hop_alg_bytes / (hop_ms / 1e3) / 1e9
    shash = source_hash("paper_2103_05034_gb300/csrc/dhop_impl.cuh")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": profile_traffic(f"hop_kernel_f32_ls{Ls}_{args.workload}", shash),
                "kernel": f"dwfk::hop_kernel<F32, Ls={Ls}> (dwf_dhop, plain epilogue)",
                "launch_ms": hop_ms, "algorithmic_bytes_per_launch": hop_alg_bytes,
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "source_hash": shash}

    # ---- end to end through the C ABI with pinned host buffers
    bh = torch.from_numpy(bfull).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    solve(xh, bh)  # warm
    ops.dwf_reset_counters(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_stats = []
    for _ in range(args.steps):
        e2e_stats.append(solve(xh, bh))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    _, e2e_bytes = ops.dwf_counters(ctx)
    if world > 1:
        tt = torch.tensor([t_e2e, e2e_bytes], dtype=torch.float64, device=dev)
        tm = tt.clone()
        dist.all_reduce(tm[:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(tt[1:], op=dist.ReduceOp.SUM)
        t_e2e, e2e_bytes = float(tm[0]), float(tt[1])
    e2e = {"value": e2e_bytes / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(bh.numel() * 8),
           "d2h_bytes_per_step": int(xh.numel() * 8),
           "note": "rbcg_solve on pinned host b and x: H2D of b and D2H of x inside the call"}

    line = None
    if rank == 0:
        s0 = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "lattice": list(L), "Ls": Ls, "M5": M5, "mf": mf,
                       "solver": "red-black CGNR, FP32 inner, FP64 reliable updates",
                       "tol_true_residual": args.tol, "l2": "flushed (512 MB write) before each step",
                       "parallelism": f"replicas{world}",
                       "hop_variant_f32": hop_variant, "hop_autotune_ms": hop_tuned_ms},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roofline,
            "e2e": e2e,
            "solve": {"iterations": s0["iterations"], "reliable_updates": s0["reliable_updates"],
                      "true_residual": s0["true_residual"], "fine_matmuls": s0["fine_matmuls"],
                      "seconds": t_max / args.steps, "wall_seconds_all_steps": t_wall},
        }
        if args.mg_compare:
            try:
                line["mg_vs_fp64"] = mg_vs_fp64(ctx, w, b, bd, args.tol)
            except Exception as e:  # reported, not hidden: the line says what failed
                line["mg_vs_fp64"] = {"error": str(e)}
        if args.cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline_leg(w, U, b)
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


def run_coarse_kernel(args):
    """`--kernel coarse_tf32|coarse_f32`: the little Dirac operator of H_DW on
    the workload's lattice (4^4 x Ls blocks, 32 basis vectors from Gaussians,
    chirality-projected and block-orthonormalised) applied to 32 right-hand
    sides, warmup + steps launches, L2 flushed before each timed launch."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import F32, F64, TF32

    w, U, _ = build_workload(args.workload, 0)
    L, Ls, mf = w["L"], w["Ls"], w["mf"]
    ctx = ops.Context(L, Ls, w["M5"], U)
    nb, nrhs, block = 32, 32, (4, 4, 4, 4)
    nfull = 2 * ctx.half_numel()  # reals of one full FP64 field
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_BASIS)
    g = torch.randn(nb * nfull, generator=gen, device="cuda", dtype=torch.float64)
    basis = torch.empty_like(g)
    half = nb // 2 * nfull
    ops.dwf_chiral_project(ctx, basis[:half], g[:half], 1, nb // 2)
    ops.dwf_chiral_project(ctx, basis[half:], g[half:], -1, nb // 2)
    del g
    ops.block_orthonormalise(ctx, basis, nb, nb // 2, block)
    Cc = ops.coarse_build(ctx, basis, nb, nb // 2, block, mf)
    del basis
    prec = {"tf32": TF32, "f32": F32}[args.kernel.split("_")[1]]
    inp = torch.randn(2 * Cc.nc * nb * nrhs, generator=gen, device="cuda", dtype=torch.float32)
    out = torch.zeros_like(inp)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(args.warmup, 1)):
        ops.coarse_apply(Cc, out, inp, nrhs, prec)
    ts = []
    for k in range(args.steps):
        flush.fill_(float(k))
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops.coarse_apply(Cc, out, inp, nrhs, prec)
        z.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(z))
    ms = float(np.median(ts))
    flop = 8.0 * 9 * nb * nb * nrhs * Cc.nc
    abytes = Cc.nc * 9 * nb * nb * 8 + 2 * Cc.nc * nb * nrhs * 8  # FP32 operator + in/out vectors
    print(json.dumps({"kernel": args.kernel, "workload": args.workload, "coarse_sites": Cc.nc, "nbasis": nb,
                      "nrhs": nrhs, "ms_median": ms, "tflops": flop / ms / 1e9,
                      "GBs_algorithmic": abytes / ms / 1e6, "flop_per_launch": flop,
                      "bytes_per_launch": abytes}))
    Cc.close()
    ctx.close()


def run_kernel(args):
    """Kernel-only loop for profiling: `--kernel dhop_f32|dhop_f64|dhop_f16|mpcdagmpc_f32`
    at the workload's size, warmup + steps launches, no solver."""
    import torch

    from paper_2103_05034_gb300 import layout, ops
    from paper_2103_05034_gb300._lib import F16S, F32, F64, HOP_VARIANTS, DWFError

    w, U, b = build_workload(args.workload, 0)
    L, Ls = w["L"], w["Ls"]
    ctx = ops.Context(L, Ls, w["M5"], U)
    kind, prec_name = args.kernel.split("_")
    prec = {"f64": F64, "f32": F32, "f16": F16S}[prec_name]
    if args.hop_variant is not None:  # pinned (profiling one variant), no tuning launches
        ops.dwf_set_hop_variant(ctx, prec, args.hop_variant)
        variant, tuned_ms = args.hop_variant, None
    else:
        variant, tuned_ms = ops.dwf_autotune(ctx, prec, 10)
    if b is not None:
        inp = torch.from_numpy(layout.complex_to_real(layout.to_half(b, L, 1), prec)).cuda()
    else:  # paper-size lattice: Gaussian input drawn on the device (seeded)
        gen = torch.Generator(device="cuda").manual_seed(synth.SEED_SOURCE)
        inp = torch.randn(ctx.half_numel(), generator=gen, device="cuda",
                          dtype=torch.float32).to({F64: torch.float64, F32: torch.float32,
                                                   F16S: torch.float16}[prec])
    out = torch.zeros_like(inp)
    fn = {"dhop": lambda: ops.dwf_dhop(ctx, out, inp, 0),
          "mpcdagmpc": lambda: ops.dwf_mpcdag_mpc(ctx, out, inp, w["mf"])}[kind]
    if args.sweep_variants and kind == "dhop":
        # every tuning variant, one launch at a time with an L2 flush before each
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        wbytes = {F64: 16, F32: 8, F16S: 4}[prec]
        nbytes = ctx.Vh * (Ls * 24 * wbytes + 72 * (16 if prec == F64 else 8))
        for v in range(HOP_VARIANTS if prec != F64 else 1):
            try:
                ops.dwf_set_hop_variant(ctx, prec, v)
            except DWFError:  # the variant does not tile this lattice
                continue
            for _ in range(3):
                fn()
            ts = []
            for k in range(10):
                flush.fill_(float(k))
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                fn()
                z.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(z))
            ms = float(np.median(ts))
            print(json.dumps({"kernel": args.kernel, "variant": v, "ms_median": ms,
                              "GBs_algorithmic": nbytes / ms / 1e6}))
        ops.dwf_set_hop_variant(ctx, prec, variant)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"kernel": args.kernel, "workload": args.workload, "ms_per_call": ms,
                      "hop_variant": variant, "autotune_ms": tuned_ms}))
    ctx.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dwf_16x16x16x32_ls16", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-mg-compare", dest="mg_compare", action="store_false",
                    help="skip the one-off FP64 RB-CG vs HDCR time-to-solution comparison")
    ap.add_argument("--kernel", default=None,
                    help="profile mode: dhop_f32, dhop_f64, dhop_f16, mpcdagmpc_f32, coarse_tf32 or coarse_f32 alone")
    ap.add_argument("--hop-variant", type=int, default=None,
                    help="with --kernel dhop_*: pin this hopping-kernel variant instead of autotuning")
    ap.add_argument("--sweep-variants", action="store_true",
                    help="with --kernel dhop_*: time every hopping-kernel tuning variant")
    args = ap.parse_args(argv)
    if args.kernel:
        if args.kernel.startswith("coarse_"):
            return run_coarse_kernel(args)
        return run_kernel(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
