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
# The oracle cannot hold a field of the 48^3 x 96 x 24 workload (49 GB per FP64
# vector), so its CPU legs run on a sample lattice with the same Ls and link
# recipe: 8^3 x 16 x Ls, about a second of numpy per D_hop.
SAMPLE_L = (8, 8, 8, 16)


def oracle_sample(w, seed):
    """(L, U, psi) of the oracle's sample lattice for workload w."""
    L = w["L"] if int(np.prod(w["L"])) * w["Ls"] <= (1 << 22) else SAMPLE_L
    U = synth.random_gauge(L, w["eps"], synth.SEED_GAUGE, ape_steps=w["ape"])
    return L, U, synth.gaussian_spinor(L, w["Ls"], seed)


def oracle_dhop_sample(L, Ls, U, psi):
    """One full-lattice FP64 oracle D_hop; returns (seconds, algorithmic bytes)."""
    from oracle import dwf
    t0 = time.perf_counter()
    dwf.dhop(U, psi)
    dt = time.perf_counter() - t0
    V4 = int(np.prod(L))
    nbytes = V4 * Ls * (24 * 16) + V4 * 8 * 9 * 16  # FP64 spinors in+out, 8 links per site
    return dt, nbytes


def _oracle_worker(args):
    """Spawned worker: `reps` oracle D_hops of its own sample; (seconds, bytes)."""
    name, seed, reps = args
    w = synth.WORKLOADS[name]
    L, U, psi = oracle_sample(w, seed)
    tot, nb = 0.0, 0
    for _ in range(reps):
        dt, b = oracle_dhop_sample(L, w["Ls"], U, psi)
        tot += dt
        nb += b
    return tot, nb


def cpu_baseline_leg(name):
    """The oracle's FP64 D_hop on the host cores: one process, then one process
    per core (spawned, single-threaded numpy each), every process on its own
    sample; value = the all-cores throughput in GB/s of algorithmic bytes."""
    import multiprocessing as mp
    w = synth.WORKLOADS[name]
    L, U, psi = oracle_sample(w, synth.SEED_SOURCE)
    oracle_dhop_sample(L, w["Ls"], U, psi)  # warm
    reps1 = 3
    t1, b1 = 0.0, 0
    for _ in range(reps1):
        dt, nb = oracle_dhop_sample(L, w["Ls"], U, psi)
        t1 += dt
        b1 += nb
    v1 = b1 / t1 / 1e9
    ncpu = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    env_before = os.environ.get("OMP_NUM_THREADS")
    os.environ["OMP_NUM_THREADS"] = "1"  # inherited by the spawned workers
    try:
        t0 = time.perf_counter()
        with ctx.Pool(ncpu) as pool:
            res = pool.map(_oracle_worker, [(name, synth.SEED_SOURCE + 10 + i, reps1) for i in range(ncpu)])
        wall = time.perf_counter() - t0
    finally:
        if env_before is None:
            os.environ.pop("OMP_NUM_THREADS", None)
        else:
            os.environ["OMP_NUM_THREADS"] = env_before
    vall = sum(r[1] for r in res) / max(r[0] for r in res) / 1e9
    V5w = int(np.prod(w["L"])) * w["Ls"]
    V5s = int(np.prod(L)) * w["Ls"]
    per_site_s = t1 / reps1 / V5s
    sample = f"FP64 numpy oracle D_hop on a {'x'.join(map(str, L))}x{w['Ls']} lattice with the workload's link recipe"
    return {"value": vall, "unit": UNIT, "cores": ncpu, "kind": "oracle",
            "sample": sample + f": {reps1} per process, {ncpu} spawned single-threaded processes",
            "single_core": {"value": v1, "cores": 1, "seconds_per_dhop": t1 / reps1},
            "all_cores_wall_s": wall,
            "workload_dhop_seconds_extrapolated": {
                "one_core": per_site_s * V5w, "all_cores": per_site_s * V5w * v1 / vall,
                "note": f"per-5D-site time of the sample x the workload's {V5w} sites (extrapolated)"}}


def run_reference(args):
    """--impl reference: the oracle (FP64 numpy, one process) timed on the host
    cores, each step one full-lattice D_hop on the sample lattice of the
    workload (its own lattice when that is small)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = synth.WORKLOADS[args.workload]
    L, U, psi = oracle_sample(w, synth.SEED_SOURCE)
    for _ in range(args.warmup):
        oracle_dhop_sample(L, w["Ls"], U, psi)
    times, nbytes = [], 0
    for _ in range(args.steps):
        dt, nb = oracle_dhop_sample(L, w["Ls"], U, psi)
        times.append(dt)
        nbytes += nb
    tot = sum(times)
    val = nbytes / tot / 1e9
    sample = f"one full-lattice FP64 numpy D_hop at {'x'.join(map(str, L))}x{w['Ls']} per step"
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "oracle": "numpy FP64",
                                             "sample_lattice": list(L), "l2": "n/a (host)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- MG vs FP64 RB-CG
# HDCR parameters: 4^4 x Ls blocks, 16 + 16 basis vectors from the paper's
# recursive Chebyshev filter (m = 500, Delta = 100, lambda_lo = 0.05, Tables 1
# and 12), pGCR(32), and the coarse CG on A^2 to 2e-3 started from the
# Chebyshev-Lanczos deflation guess (Sec. 3.5).  The smoother interval is
# lowered to [0.05, lambda_max] with order 40: on the smeared-random stand-in
# fields the Shamir bulk modes reach H^2 ~ 0.04, below the paper's [0.5, 60]
# (with [0.2, lambda_max] or [0.5, lambda_max] the solve stalls).  Deflation:
# 64 Ritz vectors from 160 Lanczos steps at 16^3 x 32 x 16; 128 from 256 at
# 24^3 x 48 x 24, where 64 did not keep the coarse solve short (the paper
# notes the same growth with volume).
MG_PARAMS = dict(block=(4, 4, 4, 4), nbasis=32, subspace="recursive", filter_order=500, delta=100,
                 lambda_lo=0.05, smooth=(0.05, None, 40), coarse_tol=2e-3, coarse_maxiter=5000,
                 nkrylov=32, maxiter=300, coarse_solver="deflated", deflation=(64, 160, 10, 0.05))
MG_PARAMS_LARGE = dict(MG_PARAMS, deflation=(128, 256, 10, 0.05))
# Algorithm F (Table 3): 2^4 x 1 blocks with 24 4D vectors (Wilson mass
# -0.95, lambda_lo 4), then one level-1 site x Ls with 32 vectors; the fine
# smoother as for HDCR; a level-1 smoother of order 4; the W-cycle of two
# level-1 GCR iterations; red-black CG on the level-2 operator
HYBRID_PARAMS = dict(block=(2, 2, 2, 2), nbasis4=24, nbasis1=32, mass4=-0.95, filter4=(4.0, 60.0, 60),
                     filter1=(0.5, None, 40), smooth=(0.05, None, 40), smooth1=(0.05, None, 4), kcycle=2,
                     coarse_tol=0.02, coarse_maxiter=5000, nkrylov=32, maxiter=300, coarse_solver="rb")
# At 24^3 x 48 x 24 a level-1 smoother of order 8 and the level-2 CG to 0.05
# (the paper's looser coarse tolerance) take the solve from 103 outer
# iterations (21012 level-2 iterations) to 66 (5066)
HYBRID_PARAMS_LARGE = dict(HYBRID_PARAMS, smooth1=(0.05, None, 8), coarse_tol=0.05)


def mg_vs_fp64(ctx, w, bd, tol, params=MG_PARAMS, eta_seed=None):
    """Time to a true residual of `tol` on the same GPU and source: plain FP64
    red-black CG (and the mixed-precision one) against HDCR setup + solve
    (mixed precision), and setup + two solves (the second source a shifted
    copy of the first).  One run each, outside the timed steps; every call
    synchronises, so host-clock times are GPU times.  The multigrid's random
    inputs (the power method's start vector and the subspace Gaussian) are
    drawn on the device by torch's seeded generator."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import (COARSE_CG, COARSE_DEFLATED, COARSE_RB, F32, SOLVE_F64,
                                             SOLVE_MIXED_F32, SUBSPACE_BATCH, SUBSPACE_RECURSIVE)

    mf = w["mf"]
    out = {"workload": "x".join(map(str, w["L"])) + f"x{w['Ls']}", "mf": mf}
    x = torch.zeros_like(bd)
    for pol, name in ((SOLVE_F64, "fp64_rbcg"), (SOLVE_MIXED_F32, "mixed_rbcg")):
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ops.rbcg_solve(ctx, x, bd, mf, tol, 100000, pol)
        out[name + "_s"] = time.perf_counter() - t0
        out[name + "_iterations"] = st["iterations"]
        out[name + "_true_residual"] = st["true_residual"]
    p = dict(params)
    nb = p["nbasis"]
    recursive = p["subspace"] == "recursive"
    gen = torch.Generator(device="cuda").manual_seed(77)
    v0 = torch.randn(bd.numel(), generator=gen, device="cuda", dtype=torch.float64)
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_BASIS if eta_seed is None else eta_seed)
    eta = torch.randn(bd.numel() * (1 if recursive else nb), generator=gen, device="cuda", dtype=torch.float64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # lambda_max of D^dag D bounds the filter and smoother intervals (power
    # method in FP32, 100 iterations, 10 % margin: the Rayleigh quotient
    # approaches the top of the spectrum from below)
    lmax = ops.dwf_power_max(ctx, v0, mf, 100, F32) * 1.10
    cs = {"cg": COARSE_CG, "rb": COARSE_RB, "deflated": COARSE_DEFLATED}[p["coarse_solver"]]
    prm = ops.mg_params(p["block"], nb, mf, subspace_mode=SUBSPACE_RECURSIVE if recursive else SUBSPACE_BATCH,
                        lambda_lo=p["lambda_lo"], lambda_max=lmax, filter_order=p["filter_order"],
                        delta=p["delta"], smooth=(p["smooth"][0], lmax, p["smooth"][2]),
                        coarse_tol=p["coarse_tol"], coarse_maxiter=p["coarse_maxiter"], nkrylov=p["nkrylov"],
                        maxiter=p["maxiter"], coarse_solver=cs,
                        deflation=p["deflation"] if cs == COARSE_DEFLATED else (0, 0, 0, 0.0))
    G = ops.MG(ctx, prm, eta)
    del eta
    torch.cuda.synchronize()
    out["mg_setup_s"] = time.perf_counter() - t0
    solves = []
    for k in range(2):
        src = bd if k == 0 else torch.roll(bd, 24)  # a second source: the first shifted by one complex spinor row
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sm = ops.mg_solve(G, x, src, tol)
        solves.append((time.perf_counter() - t0, sm))
    (t1, s1), (t2, s2) = solves
    out.update({"mg_solve_s": t1, "mg_outer_iterations": s1["iterations"],
                "mg_coarse_iterations": s1["coarse_iterations"], "mg_fine_matmuls": s1["fine_matmuls"],
                "mg_true_residual": s1["true_residual"], "mg_subspace_s": s1["setup_seconds"],
                "mg_coarse_op_s": s1["coarse_op_seconds"], "mg_graph_replays": s1["graph_replays"],
                "mg_second_solve_s": t2, "mg_second_solve_outer_iterations": s2["iterations"],
                "mg_second_solve_true_residual": s2["true_residual"]})
    out["mg_total_s"] = out["mg_setup_s"] + t1
    out["mg_setup_plus_two_solves_s"] = out["mg_total_s"] + t2
    # The two-flavour determinant needs two solves of the unsquared operator
    # (the MG solve) against one of the squared operator (CGNR): the paper's
    # break-even criterion is setup + two MG solves against one CGNR solve.
    out["speedup_fp64_over_mg"] = out["fp64_rbcg_s"] / out["mg_total_s"]
    out["speedup_fp64_over_mg_setup_two_solves"] = out["fp64_rbcg_s"] / out["mg_setup_plus_two_solves_s"]
    out["lambda_max"] = lmax
    out["params"] = {k: v for k, v in p.items()}
    G.close()
    return out


def hop_variant_label(v, Ls):
    """The FP32 hopping kernel that tuning variant v launches (the variant table
    of csrc/dhop_impl.cuh: register cap and inner-loop form)."""
    regs = {1: 96, 2: 80, 3: 64, 4: 128, 5: 96, 6: 64, 7: 80, 8: 64, 9: 80, 10: 128, 11: 112, 12: 96, 14: 64, 15: 80,
            16: 64, 17: 80, 18: 56, 19: 48, 23: 64, 24: 64, 25: 80}.get(v, 0)
    if 10 <= v <= 13 or 20 <= v <= 22:
        form = "two s-slices per thread, packed FP32" + (", cp.async staging" if v >= 20 else "")
        name = "hop_kernel_pair"
    else:
        form = ("scalar" if v in (0, 1, 2, 3, 18, 19) else "neighbour prefetch" if v in (4, 5)
                else "packed FP32 (re, im)" if v in (6, 7) else "2^4 hypercube tiles" if v in (8, 9)
                else "y-row CTAs" if 14 <= v <= 17 else "L2 prefetch")
        name = "hop_kernel"
    cap = f"{regs} registers" if regs else "no register cap"
    return f"dwfk::{name}<F32, Ls={Ls}> (dwf_dhop, plain epilogue; variant {v}: {form}, {cap})"


def hybrid_vs_fp64(ctx, w, bd, tol, fp64_s, params=HYBRID_PARAMS):
    """Algorithm F (the hybrid three-level multigrid) on the source of
    mg_vs_fp64: setup (4D level and level-2 parts), two solves, against the
    FP64 red-black CG time measured there.  One run each, host clock around
    synchronising calls."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import COARSE_CG, COARSE_RB, F32

    p = dict(params)
    mf = w["mf"]
    L, Ls = w["L"], w["Ls"]
    gen = torch.Generator(device="cuda").manual_seed(77)
    v0 = torch.randn(bd.numel(), generator=gen, device="cuda", dtype=torch.float64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lmax = ops.dwf_power_max(ctx, v0, mf, 100, F32) * 1.10
    del v0
    cs = {"cg": COARSE_CG, "rb": COARSE_RB}[p["coarse_solver"]]
    prm = ops.mg_params(p["block"], 0, mf, smooth=(p["smooth"][0], lmax, p["smooth"][2]), coarse_tol=p["coarse_tol"],
                        coarse_maxiter=p["coarse_maxiter"], nkrylov=p["nkrylov"], maxiter=p["maxiter"],
                        coarse_solver=cs)
    f1 = p["filter1"]
    hp = ops.hybrid_params(p["block"], p["nbasis4"], p["nbasis1"], mass4=p["mass4"], filter4=p["filter4"],
                           filter1=(f1[0], lmax, f1[2]), smooth1=(p["smooth1"][0], lmax, p["smooth1"][2]),
                           kcycle=p["kcycle"])
    nc1 = int(np.prod([L[m] // p["block"][m] for m in range(4)]))
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_BASIS)
    eta4 = torch.randn(2 * 2 * ctx.Vh * 12 * p["nbasis4"], generator=gen, device="cuda", dtype=torch.float64)
    eta1 = torch.randn(2 * nc1 * p["nbasis4"] * Ls * p["nbasis1"], generator=gen, device="cuda", dtype=torch.float64)
    G = ops.HybridMG(ctx, prm, hp, eta4, eta1)
    del eta4, eta1
    torch.cuda.synchronize()
    out = {"workload": "x".join(map(str, L)) + f"x{Ls}", "mf": mf, "setup_s": time.perf_counter() - t0}
    x = torch.zeros_like(bd)
    for k in range(2):
        src = bd if k == 0 else torch.roll(bd, 24)
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ops.mg_solve(G, x, src, tol)
        key = "solve" if k == 0 else "second_solve"
        out[key + "_s"] = time.perf_counter() - t0
        out[key + "_outer_iterations"] = st["iterations"]
        out[key + "_level2_iterations"] = st["coarse_iterations"]
        out[key + "_fine_matmuls"] = st["fine_matmuls"]
        out[key + "_true_residual"] = st["true_residual"]
    out["setup_4d_level_s"] = st["setup_seconds"]
    out["setup_level2_s"] = st["coarse_op_seconds"]
    out["total_s"] = out["setup_s"] + out["solve_s"]
    out["setup_plus_two_solves_s"] = out["total_s"] + out["second_solve_s"]
    out["fp64_rbcg_s"] = fp64_s
    out["speedup_fp64_over_hybrid"] = fp64_s / out["total_s"]
    out["speedup_fp64_over_hybrid_setup_two_solves"] = fp64_s / out["setup_plus_two_solves_s"]
    out["lambda_max"] = lmax
    out["params"] = {k: v for k, v in p.items()}
    G.close()
    return out


# ---------------------------------------------------------------------- GPU leg
def reduce_ranks(seconds, nbytes, device):
    """Whole-job figures of N independent replicas: the slowest rank's time
    and the bytes of all ranks (every rank calls this with its own values)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    b = torch.tensor([nbytes], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return float(t[0]), float(b[0])


def host_mem_available():
    """MemAvailable of the host in bytes (0 if unknown)."""
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def device_source(ctx, w, b, rank, dev):
    """The FP64 full-field source on the device: the host Gaussian of the
    workload when it has one, else a Gaussian drawn on the device (seeded)."""
    import torch

    from paper_2103_05034_gb300 import layout
    from paper_2103_05034_gb300._lib import F64
    if b is not None:
        return torch.from_numpy(layout.complex_to_real(layout.to_full(b, w["L"]), F64)).to(dev)
    gen = torch.Generator(device=dev).manual_seed(synth.SEED_SOURCE + rank)
    return torch.randn(2 * ctx.half_numel(), generator=gen, device=dev, dtype=torch.float64)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import F32, SOLVE_F64, SOLVE_MIXED_F32

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
    del U
    hop_variant, hop_tuned_ms = ops.dwf_autotune(ctx, F32, 20)  # setup, not timed
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # ---- dominant kernel first (before the solver's workspace exists): the
    # FP32 hopping term, timed alone with an L2 flush before each launch
    gen = torch.Generator(device=dev).manual_seed(synth.SEED_SOURCE + 1)
    inp = torch.randn(ctx.half_numel(), generator=gen, device=dev, dtype=torch.float32)
    out = torch.zeros_like(inp)
    hop_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for _ in range(3):
        ops.dwf_dhop(ctx, out, inp, 0)
    for k, (e0, e1) in enumerate(hop_ev):
        flush.fill_(float(k))
        e0.record(stream)
        ops.dwf_dhop(ctx, out, inp, 0)
        e1.record(stream)
    torch.cuda.synchronize()
    hop_ms = float(np.mean([a.elapsed_time(bq) for a, bq in hop_ev]))
    del inp, out
    torch.cuda.empty_cache()
    Vh = ctx.Vh
    hop_alg_bytes = Vh * (Ls * 24 * 8 + 72 * 8)
    peaks, peak_kind = measured_peaks()
    achieved = hop_alg_bytes / (hop_ms / 1e3) / 1e9
    shash = source_hash("paper_2103_05034_gb300/csrc/dhop_impl.cuh", "paper_2103_05034_gb300/csrc/dhop_pair.cuh")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": profile_traffic(f"hop_kernel_f32_ls{Ls}_v{hop_variant}_{args.workload}", shash),
                "kernel": hop_variant_label(hop_variant, Ls),
                "launch_ms": hop_ms, "algorithmic_bytes_per_launch": hop_alg_bytes,
                "peak_source": f"{peak_kind} hbm_gbs (burst copy)", "source_hash": shash}

    # ---- the timed steps: a block of the mixed-precision red-black CG
    bd = device_source(ctx, w, b, rank, dev)
    xd = torch.zeros_like(bd)
    step_iters = args.step_iters if args.step_iters > 0 else 100000

    def step(x, bb):
        return ops.rbcg_solve(ctx, x, bb, mf, args.tol, step_iters, SOLVE_MIXED_F32, noconv_ok=True)

    for _ in range(args.warmup):
        step(xd, bd)
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
        st = step(xd, bd)
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
        t_max, tot_bytes = reduce_ranks(t_dev, hop_bytes, dev)
    value = tot_bytes / t_max / 1e9

    line = None
    legs = {}
    if rank == 0 and args.legs:
        # time to the tolerance on the same GPU: the mixed-precision solve, and
        # FP64 red-black CG (whole solve with --fp64-full; otherwise a
        # 16-iteration block whose per-iteration cost projects the solve)
        try:
            xd.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sm = ops.rbcg_solve(ctx, xd, bd, mf, args.tol, 100000, SOLVE_MIXED_F32)
            torch.cuda.synchronize()
            legs["mixed_rbcg_to_tol"] = {"seconds": time.perf_counter() - t0, "iterations": sm["iterations"],
                                         "reliable_updates": sm["reliable_updates"],
                                         "true_residual": sm["true_residual"], "fine_matmuls": sm["fine_matmuls"]}
        except Exception as e:
            legs["mixed_rbcg_to_tol"] = {"error": str(e)}
        try:
            legs["fp64_rbcg"] = fp64_rbcg_leg(ops, ctx, xd, bd, mf, args, legs.get("mixed_rbcg_to_tol", {}))
        except Exception as e:
            legs["fp64_rbcg"] = {"error": str(e)}

    # ---- end to end through the C ABI with host buffers (the library copies b
    # in and x out inside the call); the device copies are freed first
    n_full = bd.numel()
    e2e_steps = min(args.steps, args.e2e_steps)
    need = 2 * n_full * 8
    avail = host_mem_available()
    # page-locked buffers (full-speed DMA over the CPU-GPU link) when at least
    # 64 GB of host memory stays free beside them; pageable otherwise
    pinned = avail > need + 64e9
    try:
        bh = torch.empty(n_full, dtype=torch.float64, pin_memory=pinned)
        xh = torch.zeros(n_full, dtype=torch.float64, pin_memory=pinned)
    except RuntimeError:
        pinned = False
        bh = torch.empty(n_full, dtype=torch.float64)
        xh = torch.zeros(n_full, dtype=torch.float64)
    bh.copy_(bd)  # the same source, now in host memory
    del bd, xd
    torch.cuda.empty_cache()
    step(xh, bh)  # warm (workspace for host buffers)
    ops.dwf_reset_counters(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(xh, bh)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    _, e2e_bytes = ops.dwf_counters(ctx)
    if world > 1:
        t_e2e, e2e_bytes = reduce_ranks(t_e2e, e2e_bytes, dev)
    e2e = {"value": e2e_bytes / t_e2e / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(bh.numel() * 8),
           "d2h_bytes_per_step": int(xh.numel() * 8), "steps": e2e_steps,
           "note": f"rbcg_solve on {'pinned' if pinned else 'pageable'} host b and x: H2D of b and D2H of x "
                   f"inside the call, host clock"}
    del bh, xh
    if pinned and hasattr(torch._C, "_host_emptyCache"):
        torch._C._host_emptyCache()  # hand the page-locked buffers back to the host
    ctx.close()
    torch.cuda.empty_cache()

    if rank == 0:
        s0 = stats[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "lattice": list(L), "Ls": Ls, "M5": M5, "mf": mf,
                       "step": (f"rbcg_solve from x = 0 stopped after {args.step_iters} CG iterations "
                                f"(source preparation, FP32 inner CG, FP64 reliable updates, reconstruction, "
                                f"FP64 true residual)" if args.step_iters > 0 else
                                f"rbcg_solve to a true residual of {args.tol}"),
                       "tol_true_residual": args.tol,
                       "l2": "inputs larger than L2 (one FP32 half field 12 GB) and 512 MB flush before each step",
                       "parallelism": f"replicas{world}",
                       "hop_variant_f32": hop_variant, "hop_autotune_ms": hop_tuned_ms},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "roofline": roofline,
            "e2e": e2e,
            "step_solve": {"iterations": s0["iterations"], "reliable_updates": s0["reliable_updates"],
                           "true_residual": s0["true_residual"], "fine_matmuls": s0["fine_matmuls"],
                           "seconds": t_max / args.steps, "wall_seconds_all_steps": t_wall},
        }
        line.update(legs)
        # legs on the 16^3 x 32 x 16 workload (the fields of the 48^3 one are
        # too large for their setups): tensor-core coarse stencil, batched
        # pseudofermion solves, MG against FP64 RB-CG
        small = "dwf_16x16x16x32_ls16"
        try:
            if not args.legs:
                raise StopIteration
            ws_, Us, bs = build_workload(small, 0)
            cs = ops.Context(ws_["L"], ws_["Ls"], ws_["M5"], Us)
            ops.dwf_autotune(cs, F32, 10)
            try:
                line["coarse_apply_tc"] = coarse_apply_measure(cs, ws_, "tf32", 3, 20)
            except Exception as e:
                line["coarse_apply_tc"] = {"error": str(e)}
            try:
                line["batched_solves"] = batched_solves_measure(cs, 1e-10)
            except Exception as e:
                line["batched_solves"] = {"error": str(e)}
            if args.mg_compare:
                try:
                    bsd = device_source(cs, ws_, bs, 0, dev)
                    line["mg_vs_fp64"] = mg_vs_fp64(cs, ws_, bsd, args.tol)
                    line["hybrid_vs_fp64"] = hybrid_vs_fp64(cs, ws_, bsd, args.tol, line["mg_vs_fp64"]["fp64_rbcg_s"])
                    del bsd
                except Exception as e:  # reported, not hidden: the line says what failed
                    line.setdefault("mg_vs_fp64", {"error": str(e)})
                    line.setdefault("hybrid_vs_fp64", {"error": str(e)})
            cs.close()
        except StopIteration:
            pass
        except Exception as e:
            line["small_workload_legs"] = {"error": str(e)}
        torch.cuda.empty_cache()
        if args.legs and args.mg_compare and args.mg_large:
            # the multigrid at the largest volume its 32-vector FP32 basis fits
            # (24^3 x 48 x 24, the 48^3 workload's Ls and mass) against FP64 RB-CG
            try:
                large = "dwf_24x24x24x48_ls24"
                wl, Ul, _ = build_workload(large, 0)
                cl = ops.Context(wl["L"], wl["Ls"], wl["M5"], Ul)
                del Ul
                ops.dwf_autotune(cl, F32, 10)
                bl = device_source(cl, wl, None, 0, dev)
                line["mg_vs_fp64_large"] = mg_vs_fp64(cl, wl, bl, args.tol, MG_PARAMS_LARGE)
                if args.hybrid_large:
                    try:
                        line["hybrid_vs_fp64_large"] = hybrid_vs_fp64(cl, wl, bl, args.tol,
                                                                      line["mg_vs_fp64_large"]["fp64_rbcg_s"],
                                                                      HYBRID_PARAMS_LARGE)
                    except Exception as e:
                        line["hybrid_vs_fp64_large"] = {"error": str(e)}
                del bl
                cl.close()
            except Exception as e:
                line["mg_vs_fp64_large"] = {"error": str(e)}
        if args.cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline_leg(args.workload)
            line["host"] = {"cpu_count": os.cpu_count(), "mem_available_gb": host_mem_available() / 1e9}
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None:
        print(json.dumps(line), flush=True)
    return 0


def fp64_rbcg_leg(ops, ctx, xd, bd, mf, args, mixed):
    """FP64 red-black CG on the same source.  With --fp64-full the whole solve
    to the tolerance; otherwise blocks of 8 and 16 iterations give the cost of
    an FP64 iteration (their difference / 8) and of the fixed work (source
    preparation, reconstruction, true residual), and the solve time is
    projected with the mixed solve's iteration count (FP64 CG needs the same
    count here to within a few per cent: 336 against 336 at 16^3 x 32 x 16)."""
    import torch

    from paper_2103_05034_gb300._lib import SOLVE_F64

    def run(maxiter):
        xd.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = ops.rbcg_solve(ctx, xd, bd, mf, args.tol, maxiter, SOLVE_F64, noconv_ok=True)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, st

    if args.fp64_full:
        sec, st = run(100000)
        return {"seconds": sec, "iterations": st["iterations"], "true_residual": st["true_residual"],
                "measured": "whole solve"}
    t8, _ = run(8)
    t16, _ = run(16)
    per_it = (t16 - t8) / 8
    fixed = t8 - 8 * per_it
    out = {"seconds_per_iteration": per_it, "fixed_seconds": fixed, "measured": "blocks of 8 and 16 iterations"}
    if "iterations" in mixed:
        out["projected_seconds_to_tol"] = fixed + per_it * mixed["iterations"]
        out["projected_with_iterations"] = mixed["iterations"]
        out["speedup_mixed_over_fp64_projected"] = out["projected_seconds_to_tol"] / mixed["seconds"]
    return out


def batched_solves_measure(ctx, tol):
    """The pseudofermion solves of the force workload: x_i = (M_pc(m_i)^dag
    M_pc(m_i))^-1 phi_i for the Hasenbusch masses 0.01, 0.05, 0.2, 1.0 on the
    context's lattice (Gaussian FP64 phi_i, seeded), once as one batch
    (rbcg_normal_solve_batch) and once as four single-system solves; FP32
    inner CG, FP64 reliable updates, tol on the FP64 residual.  Wall time of
    each after one warm call, and the algorithmic hopping bytes each moved."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import SOLVE_MIXED_F32

    masses = [0.01, 0.05, 0.2, 1.0]
    n, nh = len(masses), ctx.half_numel()
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_SOURCE + 5)
    phi = torch.randn(n * nh, generator=gen, device="cuda", dtype=torch.float64)
    x = torch.zeros_like(phi)
    xs, ps = x.view(n, -1), phi.view(n, -1)

    def batch():
        return ops.rbcg_normal_solve_batch(ctx, x, phi, masses, tol, 100000, SOLVE_MIXED_F32)

    def singles():
        return [ops.rbcg_normal_solve(ctx, xs[i], ps[i], m, tol, 100000, SOLVE_MIXED_F32)
                for i, m in enumerate(masses)]

    res = {"masses": masses, "tol": tol, "policy": "FP32 inner, FP64 reliable updates"}
    for name, fn in (("batch", batch), ("singles", singles)):
        fn()
        torch.cuda.synchronize()
        ops.dwf_reset_counters(ctx)
        t0 = time.perf_counter()
        st = fn()
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        launches, hbytes = ops.dwf_counters(ctx)
        res[name] = {"seconds": sec, "iterations": [s["iterations"] for s in st],
                     "reliable_updates": [s["reliable_updates"] for s in st],
                     "true_residual": [s["true_residual"] for s in st],
                     "hop_GBs_algorithmic": hbytes / sec / 1e9, "launches": int(launches)}
    res["speedup_batch_vs_singles"] = res["singles"]["seconds"] / res["batch"]["seconds"]
    return res


def coarse_apply_measure(ctx, w, prec_name, warmup, steps):
    """The little Dirac operator of H_DW on the context's lattice (4^4 x Ls
    blocks, 32 basis vectors from Gaussians, chirality-projected and
    block-orthonormalised) applied to 32 right-hand sides; median CUDA-event
    time of `steps` calls with L2 flushed before each."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import F32, TF32

    mf = w["mf"]
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
    prec = {"tf32": TF32, "f32": F32}[prec_name]
    inp = torch.randn(2 * Cc.nc * nb * nrhs, generator=gen, device="cuda", dtype=torch.float32)
    out = torch.zeros_like(inp)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(max(warmup, 1)):
        ops.coarse_apply(Cc, out, inp, nrhs, prec)
    ts = []
    for k in range(steps):
        flush.fill_(float(k))
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ops.coarse_apply(Cc, out, inp, nrhs, prec)
        z.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(z))
    ops.coarse_apply_status(Cc)  # raises if a bounded wait of any timed call gave up
    ms = float(np.median(ts))
    flop = 8.0 * 9 * nb * nb * nrhs * Cc.nc
    abytes = Cc.nc * 9 * nb * nb * 8 + 2 * Cc.nc * nb * nrhs * 8  # FP32 operator + in/out vectors
    res = {"kernel": f"coarse_{prec_name}", "coarse_sites": Cc.nc, "nbasis": nb, "nrhs": nrhs,
           "ms_median": ms, "tflops": flop / ms / 1e9, "GBs_algorithmic": abytes / ms / 1e6,
           "flop_per_launch": flop, "bytes_per_launch": abytes}
    peaks, kind = measured_peaks()
    if prec_name == "tf32" and "bf16_tflops" in peaks:
        tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25  # nominal dense TF32 / BF16 ratio
        res["frac_of_tf32_peak"] = res["tflops"] / tf32_peak
        res["tf32_peak_tflops"] = tf32_peak
        res["peak_source"] = f"{kind} bf16_tflops x 1.1/2.25 (nominal TF32/BF16 dense ratio)"
    res["frac_of_hbm"] = res["GBs_algorithmic"] / peaks["hbm_gbs"]
    Cc.close()
    return res


def run_coarse_kernel(args):
    """`--kernel coarse_tf32|coarse_f32`: the coarse stencil alone (see
    coarse_apply_measure), warmup + steps calls."""
    from paper_2103_05034_gb300 import ops

    w, U, _ = build_workload(args.workload, 0)
    ctx = ops.Context(w["L"], w["Ls"], w["M5"], U)
    res = coarse_apply_measure(ctx, w, args.kernel.split("_")[1], args.warmup, args.steps)
    res["workload"] = args.workload
    print(json.dumps(res))
    ctx.close()


def run_rows(args):
    """`--rows`: every step of the hot path measured alone on the workload
    (CUDA events, L2 flushed before each timed call, median), with its
    algorithmic bytes or flops and the fraction of the measured peak, and the
    oracle's time for the same step on the small 4^4 x 8 lattice beside it.
    One JSON line per step."""
    import torch

    from oracle import cheby as o_cheby
    from oracle import dwf as o_dwf
    from paper_2103_05034_gb300 import layout, ops
    from paper_2103_05034_gb300._lib import (ARITH_FLOAT_FLOAT, ARITH_FP64, F16S, F32, F64, SOLVE_MIXED_F32,
                                             SUBSPACE_BATCH)

    # the rows use host-side inputs: a paper-size workload is replaced by the
    # 16^3 x 32 x 16 one
    name = args.workload if int(np.prod(synth.WORKLOADS[args.workload]["L"])) <= (1 << 20) else "dwf_16x16x16x32_ls16"
    args.workload = name
    w, U, b = build_workload(name, 0)
    L, Ls, M5, mf = w["L"], w["Ls"], w["M5"], w["mf"]
    ctx = ops.Context(L, Ls, M5, U)
    ops.dwf_autotune(ctx, F32, 10)
    ops.dwf_autotune(ctx, F16S, 10)
    peaks, kind = measured_peaks()
    hbm = peaks["hbm_gbs"]
    # FP64 and FP32 FMA rates of this GPU, measured by the library's own
    # FMA-chain microbenchmark (the denominators of the ALU-bound rows)
    fp64_peak, fp32_peak = ops.dwf_measure_fma_peaks()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_SOURCE)
    nh = ctx.half_numel()  # reals of one half field

    def field(n, dtype):
        return torch.randn(n, generator=gen, device="cuda", dtype=torch.float32).to(dtype)

    def timed(fn, reps=10):
        fn()
        torch.cuda.synchronize()
        ts = []
        for k in range(reps):
            flush.fill_(float(k))
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            z.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(z))
        return float(np.median(ts))

    def hop_bytes(fn):
        ops.dwf_reset_counters(ctx)
        fn()
        torch.cuda.synchronize()
        return ops.dwf_counters(ctx)[1]

    # CPU baseline beside each step: the oracle (FP64 numpy, one process) on the
    # small 4^4 x 8 lattice, in ns per 5D site
    sw = synth.WORKLOADS["dwf_4x4x4x4_ls8"]
    sL, sLs = sw["L"], sw["Ls"]
    sU = synth.random_gauge(sL, sw["eps"], synth.SEED_GAUGE)
    spsi = synth.gaussian_spinor(sL, sLs, synth.SEED_SOURCE)
    s5 = int(np.prod(sL)) * sLs

    def oracle_ns_per_site(fn, reps=3):
        t0 = time.perf_counter()
        for _ in range(reps):
            fn()
        return (time.perf_counter() - t0) / reps / s5 * 1e9

    rows = []

    def emit(row, entry, ms, work=None, unit=None, peak=None, bound=None, oracle=None, nrhs=1, **extra):
        d = {"row": row, "entry": entry, "workload": args.workload, "gpu_ms": ms}
        if work is not None:
            rate = work / (ms / 1e3) / (1e9 if unit == "GB/s" else 1e12)
            d.update({"work_per_call": work, "achieved": rate, "unit": unit, "bound": bound,
                      "peak": peak, "frac": rate / peak if peak else None})
        if oracle is not None:
            d["cpu_baseline_ns_per_5d_site"] = oracle  # the oracle, 4^4 x 8
            d["gpu_ns_per_5d_site"] = ms * 1e6 / (2 * ctx.Vh * Ls * nrhs)  # per right-hand side
        d.update(extra)
        rows.append(d)
        print(json.dumps(d), flush=True)

    emit("peaks", "FMA microbenchmark (dwf_measure_fma_peaks)", 0.0, fp64_tflops=fp64_peak, fp32_tflops=fp32_peak)
    V5h = ctx.Vh * Ls
    pe = o_dwf.project_parity(spsi, sL, 1)
    a32 = field(nh, torch.float32)
    o32 = torch.zeros_like(a32)
    a64, o64 = a32.double(), torch.zeros(nh, dtype=torch.float64, device="cuda")
    a16, o16 = a32.half(), torch.zeros(nh, dtype=torch.float16, device="cuda")
    f = lambda: ops.dwf_dhop(ctx, o32, a32, 0)
    emit("a1", "dwf_dhop F32", timed(f), hop_bytes(f), "GB/s", hbm, "hbm",
         oracle_ns_per_site(lambda: o_dwf.dhop(sU, pe)) * 2)
    f = lambda: ops.dwf_dhop(ctx, o16, a16, 0)
    emit("a1", "dwf_dhop F16 storage", timed(f), hop_bytes(f), "GB/s", hbm, "hbm")
    f = lambda: ops.dwf_dhop(ctx, o64, a64, 0)
    emit("a1", "dwf_dhop F64", timed(f, 5), 1320.0 * V5h, "TFLOP/s", fp64_peak, "fp64 alu (measured FMA rate)")
    # the same FP64 fields in float-float arithmetic on the FP32 units
    ops.set_f64_arithmetic(ctx, ARITH_FLOAT_FLOAT)
    v64, _ = ops.dwf_autotune(ctx, F64, 5)
    emit("a1", "dwf_dhop F64 storage, float-float arithmetic", timed(f, 5), 1320.0 * V5h, "TFLOP/s", fp64_peak,
         "fp64-equivalent flop over the measured FP64 rate", variant=v64)
    ops.set_f64_arithmetic(ctx, ARITH_FP64)
    f = lambda: ops.dwf_mooee_inv(ctx, o32, a32, mf)
    emit("a2", "dwf_mooee_inv F32", timed(f), V5h * 24 * 8.0, "GB/s", hbm, "hbm",
         oracle_ns_per_site(lambda: o_dwf.mooee_inv(spsi, M5, mf)))
    f = lambda: ops.dwf_mpcdag_mpc(ctx, o32, a32, mf)
    emit("a3", "dwf_mpcdag_mpc F32", timed(f), hop_bytes(f), "GB/s", hbm, "hbm",
         oracle_ns_per_site(lambda: o_dwf.mpc_dag(sU, o_dwf.mpc(sU, o_dwf.project_parity(spsi, sL, 0), M5, mf),
                                                   M5, mf)) * 2)
    bd = torch.from_numpy(layout.complex_to_real(layout.to_full(b, L), F64)).cuda()
    xd = torch.zeros_like(bd)
    st = {}

    def solve():
        xd.zero_()
        st.update(ops.rbcg_solve(ctx, xd, bd, mf, args.tol, 100000, SOLVE_MIXED_F32))
    ms = timed(solve, 3)
    emit("a4", "rbcg_solve mixed FP32/FP64", ms, hop_bytes(solve), "GB/s", hbm, "hbm",
         iterations=st["iterations"], true_residual=st["true_residual"],
         note="achieved = algorithmic hopping bytes of the whole solve / its time")
    bs = batched_solves_measure(ctx, 1e-10)
    emit("a4", "rbcg_normal_solve_batch, masses 0.01 0.05 0.2 1.0", 1e3 * bs["batch"]["seconds"],
         bs["batch"]["hop_GBs_algorithmic"] * bs["batch"]["seconds"] * 1e9, "GB/s", hbm, "hbm",
         singles_ms=1e3 * bs["singles"]["seconds"], speedup_batch_vs_singles=bs["speedup_batch_vs_singles"],
         iterations=bs["batch"]["iterations"], true_residual=bs["batch"]["true_residual"],
         note="one warm call timed on the host clock; achieved = algorithmic hopping bytes / time")
    # the unpreconditioned baseline of the Krylov comparison (FP64 CGNR on the
    # full lattice), one call on the host clock
    ops.dwf_reset_counters(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sc = ops.cgnr_solve(ctx, xd, bd, mf, args.tol, 100000)
    torch.cuda.synchronize()
    t_cg = time.perf_counter() - t0
    emit("a4", "cgnr_solve unpreconditioned FP64 (full lattice)", 1e3 * t_cg, ops.dwf_counters(ctx)[1], "GB/s",
         hbm, "hbm", iterations=sc["iterations"], true_residual=sc["true_residual"],
         fine_matmuls=sc["fine_matmuls"], rbcg_iterations=st["iterations"],
         note="FP64 hopping launches are ALU-bound on GB300; compare iterations with the red-black row")
    f = lambda: ops.dwf_norm2(ctx, a32)
    emit("a5", "dwf_norm2 F32 (half field)", timed(f), nh * 4.0, "GB/s", hbm, "hbm")
    f = lambda: ops.dwf_cdot(ctx, a64, a64)
    emit("a5", "dwf_cdot F64 (half field)", timed(f), 2 * nh * 8.0, "GB/s", hbm, "hbm")
    full32 = field(2 * nh, torch.float32)
    fo32 = torch.zeros_like(full32)
    f = lambda: ops.dwf_hdw(ctx, fo32, full32, mf)
    emit("a6", "dwf_hdw F32 (full field)", timed(f), hop_bytes(f), "GB/s", hbm, "hbm",
         oracle_ns_per_site(lambda: o_dwf.hdw(sU, spsi, M5, mf)))
    v0 = torch.from_numpy(layout.complex_to_real(layout.to_full(synth.gaussian_spinor(L, Ls, 77), L), F64)).cuda()
    f = lambda: ops.dwf_power_max(ctx, v0, mf, 100, F32)
    emit("a7", "dwf_power_max F32, 100 iterations", timed(f, 3), hop_bytes(f), "GB/s", hbm, "hbm")
    nr = 8
    fin = field(2 * nh * nr, torch.float32)
    fout = torch.zeros_like(fin)
    f = lambda: ops.cheby_filter(ctx, fout, fin, nr, 0.02, 60.0, 60, mf)
    emit("a8", f"cheby_filter F32, order 60, {nr} RHS", timed(f, 3), hop_bytes(f), "GB/s", hbm, "hbm",
         oracle_ns_per_site(lambda: o_cheby.cheby_filter(lambda v: o_dwf.mdagm(sU, v, M5, mf), spsi, 4, 0.02,
                                                          60.0), 1) * 60 / 4, nrhs=nr)
    del fin, fout
    nb, block = 32, (4, 4, 4, 4)
    g64 = field(nb * 2 * nh, torch.float64)
    basis = torch.empty_like(g64)
    half = nb // 2 * 2 * nh
    ops.dwf_chiral_project(ctx, basis[:half], g64[:half], 1, nb // 2)
    ops.dwf_chiral_project(ctx, basis[half:], g64[half:], -1, nb // 2)
    work = basis.clone()

    def ortho():
        work.copy_(basis)
        ops.block_orthonormalise(ctx, work, nb, nb // 2, block)
    ms = timed(ortho, 3)
    copy_ms = timed(lambda: work.copy_(basis), 3)
    nfull_c = nh  # complex numbers of one full field (= reals of one half field)
    emit("a9", "block_orthonormalise FP64, 32 vectors, 4^4 x Ls blocks", ms - copy_ms,
         2 * 1.5 * 8.0 * nb * nb * nfull_c, "TFLOP/s", fp64_peak, "fp64 alu (measured FMA rate)",
         note="work = Cholesky-QR2: two passes of a Gram matrix (nb^2 complex multiply-adds per field"
              " entry) and the R^-1 update of each chirality group (2 (nb/2)^2), 8 flop per complex"
              " multiply-add, all in FP64 as the orthonormalisation requires")
    del g64, basis
    Cc = [None]

    work32 = work.float()  # the multigrid setup builds from the FP32 copy of the basis
    del work

    def build():
        if Cc[0] is not None:
            Cc[0].close()
        Cc[0] = ops.coarse_build(ctx, work32, nb, nb // 2, block, mf)
    ms = timed(build, 3)
    emit("a10", "coarse_build (9-point H_DW stencil), nb 32, 4^4 x Ls blocks, FP32 basis", ms, None,
         note="face hops of the 32 basis fields and block inner products, as in mg_setup")
    del work32
    coarse = Cc[0]
    r = field(2 * coarse.nc * nb, torch.float32)
    e = torch.zeros_like(r)
    its = []

    def csolve():
        its.append(ops.coarse_solve(coarse, e, r, 1e-4, 5000))
    ms = timed(csolve, 5)
    emit("a12", "coarse_solve (persistent coarse CG on A^2), Gaussian right-hand side, to 1e-4", ms, None,
         iterations=its[-1], us_per_iteration=1e3 * ms / max(its[-1], 1))
    coarse.close()
    for pn in ("tf32", "f32"):
        res = coarse_apply_measure(ctx, w, pn, 3, 10)
        emit("a11", f"coarse_apply {pn.upper()}, nb 32, 32 RHS, 512 coarse sites", res["ms_median"],
             res["flop_per_launch"], "TFLOP/s",
             res.get("tf32_peak_tflops") if pn == "tf32" else None, "tensor (TF32)" if pn == "tf32" else "fp32",
             GBs_algorithmic=res["GBs_algorithmic"], frac_of_hbm=res["frac_of_hbm"])
    lmax = ops.dwf_power_max(ctx, v0, mf, 100, F32) * 1.1
    prm = ops.mg_params(block, nb, mf, subspace_mode=SUBSPACE_BATCH, lambda_lo=0.05, lambda_max=lmax,
                        filter_order=60, smooth=(0.05, lmax, 32), coarse_tol=0.02)
    eta = field(nb * 2 * nh, torch.float64)
    G = ops.MG(ctx, prm, eta)
    del eta
    f = lambda: ops.mg_smooth(G, fo32, full32)
    emit("a13", "mg_smooth S_cheb([0.05, lmax], 32), F32 full field", timed(f, 3), hop_bytes(f), "GB/s", hbm,
         "hbm", note="achieved counts the hopping launches' algorithmic bytes only (the Chebyshev updates add"
                     " six field passes per order)")
    G.close()
    npf = 4
    X = field(npf * nh, torch.float32)
    force = torch.zeros(int(np.prod(L)) * 4 * 9 * 2, dtype=torch.float64, device="cuda")
    f = lambda: ops.dwf_force(ctx, force, X, [0.01, 0.05, 0.2, 1.0])
    fbytes = npf * 4 * nh * 4.0 + 2 * ctx.Vh * 72 * 8 * 2 + force.numel() * 8 * 2
    emit("a15", "dwf_force, 4 pseudofermions, FP32 fields", timed(f, 3), fbytes, "GB/s", hbm, "hbm",
         note="work = X, Y, X', Y' half fields per pseudofermion + links + force read and write; the hops"
              " forming Y, X', Y' are inside the call")
    print(json.dumps({"rows_measured": len(rows), "peak_source": kind}), flush=True)
    ctx.close()


def run_vcycle(args):
    """Profile modes `--kernel mg_vcycle` (HDCR, MG_PARAMS, or MG_PARAMS_LARGE
    above 2^24 4D sites) and `--kernel hybrid_vcycle` (Algorithm F,
    HYBRID_PARAMS): the setup on the workload, one warm-up V-cycle, then one
    V-cycle inside the NVTX range "vcycle" (for `ncu --nvtx --nvtx-include
    vcycle/`); prints the setup and V-cycle host-clock times."""
    import torch

    from paper_2103_05034_gb300 import ops
    from paper_2103_05034_gb300._lib import COARSE_CG, COARSE_DEFLATED, COARSE_RB, F32, SUBSPACE_RECURSIVE

    w, U, b = build_workload(args.workload, 0)
    L, Ls, mf = w["L"], w["Ls"], w["mf"]
    ctx = ops.Context(L, Ls, w["M5"], U)
    del U
    ops.dwf_autotune(ctx, F32, 10)
    gen = torch.Generator(device="cuda").manual_seed(77)
    v0 = torch.randn(2 * ctx.half_numel(), generator=gen, device="cuda", dtype=torch.float64)
    lmax = ops.dwf_power_max(ctx, v0, mf, 100, F32) * 1.10
    del v0
    cs_of = {"cg": COARSE_CG, "rb": COARSE_RB, "deflated": COARSE_DEFLATED}
    gen = torch.Generator(device="cuda").manual_seed(synth.SEED_BASIS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.kernel == "hybrid_vcycle":
        p = dict(HYBRID_PARAMS)
        prm = ops.mg_params(p["block"], 0, mf, smooth=(p["smooth"][0], lmax, p["smooth"][2]),
                            coarse_tol=p["coarse_tol"], coarse_maxiter=p["coarse_maxiter"], nkrylov=p["nkrylov"],
                            maxiter=p["maxiter"], coarse_solver=cs_of[p["coarse_solver"]])
        hp = ops.hybrid_params(p["block"], p["nbasis4"], p["nbasis1"], mass4=p["mass4"], filter4=p["filter4"],
                               filter1=(p["filter1"][0], lmax, p["filter1"][2]),
                               smooth1=(p["smooth1"][0], lmax, p["smooth1"][2]), kcycle=p["kcycle"])
        nc1 = int(np.prod([L[m] // p["block"][m] for m in range(4)]))
        eta4 = torch.randn(2 * 2 * ctx.Vh * 12 * p["nbasis4"], generator=gen, device="cuda", dtype=torch.float64)
        eta1 = torch.randn(2 * nc1 * p["nbasis4"] * Ls * p["nbasis1"], generator=gen, device="cuda",
                           dtype=torch.float64)
        G = ops.HybridMG(ctx, prm, hp, eta4, eta1)
        del eta4, eta1
    else:
        p = dict(MG_PARAMS_LARGE if int(np.prod(L)) > (1 << 24) else MG_PARAMS)
        cs = cs_of[p["coarse_solver"]]
        prm = ops.mg_params(p["block"], p["nbasis"], mf, subspace_mode=SUBSPACE_RECURSIVE,
                            lambda_lo=p["lambda_lo"], lambda_max=lmax, filter_order=p["filter_order"],
                            delta=p["delta"], smooth=(p["smooth"][0], lmax, p["smooth"][2]),
                            coarse_tol=p["coarse_tol"], coarse_maxiter=p["coarse_maxiter"], nkrylov=p["nkrylov"],
                            maxiter=p["maxiter"], coarse_solver=cs,
                            deflation=p["deflation"] if cs == COARSE_DEFLATED else (0, 0, 0, 0.0))
        eta = torch.randn(2 * ctx.half_numel(), generator=gen, device="cuda", dtype=torch.float64)
        G = ops.MG(ctx, prm, eta)
        del eta
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    r = torch.randn(2 * ctx.half_numel(), generator=gen, device="cuda", dtype=torch.float32)
    out = torch.zeros_like(r)
    ops.mg_precondition(G, out, r)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    torch.cuda.nvtx.range_push("vcycle")
    ops.mg_precondition(G, out, r)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"kernel": args.kernel, "workload": args.workload, "setup_s": setup_s,
                      "vcycle_s": time.perf_counter() - t0}))
    G.close()
    ctx.close()
    return 0


def run_kernel(args):
    """Kernel-only loop for profiling: `--kernel dhop_f32|dhop_f64|dhop_f16|mpcdagmpc_f32|force_f32`
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
    if kind == "force":  # the force workload: four pseudofermions (X drawn on the device)
        gen = torch.Generator(device="cuda").manual_seed(synth.SEED_SOURCE)
        X = torch.randn(4 * ctx.half_numel(), generator=gen, device="cuda", dtype=torch.float32).to(inp.dtype)
        force = torch.zeros(int(np.prod(L)) * 4 * 9 * 2, dtype=torch.float64, device="cuda")
    fn = {"dhop": lambda: ops.dwf_dhop(ctx, out, inp, 0),
          "mpcdagmpc": lambda: ops.dwf_mpcdag_mpc(ctx, out, inp, w["mf"]),
          "force": lambda: ops.dwf_force(ctx, force, X, [0.01, 0.05, 0.2, 1.0])}[kind]
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
    ap.add_argument("--workload", default="dwf_48x48x48x96_ls24", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--step-iters", type=int, default=48,
                    help="CG iterations of one timed step (a block of the mixed-precision solve); 0: whole solve")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end (host buffer) measurement")
    ap.add_argument("--fp64-full", action="store_true",
                    help="run the whole FP64 red-black CG solve (minutes at 48^3) instead of projecting it")
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-mg-compare", dest="mg_compare", action="store_false",
                    help="skip the one-off FP64 RB-CG vs HDCR time-to-solution comparisons")
    ap.add_argument("--no-legs", dest="legs", action="store_false",
                    help="only the timed steps, the roofline kernel and e2e (for profiling the step)")
    ap.add_argument("--no-mg-large", dest="mg_large", action="store_false",
                    help="skip the 24^3x48x24 comparison (about two minutes)")
    ap.add_argument("--hybrid-large", action="store_true",
                    help="add Algorithm F (hybrid three-level multigrid) to the 24^3x48x24 comparison "
                         "(about four minutes)")
    ap.add_argument("--kernel", default=None,
                    help="profile mode: dhop_f32, dhop_f64, dhop_f16, mpcdagmpc_f32, force_f32 (dwf_force, four "
                         "pseudofermions), coarse_tf32 or coarse_f32 alone, "
                         "or mg_vcycle / hybrid_vcycle (one HDCR / Algorithm F V-cycle in an NVTX range)")
    ap.add_argument("--rows", action="store_true",
                    help="measure every step of the hot path alone (one JSON line per step)")
    ap.add_argument("--hop-variant", type=int, default=None,
                    help="with --kernel dhop_*: pin this hopping-kernel variant instead of autotuning")
    ap.add_argument("--sweep-variants", action="store_true",
                    help="with --kernel dhop_*: time every hopping-kernel tuning variant")
    args = ap.parse_args(argv)
    if args.rows:
        return run_rows(args)
    if args.kernel:
        if args.kernel.startswith("coarse_"):
            return run_coarse_kernel(args)
        if args.kernel in ("hybrid_vcycle", "mg_vcycle"):
            return run_vcycle(args)
        return run_kernel(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
