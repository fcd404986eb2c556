#!/usr/bin/env python
"""Benchmark of the QS^3 hot path on GB300.

Workload (default): the isotropic Heisenberg model on the periodic 10x10
square lattice, J = Jz = 1, N_down = 4, all 100 momentum sectors (total
dimension C(100,4) = 3,921,225), complex double (IEEE binary64).  One step is
the batched ground-state solve of all 100 sectors: the device-built basis is
reused, a seeded start vector is drawn on the device, and conventional
Lanczos with full reorthogonalisation runs every sector to its lowest
eigenvalue (Ritz value change <= 1e-14 and Ritz residual <= 1e-12 |E|) on the
binary64 engine, eigenvectors assembled in binary64.  The metric is H Phi
throughput over the whole step: structural non-zeros applied by all H Phi
launches of the step divided by the step time (Gnnz/s).

Also reported:
- roofline of the step's largest kernel (the Gram-Schmidt dot pass, exact
  integer dots on the digit images, HBM-bound) from CUDA events recorded
  inside the library on the solve's stream, against the measured HBM copy
  bandwidth, with H Phi's figures beside it;
- e2e: the same step through the C ABI from host buffers (basis built from
  host lattice arrays, eigenvectors copied back to host) per step;
- variants of the same solve: strict64 (every Gram-Schmidt update on binary64
  FMAs) and the double-float engine (48-bit significands on the fp32 units),
  each with its time and its largest |dE| against the binary64 step;
- the batched fp32-H Phi + binary64-refinement solve against plain binary64
  on the same workload (seconds and eigenvalue agreement);
- cpu_baseline: the oracle's H Phi (Alg. 9 as printed: every bond, every
  translation) timed on the host cores on a bounded sample of rows.

--impl reference times the oracle instead (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import qs3_inputs as qi  # noqa: E402

PEAKS_FALLBACK = {"hbm_gbs": 6800.0}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ncu figures of kernels of the solve (see the named summaries), as DRAM
# bytes (dram__bytes_read.sum + dram__bytes_write.sum) over the launch's
# algorithmic bytes; the ratio scales to the launches of a run (None: not
# captured since the kernel last changed).
GS_PROFILE = {"kernel": "k_dotb<complex> (exact fixed-point Gram-Schmidt dot products, digits through a "
                        "shared-memory ring filled by bulk copies)",
              # (540.7 MB read + 8.6 MB written) / 539.4 MB algorithmic, 20 sectors, 42 stored vectors
              "dram_over_alg": 1.0184,
              "profile": "profiles/k_dotb_square10x10_nd4_20k.md"}

WORKLOADS = {
    # name: (lattice factory, n_down, momenta)
    "square10x10_nd4_all_k": (lambda: qi.square(10), 4, lambda: qi.all_k((10, 10, 1))),
    "chain16_nd3_u1": (lambda: qi.chain(16), 3, lambda: None),
    # the bond-disordered open 32x32 square lattice, N_down = 3 (dim 178,433,024)
    "open32x32_nd3_u1": (lambda: qi.disordered_open_square(32), 3, lambda: None),
    # the 10x10x10 cube: N_down = 4 at k = 0 (dim 41,417,998) and N_down = 3 on the k-path
    "cubic10_nd4_k0": (lambda: qi.cubic(10), 4, lambda: [(0, 0, 0)]),
    "cubic10_nd3_kpath": (lambda: qi.cubic(10), 3, lambda: list(dict.fromkeys(qi.cubic_kpath(10)))),
    "cubic10_nd4_kpath": (lambda: qi.cubic(10), 4, lambda: list(dict.fromkeys(qi.cubic_kpath(10)))),
    # the paper's own OpenMP benchmark system: 6x6x6, N_down = 5, k = 0 (dim 17,313,563)
    # a smaller cube for profiling the stored-term kernel (~1 GB of terms)
    "cubic8_nd4_k0": (lambda: qi.cubic(8), 4, lambda: [(0, 0, 0)]),
    "cubic6_nd5_k0": (lambda: qi.cubic(6), 5, lambda: [(0, 0, 0)]),
}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200",
                 "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index: int = 0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9 or not f[0].isdigit() or int(f[0]) != gpu_index:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = max(mx, float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- our arm

def reduce_ranks(t_local: float, units: float, world: int, device):
    """Whole-job figures of a replicated run: the slowest rank's time and the
    units (non-zeros applied) of all ranks.  No data-path collective: each
    rank solves its own replica; only these two scalars are exchanged."""
    if world <= 1:
        return t_local, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([units], device=device, dtype=torch.float64)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def sector_subset(Ks, n):
    """The first n momenta of a workload (all of them for n <= 0 or a U(1) workload)."""
    if Ks is None or n <= 0:
        return Ks
    return list(Ks)[:n]


def run_ours(args, rank, world):
    import torch

    import paper_2107_00872_gb300 as qs3

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    mk, nd, ks = WORKLOADS[args.workload]
    spec = mk()
    Ks = sector_subset(ks(), args.sectors)
    basis = qs3.Basis(spec, nd, Ks)
    if args.dot_vectors64:
        basis.tuning(dot_vectors64=args.dot_vectors64)
    nnz_h = basis.nnz()
    stream = torch.cuda.current_stream()
    # the pipes' measured throughput: the fp64 FMA rate is the roof of the
    # binary64 dot products
    pipes = qs3.probe_peaks(stream=stream)
    # direct launches (no CUDA graphs) so every H Phi and dot-product launch
    # is timed for the roofline; the graphs leg below times graph replay
    opts = qs3.SolveOpts(use_graphs=False, n_max=args.n_max, min_iter=20, check_every=5, eps=1e-14, res_tol=1e-12,
                         precision="f64", seed=1 + rank)

    def step(seed):
        opts.seed = seed
        return basis.lanczos(opts, vectors=True, stream=stream)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for w in range(args.warmup):
        step(1000 + w)
    torch.cuda.synchronize()
    launches0 = qs3.load().qs3_kernel_launches()
    clk = ClockSampler()
    clk.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    evals = None
    for k in range(args.steps):
        evals, vec, info = step(1 + k + 17 * rank)
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop(dev.index or 0)
    ms_total = ev0.elapsed_time(ev1)
    launches = qs3.load().qs3_kernel_launches() - launches0
    nnz_steps = sum(i["hphi_nnz"] for i in infos)
    hphi_s = sum(i["hphi_seconds"] for i in infos)
    hphi_calls = sum(i["hphi_calls"] for i in infos)
    t_local = ms_total / 1e3
    t_max, nnz_all = reduce_ranks(t_local, float(nnz_steps), world, dev)
    value = nnz_all / t_max / 1e9

    # H Phi launches: per full launch (sectors drop out of the launches as
    # they converge, so figures scale by the average work per launch)
    peaks, peak_kind = load_peaks()
    hbm_peak = peaks.get("hbm_gbs")
    D = basis.total_dim
    s_phi = 16
    per_launch_nnz = nnz_steps / max(hphi_calls, 1)
    frac_work = per_launch_nnz / nnz_h
    t_launch = hphi_s / max(hphi_calls, 1)
    # algorithmic bytes of one full launch: diagonal read, one gather per term,
    # psi write, sigma row rank, one sigma probe per term
    B_alg = frac_work * (D * s_phi + (nnz_h - D) * s_phi + D * s_phi + D * 8 + (nnz_h - D) * 8)
    hphi = {"kernel": "k_hphi_o (complex128, products on the integer units, orbit-batched over the sectors)", "full_launch_ms": round(1e3 * t_launch / frac_work, 4),
            "avg_launch_ms": round(1e3 * t_launch, 4), "launch_gnnz_s": round(per_launch_nnz / t_launch / 1e9, 2),
            "alg_gbs": round(B_alg / t_launch / 1e9, 1), "hbm_frac_alg": round(B_alg / t_launch / 1e9 / hbm_peak, 4),
            "share_of_step": round(hphi_s / t_local, 3)}
    # the Gram-Schmidt dot pass (timed by the library around its launches)
    gs_s = sum(i["gs_dot_seconds"] for i in infos)
    gs_b = sum(i["gs_dot_bytes"] for i in infos)
    gs_calls = sum(i["gs_dot_calls"] for i in infos)
    ratio = GS_PROFILE["dram_over_alg"]
    ach = gs_b / gs_s / 1e9 if gs_s > 0 else 0.0
    roof = {"kernel": GS_PROFILE["kernel"], "bound": "hbm",
            "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(ach / hbm_peak, 4) if hbm_peak else None,
            "traffic": int(ratio * gs_b / gs_calls) if (ratio and gs_calls) else None,
            "traffic_source": GS_PROFILE["profile"],
            "alg_bytes_per_launch": int(gs_b / max(gs_calls, 1)),
            "launch_ms": round(1e3 * gs_s / max(gs_calls, 1), 4),
            "share_of_step": round(gs_s / t_local, 3), "hphi": hphi,
            "peak_source": (f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"),
            "fp64_pipe_bound_gbs": round(16.0 / 4.0 * pipes["fp64_fma_per_s"] / 1e9, 1)}

    out = {
        "metric": "H Phi Gnnz/s (batched Lanczos ground-state solve)",
        "value": round(value, 3),
        "unit": "Gnnz/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(1e3 * t_max / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": args.workload + (f"_first{args.sectors}k" if args.sectors > 0 else ""),
                   "lattice": spec.name, "n_sites": spec.n_sites, "n_down": nd,
                   "sectors": basis.n_sectors, "total_dim": D, "nnz_per_hphi": nnz_h,
                   "solver": "Lanczos (Alg. 10) with full reorthogonalisation every step on the binary64 engine: "
                             "Lanczos vectors stored as IEEE binary64 beside a fixed-point digit image; H Phi "
                             "with each term formed exactly on the integer units and each row rounded once; "
                             "alpha_x = Re psi_x^H w and the three-term update w -= beta psi_{x-1} + alpha psi_x "
                             "in binary64 FMAs; dot products summed exactly in 64-bit integers on 53-bit "
                             "fixed-point images of the operands (each rounded once, by at most 2^-53 of the "
                             "largest magnitude among its warp's 128 rows); the Gram-Schmidt update with "
                             "coefficients below 2^-40 |w| in sum forms its correction in fp32 from the top "
                             "digits (error below 2^-55 |w|)",
                   "l2": "working set > L2 (Krylov basis of ~100 vectors x 63 MB)",
                   "parallelism": f"replicas x{world} (independent sectors per GPU)"},
        "roofline": roof,
        "gpu_launches": int(launches),
        "tuning": basis.tuning(),
        "pipes": {k: v for k, v in pipes.items()},
        "clocks": clocks,
        "lowest_E": float(np.min(evals)),
        "_evals": evals[:, 0].tolist(),
        "lanczos_steps_per_solve": [int(i["iterations"]) for i in infos],
        "max_residual": max(i["max_residual"] for i in infos),
    }
    return out, basis, spec, nd, Ks


def variants_leg(args, basis, e_ref, ms_ref):
    """The same solve on the other arithmetic of the library: strict64 (every
    dot product and Gram-Schmidt update on binary64 FMAs) and the double-float engine (Krylov
    basis and the whole step in pairs of fp32, ~48-bit significands): seconds
    per solve, speed relative to the binary64 step and the largest |dE| / |E|
    against it."""
    import torch

    import paper_2107_00872_gb300 as qs3
    res = {}
    for name, kw in (("strict64", dict(precision="f64", strict64=True)), ("double_float", dict(precision="df"))):
        o = qs3.SolveOpts(use_graphs=False, n_max=args.n_max, min_iter=20, check_every=5, eps=1e-14, res_tol=1e-12,
                          seed=1, **kw)
        basis.lanczos(o, vectors=True)
        torch.cuda.synchronize()
        reps = 2
        t0 = time.perf_counter()
        for _ in range(reps):
            e, _, info = basis.lanczos(o, vectors=True)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / reps
        res[name] = {"seconds_per_solve": round(dt, 4), "speedup_vs_binary64_step": round(1e-3 * ms_ref / dt, 3),
                     "max_rel_dE_vs_binary64": float(np.max(np.abs(e[:, 0] - e_ref) / np.abs(e_ref))),
                     "steps": int(info["iterations"]), "gnnz_s": round(info["hphi_nnz"] / dt / 1e9, 3)}
    return res


def e2e_ours(args, spec, nd, Ks):
    """Same step through the public API from host buffers: basis built from
    the host lattice arrays (H2D), solve, eigenvectors and eigenvalues back to
    host (D2H), every step."""
    import torch

    import paper_2107_00872_gb300 as qs3
    stream = torch.cuda.current_stream()
    h2d = sum(np.asarray(a).nbytes for a in (spec.bi, spec.bj, spec.jxy, spec.jz)) + (12 * len(Ks) if Ks else 0)
    times = []
    nnz = 0
    d2h = 0
    for k in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B = qs3.Basis(spec, nd, Ks)
        ev, vec, info = B.lanczos(qs3.SolveOpts(use_graphs=False, n_max=args.n_max, eps=1e-14, res_tol=1e-12, seed=7 + k),
                                  vectors=True, stream=stream)
        host = vec.cpu().numpy()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        nnz += info["hphi_nnz"]
        d2h = host.nbytes + ev.nbytes
        B.close()
    t = float(np.sum(times))
    return {"value": round(nnz / t / 1e9, 3), "unit": "Gnnz/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "seconds_per_step": round(t / len(times), 4),
            "includes": "basis build from host arrays + solve + eigenvector D2H"}


def fp32_vs_fp64(args, basis, e_ref):
    """Batched fp32 H Phi + fp64 recurrences / binary64 refinement against
    plain binary64 (the IEEE engine),
    both run to |dE| <= 1e-9 |E| (Ritz value stable to 1e-10 relative); the
    achieved |dE| is measured against the tightly converged fp64 solve of the
    timed steps (Ritz residual <= 1e-12 |E|)."""
    import torch

    import paper_2107_00872_gb300 as qs3
    res = {"target": "|dE| <= 1e-9 |E| in every sector"}
    for prec in ("f64", "f32"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # same stopping rule for both: Ritz value stable to 1e-10 and Ritz
        # residual <= 1e-9 |E| (near-degenerate sectors need the residual well
        # below the gap); the fp32 run refines in fp64
        o = qs3.SolveOpts(n_max=args.n_max, eps=1e-10, res_tol=1e-9, precision=prec, refine_tol=1e-9, seed=3)
        e, _, info = basis.lanczos(o, vectors=False)
        torch.cuda.synchronize()
        res[prec] = {"seconds": round(time.perf_counter() - t0, 4), "steps": int(info["iterations"]),
                     "refine_steps": int(info["refine_iterations"]), "status": info["status"],
                     "max_rel_dE": float(np.max(np.abs(e[:, 0] - e_ref) / np.abs(e_ref)))}
    res["speedup_f32_over_f64"] = round(res["f64"]["seconds"] / res["f32"]["seconds"], 3)
    return res


def graphs_leg(args, basis):
    """fp64 Lanczos with every step after the first replayed as a CUDA graph,
    against direct launches: one solve of the workload, and the 16-site chain
    (N_down = 3, dim 560), where launch overhead dominates a step."""
    import torch

    import paper_2107_00872_gb300 as qs3
    res = {}
    for name, b, reps in (("workload", basis, 2), ("chain16_nd3_u1", qs3.Basis(qi.chain(16), 3, None), 20)):
        r = {}
        for g in (False, True):
            o = qs3.SolveOpts(use_graphs=g, n_max=args.n_max, min_iter=20, check_every=5, eps=1e-14, res_tol=1e-12,
                              precision="f64", seed=1)
            b.lanczos(o, vectors=False)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                _, _, info = b.lanczos(o, vectors=False)
            torch.cuda.synchronize()
            dt = (time.perf_counter() - t0) / reps
            r["graphs" if g else "direct"] = {"seconds_per_solve": round(dt, 5), "steps": int(info["iterations"]),
                                             "lanczos_steps_per_s": round(info["iterations"] / dt, 1)}
        r["speedup"] = round(r["direct"]["seconds_per_solve"] / r["graphs"]["seconds_per_solve"], 3)
        res[name] = r
    return res


# --------------------------------------------------------- oracle timing

def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm
    implementer and part codes), for the oracle baseline's record."""
    try:
        lines = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return platform.machine()
    for key in ("model name", "Model name", "Hardware"):
        for line in lines:
            if line.startswith(key) and ":" in line:
                return line.split(":", 1)[1].strip()
    codes = {}
    for line in lines:
        for key in ("CPU implementer", "CPU part"):
            if line.startswith(key) and key not in codes:
                codes[key] = line.split(":", 1)[1].strip()
    if codes:
        return f"{platform.machine()} implementer {codes.get('CPU implementer')} part {codes.get('CPU part')}"
    return platform.machine()


def oracle_sample(args, seconds_budget: float = 15.0, threads: int | None = None):
    """Oracle H Phi (Alg. 9 literally) on sampled rows of one sector of the
    workload; returns (Gnnz/s, cores, description)."""
    import oracle as orc
    mk, nd, ks = WORKLOADS[args.workload]
    spec = mk()
    Ks = ks()
    lat = orc.Lattice(**spec.as_dict())
    cores = orc.set_threads(threads or os.cpu_count() or 1)
    if Ks:
        K = Ks[1]
        sec = orc.mk_list(lat, nd, K)
        d = sec.dim
        x = qi.gaussian_start(5, d, True)
        rng = np.random.default_rng(0)
        n = 256
        done_rows, done_nnz, t_sum = 0, 0, 0.0
        while t_sum < seconds_budget and done_rows < d:
            rows = rng.integers(0, d, n)
            t0 = time.perf_counter()
            y, cnt = orc.hphi_k_rows(sec, x, rows, count=True)
            t_sum += time.perf_counter() - t0
            done_rows += n
            done_nnz += cnt
            n = min(n * 2, 1 << 16)
        desc = f"{done_rows} random rows of sector K={K} (dim {d}) of {spec.name}, N_down={nd}"
    else:
        D = math.comb(spec.n_sites, nd)
        x = qi.gaussian_start(5, D, False)
        rows = np.arange(D)
        t0 = time.perf_counter()
        y, cnt = orc.hphi_u1_rows(lat, nd, x, rows, count=True)
        t_sum = time.perf_counter() - t0
        done_nnz = cnt
        desc = f"all {D} rows of {spec.name}, N_down={nd}"
    return done_nnz / t_sum / 1e9, cores, desc


def run_reference(args, rank, world):
    if rank != 0:
        return None
    t_all = []
    rate_all = []
    cores = 1
    desc = ""
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        rate, cores, desc = oracle_sample(args, seconds_budget=4.0)
        if k >= args.warmup:
            t_all.append(time.perf_counter() - t0)
            rate_all.append(rate)
    value = float(np.mean(rate_all))
    return {"impl": "reference", "metric": "H Phi Gnnz/s (batched Lanczos ground-state solve)",
            "value": round(value, 6), "unit": "Gnnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(t_all)), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "cpu_baseline": {"value": round(value, 6), "unit": "Gnnz/s", "cores": cores, "kind": "oracle",
                             "sample": desc, "cpu": cpu_model()},
            "e2e": {"value": round(value, 6), "unit": "Gnnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_hphi_only(args):
    """H Phi launches alone on the workload's basis (kernel-level numbers and
    the small-footprint case for profiling): W warm-up and K timed launches
    of psi = H phi over all sectors, CUDA events on the launching stream."""
    import torch

    import paper_2107_00872_gb300 as qs3
    mk, nd, ks = WORKLOADS[args.workload]
    spec = mk()
    Ks = ks()
    B = qs3.Basis(spec, nd, Ks)
    t_store = None
    if args.stored:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B.store_terms(1)
        torch.cuda.synchronize()
        t_store = time.perf_counter() - t0
    dfm = args.dtype == "c128df"
    dt = {"c128": torch.complex128, "c128df": torch.complex128, "c64": torch.complex64, "f64": torch.float64,
          "f32": torch.float32}[args.dtype]
    if Ks and not dt.is_complex:
        raise SystemExit("k-sectors need complex vectors")
    g = torch.Generator(device="cuda").manual_seed(0)
    phi = torch.randn(B.total_dim, dtype=dt, device="cuda", generator=g)
    psi = torch.empty_like(phi)
    st = torch.cuda.current_stream()
    if dfm:
        # double-float input (re.hi, re.lo, im.hi, im.lo): 16 B per element like complex128
        phi = qs3.split_df(phi, stream=st)

    def apply():
        if dfm:
            B.hphi_df(phi, psi, st)
        else:
            B.hphi(phi, psi, st)
    for _ in range(args.warmup):
        apply()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        apply()
    e1.record(st)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    nnz = B.nnz()
    s = psi.element_size()
    D = B.total_dim
    b_alg = D * s + (nnz - D) * s + D * s + (D * 8 + (nnz - D) * 8 if Ks else 0)
    if args.stored:
        # per term: target row + code (8 B) and one gather; per row: x0, psi, diagonal, row pointer
        b_alg = D * s + (nnz - D) * s + D * s + (nnz - D) * 8 + D * 16
    peaks, kind = load_peaks()
    return {"mode": "hphi", "workload": args.workload, "dtype": args.dtype, "stored_terms": bool(args.stored),
            "store_seconds": None if t_store is None else round(t_store, 3), "total_dim": D, "nnz": nnz,
            "ms_per_launch": round(1e3 * t, 4), "gnnz_s": round(nnz / t / 1e9, 3),
            "alg_bytes_per_launch": int(b_alg), "alg_gbs": round(b_alg / t / 1e9, 1),
            "hbm_frac": round(b_alg / t / 1e9 / peaks["hbm_gbs"], 4), "peak_source": kind}


def run_trl(args):
    """Thick-restart Lanczos (Alg. 10) on the 10x10x10 cube's k-path: N_down =
    3 (28 distinct sectors, 4,652,676 rows, all at once) or, with --workload
    cubic10_nd4_kpath, N_down = 4 (41.4 M rows per sector; the first
    --sectors distinct path momenta, --group at a time, stored-term H Phi with
    --stored).  The 4 lowest eigenpairs of every sector with N_K = 8 kept and
    N_M = 32 Lanczos vectors, plain binary64 against fp32 H Phi with fp64
    recurrences and binary64 refinement; binary64 residuals of both."""
    import torch

    import paper_2107_00872_gb300 as qs3
    wl = args.workload if args.workload in ("cubic10_nd3_kpath", "cubic10_nd4_kpath") else "cubic10_nd3_kpath"
    mk, nd, ks = WORKLOADS[wl]
    spec = mk()
    Ks = sector_subset(ks(), args.sectors)
    group = len(Ks) if nd == 3 else max(1, args.group)
    out = {"mode": "trl", "workload": wl + (f"_first{len(Ks)}k" if args.sectors > 0 else ""), "sectors": len(Ks),
           "n_eig": 4, "n_keep": 8, "n_max": 32, "stored_terms": bool(args.stored), "group": group,
           "total_dim": 0, "basis_build_s": 0.0}
    res = {"f64": {"seconds": 0.0, "steps": 0, "restarts": 0, "refine_steps": 0, "max_residual": 0.0, "nnz": 0,
                   "status": []},
           "f32": {"seconds": 0.0, "steps": 0, "restarts": 0, "refine_steps": 0, "max_residual": 0.0, "nnz": 0,
                   "status": []}}
    e_all = {"f64": [], "f32": []}
    max_rel = 0.0
    for g0 in range(0, len(Ks), group):
        t0 = time.perf_counter()
        basis = qs3.Basis(spec, nd, Ks[g0:g0 + group])
        if args.stored:
            basis.store_terms(1)
        basis.nnz()
        torch.cuda.synchronize()
        out["basis_build_s"] += time.perf_counter() - t0
        out["total_dim"] += basis.total_dim
        for prec in ("f64", "f32"):
            # convergence: the paper's criterion over the N_K kept values, at 1e-10
            o = qs3.SolveOpts(n_eig=4, n_keep=8, n_max=32, max_iter=4000, eps=1e-10, precision=prec,
                              refine_tol=1e-9, seed=11)
            if g0 == 0 and nd == 3:
                basis.trlanczos(o, vectors=False)          # warm-up (tuning, module load)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e, _, info = basis.trlanczos(o, vectors=False)
            torch.cuda.synchronize()
            r = res[prec]
            r["seconds"] += time.perf_counter() - t0
            r["steps"] += int(info["iterations"])
            r["restarts"] += int(info["restarts"])
            r["refine_steps"] += int(info["refine_iterations"])
            r["max_residual"] = max(r["max_residual"], info["max_residual"])
            r["nnz"] += info["hphi_nnz"]
            r["status"].append(info["status"])
            e_all[prec].append(e)
        # lowest eigenvalue per sector; the other kept values may pick up a
        # different copy of a degenerate level from another start
        a, b = e_all["f64"][-1], e_all["f32"][-1]
        max_rel = max(max_rel, float(np.max(np.abs(b[:, 0] - a[:, 0]) / np.abs(a[:, 0]))))
        del basis
        torch.cuda.empty_cache()
    for prec in ("f64", "f32"):
        r = res[prec]
        r["seconds"] = round(r["seconds"], 4)
        r["gnnz_s"] = round(r.pop("nnz") / r["seconds"] / 1e9, 3)
        r["ms_per_restart"] = round(1e3 * r["seconds"] / max(1, r["restarts"]), 3)
        r["status"] = sorted(set(r["status"]))
        out[prec] = r
    e64 = np.concatenate(e_all["f64"])
    out["lowest_E"] = float(np.min(e64))
    out["lowest_E_per_sector"] = [float(v) for v in e64[:, 0]]
    out["f32"]["max_rel_dE_lowest_vs_f64"] = max_rel
    out["basis_build_s"] = round(out["basis_build_s"], 3)
    out["speedup_f32_over_f64"] = round(out["f64"]["seconds"] / out["f32"]["seconds"], 3)
    return out


def run_dsf(args):
    """Dynamical structure factor of the 10x10 square lattice (Eq. (cfe)):
    the N_down = 4 ground state (lowest over the 100 momenta), S^-_q of it for
    all 100 q into the N_down = 5 sectors at k0 + q (752,875 rows each), 200
    Lanczos steps with full reorthogonalisation per q, and the continued
    fraction on omega = 0:0.005:8 with eta = 0.05 and h = 4.  The q values are
    taken in groups so the Krylov store stays within device memory.  --op sz
    or splus computes S^z (same N_down, trivial q = 0 peak subtracted) or S^+
    (N_down - 1) instead."""
    import torch

    import paper_2107_00872_gb300 as qs3
    L, nd = 10, 4
    spec = qi.square(L)
    Ks = qi.all_k((L, L, 1))
    src = qs3.Basis(spec, nd, Ks)
    ev, vec, info = src.lanczos(qs3.SolveOpts(n_max=args.n_max, eps=1e-14, res_tol=1e-12, seed=1), vectors=True)
    s0 = int(np.argmin(ev[:, 0]))
    E0 = float(ev[s0, 0])
    k0 = Ks[s0]
    gs = vec[src.offsets[s0]:src.offsets[s0 + 1]].clone()
    src1 = qs3.Basis(spec, nd, [k0])
    omega = np.arange(0.0, 8.0 + 1e-9, 0.005)
    group = max(1, args.q_group)
    n_iter, eta, h = 200, 0.05, 4.0
    op = {"sminus": 2, "splus": 1, "sz": 3}[args.op]
    dn = {2: 1, 1: -1, 3: 0}[op]
    t_total = 0.0
    rows = 0
    peaks = []
    sq = []
    for g0 in range(0, len(Ks), group):
        Qs = Ks[g0:g0 + group]
        K2 = [tuple((k0[a] + Q[a]) % (L if a < 2 else 1) for a in range(3)) for Q in Qs]
        dst = qs3.Basis(spec, nd + dn, K2)
        rows += dst.total_dim
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S, al, be, n2 = qs3.dsf(src1, 0, gs, E0, dst, Qs, n_iter, eta, h, omega, op=op, subtract_trivial=(op == 3))
        torch.cuda.synchronize()
        t_total += time.perf_counter() - t0
        peaks += [float(np.max(S[i])) for i in range(len(Qs))]
        sq += [float(v) for v in n2]
        del dst
    return {"mode": "dsf", "operator": args.op, "workload": f"square10x10_nd4_to_nd{nd + dn}_all_q", "E0": E0,
            "k0": list(k0), "q_points": len(Ks),
            "rows_all_q": rows, "cf_steps": n_iter, "omega_points": len(omega), "eta": eta, "h": h,
            "q_group": group, "seconds": round(t_total, 3), "seconds_per_q": round(t_total / len(Ks), 4),
            "lanczos_steps_per_s": round(len(Ks) * n_iter / t_total, 1),
            "max_peak": max(peaks), "sum_norm2": sum(sq),
            "sum_rule": {"sminus": "N - N_down = 96", "splus": "N_down = 4", "sz": "N/4 = 25"}[args.op]}


def run_ground(args):
    """Ground state of a U(1) workload (default: the bond-disordered open 32x32
    square lattice, N_down = 3, dimension 178,433,024) by thick-restart
    Lanczos (Alg. 10), once with fp32 H Phi + fp64 recurrences + binary64
    refinement and once in plain binary64, then the local magnetisation
    <s^z_i> at every site from the refined state (Sec. "Calculating
    expectation values").  Reports both energies, their |dE| / |E|, the
    binary64 residual |H v - E v| of each, the times, and sum_i <s^z_i>
    against N/2 - N_down."""
    import torch

    import paper_2107_00872_gb300 as qs3
    mk, nd, ks = WORKLOADS[args.workload]
    spec = mk()
    if ks() is not None:
        raise SystemExit("--mode ground takes a U(1) workload")
    t0 = time.perf_counter()
    basis = qs3.Basis(spec, nd)
    nnz = basis.nnz()
    t_build = time.perf_counter() - t0
    out = {"mode": "ground", "workload": args.workload, "total_dim": basis.total_dim, "nnz_per_hphi": nnz,
           "basis_build_s": round(t_build, 3), "n_keep": args.n_keep, "n_max": args.trl_max}
    vec32 = None
    precs = ("f32", "f64") if args.prec == "both" else (args.prec,)
    for prec in precs:
        o = qs3.SolveOpts(n_eig=1, n_keep=args.n_keep, n_max=args.trl_max, max_iter=20000, eps=1e-12,
                          precision=prec, refine_tol=1e-10, seed=7)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e, v, info = basis.trlanczos(o, vectors=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[prec] = {"E": float(e[0, 0]), "seconds": round(dt, 3), "status": info["status"],
                     "steps": int(info["iterations"]), "restarts": int(info["restarts"]),
                     "refine_steps": int(info["refine_iterations"]), "residual": info["max_residual"],
                     "residual_over_E": info["max_residual"] / abs(float(e[0, 0])),
                     "gnnz_s_over_solve": round(info["hphi_nnz"] / dt / 1e9, 2)}
        if prec == "f32" or len(precs) == 1:
            vec32 = v
        else:
            del v
        torch.cuda.empty_cache()
    if len(precs) == 2:
        out["rel_dE_f32_vs_f64"] = abs(out["f32"]["E"] - out["f64"]["E"]) / abs(out["f64"]["E"])
        out["speedup_f32_over_f64"] = round(out["f64"]["seconds"] / out["f32"]["seconds"], 3)
    t0 = time.perf_counter()
    c = basis.correlations(vec32, local=True)
    torch.cuda.synchronize()
    sz = np.asarray(c["sz"])
    out["sz_local"] = {"seconds": round(time.perf_counter() - t0, 4), "sum": float(sz.sum()),
                       "expected_sum": spec.n_sites / 2 - nd, "min": float(sz.min()), "max": float(sz.max()),
                       "argmin": int(np.argmin(sz))}
    if args.dump:
        np.save(args.dump, sz)
    return out


def run_batch(args):
    """The uneven instance mix: 64 seeded XXZ instances (chains, squares,
    cubes; half with a random momentum) solved to their lowest eigenvalue in
    one batched call, fp32 H Phi with fp64 recurrences and fp64 refinement,
    against the same 64 solved one by one in plain fp64."""
    import torch

    import paper_2107_00872_gb300 as qs3
    mix = qi.instance_mix(args.n_instances)
    t0 = time.perf_counter()
    bases = [qs3.Basis(x["lattice"], x["n_down"], None if x["K"] is None else [x["K"]]) for x in mix]
    for b in bases:
        b.nnz()
    t_basis = time.perf_counter() - t0
    dims = [b.total_dim for b in bases]
    o32 = qs3.SolveOpts(n_max=args.n_max, eps=1e-10, res_tol=1e-9, precision="f32", refine_tol=1e-9, seed=5)
    o64 = qs3.SolveOpts(n_max=args.n_max, eps=1e-10, res_tol=1e-9, precision="f64", seed=5)
    qs3.batch_solve(bases[:4], o32)            # warm-up (kernel attributes, allocator)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev, infos, status = qs3.batch_solve(bases, o32, max_concurrent=args.concurrency)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    ev1 = []
    for b in bases:
        e, _, _ = b.lanczos(o64, vectors=False)
        ev1.append(e[:, 0])
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    dE = max(float(np.max(np.abs(a - c) / np.abs(c))) for a, c in zip(ev, ev1))
    nnz = sum(i["hphi_nnz"] for i in infos)
    return {"mode": "batch", "workload": f"instance_mix{len(mix)}", "instances": len(mix),
            "dim_min": int(min(dims)), "dim_max": int(max(dims)), "dim_sum": int(sum(dims)),
            "with_momentum": sum(1 for x in mix if x["K"] is not None), "basis_build_s": round(t_basis, 3),
            "batch_fp32_refined_s": round(t_batch, 3), "one_by_one_fp64_s": round(t_one, 3),
            "speedup": round(t_one / t_batch, 3), "max_rel_dE_batch_vs_fp64": dE, "status": status,
            "batch_hphi_gnnz_s": round(nnz / t_batch / 1e9, 3), "concurrency": args.concurrency,
            "target": "|dE| <= 1e-9 |E|: Ritz value stable to 1e-10, residual <= 1e-9 |E|"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="solve", choices=["solve", "hphi", "batch", "trl", "dsf", "ground"])
    ap.add_argument("--n-keep", dest="n_keep", type=int, default=8, help="--mode ground: N_K")
    ap.add_argument("--trl-max", dest="trl_max", type=int, default=48, help="--mode ground: N_M")
    ap.add_argument("--dump", default="", help="--mode ground: save <s^z_i> to this .npy file")
    ap.add_argument("--prec", default="both", choices=["both", "f32", "f64"], help="--mode ground: arithmetic")
    ap.add_argument("--q-group", dest="q_group", type=int, default=25, help="--mode dsf: q values per call")
    ap.add_argument("--group", type=int, default=2, help="--mode trl, N_down = 4: sectors per basis")
    ap.add_argument("--op", default="sminus", choices=["sminus", "splus", "sz"], help="--mode dsf: S^alpha_q")
    ap.add_argument("--stored", action="store_true", help="--mode hphi: stored-term H Phi (k-sectors)")
    ap.add_argument("--n-instances", dest="n_instances", type=int, default=64, help="--mode batch")
    ap.add_argument("--concurrency", type=int, default=16, help="--mode batch")
    ap.add_argument("--dtype", default="c128", choices=["c128", "c128df", "c64", "f64", "f32"], help="--mode hphi only")
    ap.add_argument("--workload", default="square10x10_nd4_all_k", choices=sorted(WORKLOADS))
    ap.add_argument("--n-max", dest="n_max", type=int, default=250)
    ap.add_argument("--dot-vectors64", dest="dot_vectors64", type=int, default=0,
                    help="impose the binary64 dot pass (1, 2, 4: k_dotx vectors per pass; 8: the copy rings); 0 tunes")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / fp32 / cpu_baseline legs")
    ap.add_argument("--sectors", type=int, default=0,
                    help="solve only the first N momentum sectors (a small case for profiling; 0 = all)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.mode == "hphi":
        print(json.dumps(run_hphi_only(args)), flush=True)
        return
    if args.mode == "batch":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.mode == "trl":
        print(json.dumps(run_trl(args)), flush=True)
        return
    if args.mode == "dsf":
        print(json.dumps(run_dsf(args)), flush=True)
        return
    if args.mode == "ground":
        if args.workload == "square10x10_nd4_all_k":
            args.workload = "open32x32_nd3_u1"
        print(json.dumps(run_ground(args)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out, basis, spec, nd, Ks = run_ours(args, rank, world)
    if rank == 0 and not args.no_extras:
        out["e2e"] = e2e_ours(args, spec, nd, Ks)
        out["fp32_vs_fp64"] = fp32_vs_fp64(args, basis, np.array(out["_evals"]))
        out["variants"] = variants_leg(args, basis, np.array(out["_evals"]), out["ms_per_step"])
        out["graphs"] = graphs_leg(args, basis)
        rate, cores, desc = oracle_sample(args)
        rate1, _, desc1 = oracle_sample(args, seconds_budget=5.0, threads=1)
        out["cpu_baseline"] = {"value": round(rate, 6), "unit": "Gnnz/s", "cores": cores, "kind": "oracle",
                               "sample": desc, "cpu": cpu_model(),
                               "one_thread": {"value": round(rate1, 6), "sample": desc1}}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    out.pop("_evals", None)
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
