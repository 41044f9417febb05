#!/usr/bin/env python
"""Benchmark of the GB300 Galerkin integral-equation solver.

Workload (default): the single-solve configuration, Nx = Ny = 128, Nz = 32 cells of
50 m (1,572,864 unknowns), 5-layer seeded background, 20 seeded anomalies of
0.01-0.1 ohm-m, 1 Hz, both MT polarisations; coefficients generated on the
device by the library.  One step = one mixed-precision solve of both polarisations
to ||b - A u|| <= 1e-7 ||b|| in the IE_MIXED_FP64K mode: iterative refinement whose
residual is the c128 product with the FP64 contraction, and whose corrections come
from GMRES on the c64 product (FP32 FFTs and contraction) with FP64 Krylov vectors
and Givens rotations (Gram-Schmidt on the FP64 vectors in double-float arithmetic)
-- every step of the hot path.

Printed (one JSON line, rank 0):
  value         unknowns * Krylov iterations / s over the timed steps (device-resident
                inputs), summed over ranks (replicas) / max time
  matvec        the IE matrix-vector product: algorithmic GB/s (coefficients once +
                input and output vectors) of the c64 product for both polarisations
  tts           time-to-solution at 1e-7 (median and spread of repeated solves): the
                timed mode, the c64-Krylov mode IE_MIXED and the plain FP64 solve
  roofline      the contraction kernel, timed with CUDA events during the timed steps
  err_vs_oracle residual of GPU solutions under the oracle's FFT product on a proxy
                operator of the same size (cpu_baseline leg)
  cpu_baseline  the FP64 oracle (numpy) on the host: GMRES iterations of the same grid,
                one thread and all threads
  e2e           the same metric through the C ABI with host buffers (H2D of the
                right-hand sides and D2H of the solution inside the timed region)
  c3_batch      the batched configuration (16 frequencies x 2 polarisations over four
                grids) in the timed precision: batched and one-at-a-time solved
                instances/s, and batched plain FP64 (--skip-c3 leaves it out)

--impl reference runs the oracle (the reference implementation of this tier) on the
host cores for the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time


def _pin_threads_early():
    """Thread caps of numpy's BLAS / OpenMP, set before numpy is imported: --threads T
    for a CPU sample, all host cores for the reference arm."""
    n = None
    if "--cpu-sample" in sys.argv and "--threads" in sys.argv:
        n = sys.argv[sys.argv.index("--threads") + 1]
    elif "--impl" in sys.argv and sys.argv[sys.argv.index("--impl") + 1] == "reference":
        n = str(os.cpu_count() or 1)
    if n is not None:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                  "NUMEXPR_NUM_THREADS"):
            os.environ[v] = n


_pin_threads_early()

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "IE matvec GB/s & unknowns*iters/s; GMRES time-to-solution at 1e-7, mixed vs FP64"
PRECISIONS_BY_NAME = {"fp64": 0, "mixed": 1, "fp64k": 2}  # ie.IE_FP64, IE_MIXED, IE_MIXED_FP64K
UNIT = "unknowns*iters/s"
TOL = 1e-7


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), float(d.get("sm_max_mhz", 2070.0)), "measured"
    return 6800.0, 2070.0, "fallback"


# (workload, contraction variant, right-hand sides) -> DRAM bytes per contraction launch
CONTRACT_TRAFFIC = {("C2", 3, 2): 654541312 + 86889728, ("C2", 5, 2): 654550784 + 88402176,
                    ("C2", 7, 2): 654666752 + 42406656}
VARIANT_NAMES = ["tma 1 slot", "tma 3 slots", "panel", "tma 1 slot, 1 row/thread",
                 "3xTF32 mma.sync, producer warp, 2 slots", "3xTF32 mma.sync, 1 slot, unpacked",
                 "3xTF32 tcgen05.mma, block in TMEM, warp-specialised",
                 "2xFP16 (scaled) tcgen05.mma kind::f16, block in TMEM, warp-specialised",
                 "3xTF32 mma.sync, one Nz x Nz matrix per sub-step"]
TENSOR_VARIANTS = (4, 5, 6, 7, 8)


def bf16_peak():
    """(dense bf16 TFLOP/s burst, source) from the measured peaks, else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        if "bf16_tflops" in d:
            return float(d["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def workload_desc(name, model):
    """The workload as the bench line names it (the same string on both arms)."""
    g = model.grid
    return (f"{name}: {g.nx}x{g.ny}x{g.nz} cells, {len(model.layers.sigma) - 1} layers + air, "
            f"{model.freqs[0]} Hz, 2 polarisations, tol {TOL}")


def workload(name):
    return {"C1": W.config1, "C2": W.config2, "C4": W.config4, "C5": W.config5}[name]()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: each rank solves its own copy)
# ---------------------------------------------------------------------------

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group(backend=backend)
    return rank, ws


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the oracle on the host (cpu baseline and the reference arm)
# ---------------------------------------------------------------------------

class OracleSample:
    """FP64 oracle GMRES iterations on the workload's grid for one right-hand side.

    The coefficient values do not change the oracle's cost, so a seeded random tensor
    of the workload's shape stands in for the generated one.  The spectral blocks are
    built once (setup, untimed).  run(n) times one restart cycle of n iterations (the
    oracle's GMRES with restart n, so that its Krylov array holds n + 1 vectors) and
    subtracts the one product that computes the cycle's initial residual, timed on its
    own: the result is the cost of n iterations, each one product and one CGS2 step."""

    def __init__(self, model, seed=41):
        from oracle import operator as O
        self.O = O
        self.model = model
        g = model.grid
        q = W.random_compressed_q(g.ny, g.nx, g.nz, seed=seed)
        self.qt = O.full_spectrum_blocks(O.embed_spectrum(q))
        del q
        self.b = W.random_field((3, g.nz, g.ny, g.nx), seed + 1)

    def apply(self, v):
        return self.O.fft_apply(self.model, self.qt, v)

    def run(self, n_iters):
        O = self.O
        t0 = time.perf_counter()
        self.apply(self.b)
        t_apply = time.perf_counter() - t0
        t0 = time.perf_counter()
        O.gmres(self.apply, self.b, tol=1e-30, m=n_iters, max_iter=n_iters)
        return max(time.perf_counter() - t0 - t_apply, 1e-9), n_iters


def run_cpu_sample(args):
    """Child process of the CPU baseline: thread caps already set from --threads before
    numpy was imported; prints one JSON line."""
    model = workload(args.workload)
    sample = OracleSample(model)
    t, n = sample.run(args.iters)
    print(json.dumps({"threads": int(args.threads), "seconds": t, "iters": n}), flush=True)


def cpu_leg(workload_name, threads, iters):
    """Run OracleSample in a child process with `threads` BLAS/OpenMP threads."""
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--threads", str(threads), "--iters",
           str(iters), "--workload", workload_name]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"CPU sample failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args, rank, ws):
    if rank != 0:
        return
    model = workload(args.workload)
    g = model.grid
    n_unk = 3 * g.nx * g.ny * g.nz
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", "1"))
    sample = OracleSample(model)
    for _ in range(args.warmup):
        sample.run(1)
    t, it = 0.0, 0
    for _ in range(args.steps):
        dt, n = sample.run(1)
        t += dt
        it += n
    value = n_unk * it / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": workload_desc(args.workload, model), "unknowns": n_unk,
                                            "grid": [g.nx, g.ny, g.nz]},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": threads,
                             "sample": "one FP64 GMRES iteration (FFT product + CGS2) of the oracle per step, one "
                                       "right-hand side; the cycle's initial-residual product timed apart and "
                                       f"subtracted; BLAS/OpenMP threads capped at {threads} (numpy's FFT and "
                                       "einsum run on one thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_check(model, args):
    """The cpu_baseline leg's accuracy check: GPU solutions of a proxy operator of the
    workload's size (its grid, layers and anomaly layout at a moderate contrast, a
    seeded random coefficient tensor scaled to make GMRES converge), in the timed
    mode and in IE_MIXED, and their residuals under the oracle's FFT product."""
    import torch
    from oracle import normal
    from oracle.proxy import contracting_q, moderate_contrast, oracle_residual
    from paper_1512_06126_gb300 import ie
    t0 = time.perf_counter()
    mp = moderate_contrast(model)
    q, qt = contracting_q(mp, seed=62, target=8.0)
    g = mp.grid
    b = np.stack([normal.rhs_U0(mp, mp.freqs[0], "x"), normal.rhs_U0(mp, mp.freqs[0], "y")])
    ctx = ie.Context(g, mp.layers, mp.sigma_a, mp.freqs[:1], [q], max_rhs=2, restart=args.restart,
                     inner_tol=args.inner_tol)
    del q
    bd = torch.from_numpy(b).to("cuda")
    out = {"operator": "proxy: the workload's grid, layers and anomaly layout at 3x contrast, seeded random "
                       "coefficient tensor scaled (oracle/proxy.py); residual ||b - A u|| / ||b|| of the GPU "
                       "solution (tol 1e-7) under the oracle's FFT product, max over both polarisations"}
    for name, prec in (("mixed_fp64_krylov", ie.IE_MIXED_FP64K), ("mixed_c64_krylov", ie.IE_MIXED),
                       ("fp64", ie.IE_FP64)):
        ud = torch.zeros_like(bd)
        st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), 2, TOL, precision=prec)
        torch.cuda.synchronize()
        out[name] = {"status": int(st), "iters": info.inner_iters, "gpu_res": info.final_rel_res,
                     "oracle_res": oracle_residual(mp, qt, b, ud.cpu().numpy())}
    ctx.close()
    out["seconds"] = time.perf_counter() - t0
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def _stats(xs):
    xs = sorted(xs)
    return {"median": float(np.median(xs)), "min": float(xs[0]), "max": float(xs[-1]), "n": len(xs)}


def run_ours(args, rank, ws):
    import torch
    from paper_1512_06126_gb300 import build, ie

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    model = workload(args.workload)
    g = model.grid
    R = 2
    n_unk = 3 * g.nx * g.ny * g.nz
    t0 = time.perf_counter()
    ctx = ie.Context(g, model.layers, model.sigma_a, model.freqs[:1], None, max_rhs=R, restart=args.restart,
                     inner_tol=args.inner_tol)
    t_setup = time.perf_counter() - t0
    tune_v, tune_ms = ctx.contract_tuning()
    b = torch.empty((R, 3, g.nz, g.ny, g.nx), dtype=torch.complex128, device="cuda")
    for r in range(R):
        ctx.rhs_mt(0, r, b[r].data_ptr())
    u = torch.zeros_like(b)
    torch.cuda.synchronize()
    ext = torch.cuda.ExternalStream(ctx.stream)
    PREC = ie.IE_MIXED_FP64K

    def solve(c, precision, uu=u):
        st, info = c.solve(0, b.data_ptr(), uu.data_ptr(), R, TOL, precision=precision)
        if st != ie.IE_OK:
            raise RuntimeError(f"solve did not converge: status {st}, residual {info.final_rel_res:.2e}")
        return info

    for _ in range(args.warmup):
        solve(ctx, PREC)
    # ---- timed region: K solves in the timed mode, device-resident inputs ----
    clocks = Clocks(dev)
    barrier(ws)
    torch.cuda.synchronize()
    clocks.start()
    ctx.profile(True)
    # marks the timed region for a profiler started with --profile-from-start off (no
    # effect otherwise)
    torch.cuda.profiler.start()
    l0 = ie.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    with torch.cuda.stream(ext):
        evs[0].record()
    iters = 0
    outer = 0
    res = 0.0
    for k in range(args.steps):
        info = solve(ctx, PREC)
        iters += info.inner_iters
        outer += info.outer_iters
        res = max(res, info.final_rel_res)
        with torch.cuda.stream(ext):
            evs[k + 1].record()
    evs[-1].synchronize()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    barrier(ws)
    l1 = ie.kernel_launches()
    k3_ms, k3_n = ctx.profile_read(ie.IE_C64)
    ctx.profile(False)
    clk = clocks.stop()
    t_ms = evs[0].elapsed_time(evs[-1])
    step_s = [evs[k].elapsed_time(evs[k + 1]) / 1e3 for k in range(args.steps)]
    t_max = allreduce_max(t_ms / 1e3, ws)
    units = allreduce_sum(float(n_unk) * R * iters, ws)
    value = units / t_max

    # ---- where an inner iteration goes: one more (untimed) solve per mode, every step timed ----
    def breakdown_of(precision):
        ctx.profile(2)
        info_b = solve(ctx, precision)
        spans = {}
        for key, kind in (("product_c64", ie.IE_PROF_PRODUCT_C64), ("product_c128", ie.IE_PROF_PRODUCT_C128),
                          ("gram_schmidt_c64", ie.IE_PROF_GS_C64), ("gram_schmidt_c128", ie.IE_PROF_GS_C128),
                          ("givens", ie.IE_PROF_GIVENS), ("contraction_c64", ie.IE_C64),
                          ("contraction_c128", ie.IE_C128)):
            ms_k, n_k = ctx.profile_read(kind)
            if n_k:
                spans[key] = {"ms_total": ms_k, "records": n_k, "ms_each": ms_k / n_k}
        ctx.profile(False)
        return {"inner_iters": info_b.inner_iters, "outer": info_b.outer_iters, "solve_s": info_b.t_solve,
                "spans": spans}
    breakdown = {"mixed_fp64_krylov": breakdown_of(PREC), "mixed_c64_krylov": breakdown_of(ie.IE_MIXED)}

    # ---- time-to-solution: the timed mode, IE_MIXED and the plain FP64 solve ----
    def timed_solves(c, precision, n):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
        ex = torch.cuda.ExternalStream(c.stream)
        uu = torch.zeros_like(b)
        solve(c, precision, uu)
        infos = []
        with torch.cuda.stream(ex):
            e[0].record()
        for k in range(n):
            uu.zero_()
            torch.cuda.synchronize()
            with torch.cuda.stream(ex):
                e[k].record()
            infos.append(solve(c, precision, uu))
            with torch.cuda.stream(ex):
                e[k + 1].record()
            e[k + 1].synchronize()
        return [e[k].elapsed_time(e[k + 1]) / 1e3 for k in range(n)], infos
    mx_s, mx_info = timed_solves(ctx, ie.IE_MIXED, args.tts_repeats)
    # the plain FP64 solve at its own best restart length (longer than the mixed one's),
    # on a context of its own
    if not args.skip_fp64:
        ctx64 = ie.Context(g, model.layers, model.sigma_a, model.freqs[:1], None, max_rhs=R,
                           restart=args.restart_fp64)
        fp_s, fp_info = timed_solves(ctx64, ie.IE_FP64, args.tts_repeats)
        ctx64.close()
    tts = {"timed_mode": "IE_MIXED_FP64K",
           "mixed_fp64_krylov_s": _stats(step_s), "mixed_fp64_krylov_iters": iters / args.steps,
           "mixed_fp64_krylov_outer": outer / args.steps, "mixed_fp64_krylov_final_rel_res": res,
           "mixed_c64_krylov_s": _stats(mx_s), "mixed_c64_krylov_iters": mx_info[0].inner_iters,
           "mixed_c64_krylov_final_rel_res": max(i.final_rel_res for i in mx_info),
           "speedup_c64_krylov_vs_timed": float(np.median(step_s) / np.median(mx_s))}
    if not args.skip_fp64:
        tts.update({"fp64_s": _stats(fp_s), "fp64_iters": fp_info[0].inner_iters,
                    "fp64_final_rel_res": max(i.final_rel_res for i in fp_info),
                    "speedup_timed_vs_fp64": float(np.median(fp_s) / np.median(step_s)),
                    "speedup_c64_krylov_vs_fp64": float(np.median(fp_s) / np.median(mx_s))})

    # ---- matvec GB/s (c64, both polarisations) ----
    nf = (g.nx + 1) * (g.ny + 1)
    bs = 2 * g.nz * (2 * g.nz + 1)
    q_bytes = nf * bs * 8
    xs = torch.randn((R, 3, g.nz, g.ny, g.nx), dtype=torch.complex64, device="cuda")
    ys = torch.empty_like(xs)
    torch.cuda.synchronize()
    # launched on the context's stream; events recorded on that same stream
    for _ in range(3):
        ctx.matvec(0, xs.data_ptr(), ys.data_ptr(), R, dtype=ie.IE_C64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_mv = 20
    with torch.cuda.stream(ext):
        e0.record()
    for _ in range(n_mv):
        ctx.matvec(0, xs.data_ptr(), ys.data_ptr(), R, dtype=ie.IE_C64)
    with torch.cuda.stream(ext):
        e1.record()
    e1.synchronize()
    if ctx.sync() != ie.IE_OK:
        raise RuntimeError("a contraction wait ran out during the product timing")
    mv_ms = e0.elapsed_time(e1) / n_mv
    mv_bytes = q_bytes + 2 * 8 * n_unk * R
    kern_ms = ctx.profile_matvec(0, R, ie.IE_C64, 10)
    hbm_peak, sm_max, peak_src = peaks()

    # ---- roofline of the contraction kernel (timed during the steps) ----
    k3_avg_ms = k3_ms / max(k3_n, 1)
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
    # capture of this kernel variant, as it is now, on this workload (profiles/); null for
    # any other variant or workload
    variant = int(tune_v[R - 1])
    traffic = CONTRACT_TRAFFIC.get((args.workload, variant, R))
    # algorithmic bytes of the contraction: the c64 coefficients once plus the product's
    # input and output vectors (the spectrum round trip is the kernel's own traffic)
    k3_alg = q_bytes + 2 * 8 * n_unk * R
    k3_own = q_bytes + 2 * 4 * g.nx * g.ny * 3 * g.nz * R * 8
    k3_flops = 8.0 * 4 * g.nx * g.ny * R * 9 * g.nz * g.nz
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12            # TFLOP/s, FP32 FMA pipes at max clock
    bf16 = bf16_peak()
    tf32_peak = bf16[0] * 1.1 / 2.25
    tensor = variant in TENSOR_VARIANTS
    f16 = variant == 7
    achieved = k3_alg / (k3_avg_ms * 1e-3) / 1e9
    roof = {"kernel": f"contract (c64, 2 right-hand sides, variant {variant})", "bound": "hbm",
            "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
            "peak_source": peak_src, "bytes_per_launch": k3_alg,
            "bytes_definition": "algorithmic: c64 coefficients once + input and output vectors of the product",
            "kernel_bytes_per_launch": k3_own,
            "kernel_bytes_definition": "coefficients + the spectrum read and written",
            "kernel_frac": k3_own / (k3_avg_ms * 1e-3) / 1e9 / hbm_peak,
            "traffic": traffic, "launches": k3_n, "avg_ms": k3_avg_ms,
            "compute": ("tensor, 2xFP16 split (3 products)" if f16 else "tensor, 3xTF32") if tensor else "FP32 FMA",
            "flops_per_launch": 3 * k3_flops if tensor else k3_flops,
            "compute_peak_TFLOPs": (bf16[0] if f16 else tf32_peak) if tensor else fp32_peak,
            "compute_peak_source": ((f"{bf16[1]} bf16 {bf16[0]:.0f} TFLOP/s (FP16 runs at the bf16 rate)" if f16 else
                                     f"{bf16[1]} bf16 {bf16[0]:.0f} TFLOP/s x 1.1/2.25") if tensor else
                                    f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz"),
            "compute_TFLOPs": (3 if tensor else 1) * k3_flops / (k3_avg_ms * 1e-3) / 1e12}

    # ---- e2e: through the ABI with host buffers ----
    bh = b.cpu().pin_memory()
    uh = torch.empty_like(bh).pin_memory()
    bd = torch.empty_like(b)
    ud = torch.empty_like(b)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    it_e2e = 0
    n_e2e = max(1, min(args.steps, 3))
    for _ in range(n_e2e):
        bd.copy_(bh, non_blocking=True)
        torch.cuda.synchronize()
        st, info = ctx.solve(0, bd.data_ptr(), ud.data_ptr(), R, TOL, precision=PREC)
        uh.copy_(ud, non_blocking=True)
        it_e2e += info.inner_iters
    e1.record()
    e1.synchronize()
    t_e2e = e0.elapsed_time(e1) / 1e3
    e2e_value = allreduce_sum(float(n_unk) * R * it_e2e, ws) / allreduce_max(t_e2e, ws)
    ctx.close()
    del xs, ys, bd, ud
    torch.cuda.empty_cache()

    # ---- cpu baseline and the accuracy check against the oracle (rank 0, N = 1) ----
    cpu = None
    err = None
    # the oracle holds the full spectral blocks, 4 Nx Ny (3 Nz)^2 complex128
    oracle_bytes = 4 * g.nx * g.ny * (3 * g.nz) ** 2 * 16
    if oracle_bytes > 20e9:
        err = cpu = {"skipped": f"the oracle's spectral blocks would take {oracle_bytes / 1e9:.0f} GB of host memory"}
    elif rank == 0 and ws == 1 and not args.no_cpu:
        err = oracle_check(model, args)
        ncores = os.cpu_count() or 1
        legs = [cpu_leg(args.workload, th, args.cpu_iters) for th in (1, ncores)]
        best = max(legs, key=lambda d: d["iters"] / d["seconds"])
        cpu = {"value": n_unk * best["iters"] / best["seconds"], "unit": UNIT, "cores": best["threads"],
               "kind": "oracle",
               "sample": f"{args.cpu_iters} FP64 GMRES iterations (FFT product + CGS2) of the numpy oracle, one "
                         "right-hand side, same grid, random coefficient tensor of the same shape; the cycle's "
                         "initial-residual product timed apart and subtracted; run with BLAS/OpenMP threads capped "
                         "at 1 and at all host cores (numpy's FFT and einsum use one thread either way)",
               "legs": [{"threads": d["threads"], "value": n_unk * d["iters"] / d["seconds"],
                         "seconds": d["seconds"], "iters": d["iters"]} for d in legs]}

    # ---- the batched configuration (four grids, 32 instances) in the timed precision ----
    c3 = None
    if rank == 0 and ws == 1 and args.workload == "C2" and not args.skip_c3:
        c3 = c3_summary(args, ie.IE_MIXED_FP64K, with_fp64=not args.skip_fp64)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "c64 products (FP32 FFTs and contraction) in the inner GMRES, FP64 Krylov vectors "
                         "and rotations, Gram-Schmidt on them in double-float; c128 refinement residual "
                         "with the FP64 contraction",
                "data": "synthetic",
                "config": {"workload": workload_desc(args.workload, model),
                           "unknowns": n_unk, "rhs": R, "restart": args.restart,
                           "inner_tol": args.inner_tol, "restart_fp64": args.restart_fp64,
                           "precision": "IE_MIXED_FP64K",
                           "l2": "inputs larger than L2 (c64 coefficients %.0f MB)" % (q_bytes / 1e6),
                           "parallelism": f"replicas x{ws}", "coefficients": "generated on the device",
                           "setup_s": t_setup},
                "matvec": {"GBs": mv_bytes / (mv_ms * 1e-3) / 1e9, "frac": mv_bytes / (mv_ms * 1e-3) / 1e9 / hbm_peak,
                           "ms": mv_ms, "bytes": mv_bytes,
                           "kernel_ms": {"rows_fwd": kern_ms[0], "cols_fwd": kern_ms[1], "contract": kern_ms[2],
                                         "cols_inv": kern_ms[3], "rows_inv": kern_ms[4]}},
                "tts": tts,
                "roofline": roof,
                "err_vs_oracle": err,
                "solve_breakdown": breakdown,
                "contract_tuning": {"variants": VARIANT_NAMES, "chosen_for_2_rhs": variant,
                                    "ms_per_launch_2_rhs": [float(v) for v in tune_ms[1]]},
                "c3_batch": c3,
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b.numel() * 16),
                        "d2h_bytes_per_step": int(b.numel() * 16)},
                "gpu_launches": int(l1 - l0),
                "clocks": clk}
        print(json.dumps(line), flush=True)


def run_matvec_only(args):
    """Setup plus --warmup + --steps c64 products of both polarisations (used for kernel
    profiles of the product on its own)."""
    import torch
    from paper_1512_06126_gb300 import build, ie
    build.build()
    model = workload(args.workload)
    g = model.grid
    R = 2
    ctx = ie.Context(g, model.layers, model.sigma_a, model.freqs[:1], None, max_rhs=R,
                     autotune=args.variant < 0)
    if args.variant >= 0:
        ctx.set_contract_variant(R, args.variant)
    xs = torch.randn((R, 3, g.nz, g.ny, g.nx), dtype=torch.complex64, device="cuda")
    ys = torch.empty_like(xs)
    torch.cuda.synchronize()
    ext = torch.cuda.ExternalStream(ctx.stream)
    for _ in range(args.warmup):
        ctx.matvec(0, xs.data_ptr(), ys.data_ptr(), R, dtype=ie.IE_C64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # the timed products are the region a profiler started with --profile-from-start off sees
    torch.cuda.profiler.start()
    with torch.cuda.stream(ext):
        e0.record()
    for _ in range(args.steps):
        ctx.matvec(0, xs.data_ptr(), ys.data_ptr(), R, dtype=ie.IE_C64)
    with torch.cuda.stream(ext):
        e1.record()
    e1.synchronize()
    torch.cuda.profiler.stop()
    if ctx.sync() != ie.IE_OK:
        raise RuntimeError("a contraction wait ran out")
    kern = ctx.profile_matvec(0, R, ie.IE_C64, max(args.steps, 1))
    print(json.dumps({"mode": "matvec", "workload": args.workload, "variant": args.variant,
                      "ms_per_product": e0.elapsed_time(e1) / args.steps,
                      "kernel_ms": dict(zip(("rows_fwd", "cols_fwd", "contract", "cols_inv", "rows_inv"), kern))}))
    ctx.close()


def c3_summary(args, precision, with_fp64=True):
    """The batched configuration: 16 frequencies x 2 polarisations over four grids
    (64^2x16, 96^2x24, 128^2x32, 192^2x48; frequency k on grid k mod 4).  Per grid, its
    four frequencies (8 right-hand sides) are solved in one batched solve
    (ie_solve_batch) in `precision`, then one instance at a time in the same precision,
    then (with_fp64) batched in plain FP64 on a context of its own (restart
    --restart-fp64).  Device time with CUDA events on the library stream, after one
    untimed solve of each kind."""
    import torch
    from paper_1512_06126_gb300 import build, ie
    build.build()
    out = []
    t_b = t_s = t_64 = 0.0

    def timed(ctx, fn):
        ext = torch.cuda.ExternalStream(ctx.stream)
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(ext):
            e0.record()
        r = fn()
        with torch.cuda.stream(ext):
            e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3, r

    for m in W.config3():
        g = m.grid
        nf = len(m.freqs)
        ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs, None, max_rhs=2 * nf, restart=args.restart,
                         inner_tol=args.inner_tol)
        b = torch.empty((nf, 2, 3, g.nz, g.ny, g.nx), dtype=torch.complex128, device="cuda")
        for k in range(nf):
            for p in range(2):
                ctx.rhs_mt(k, p, b[k, p].data_ptr())
        u = torch.zeros_like(b)
        torch.cuda.synchronize()
        insts = list(range(nf))

        def batched(c=ctx, prec=precision, uu=u):
            uu.zero_()
            return c.solve_batch(insts, b.data_ptr(), uu.data_ptr(), 2, TOL, precision=prec)
        tb, (st, info) = timed(ctx, batched)
        u1 = torch.zeros_like(b[0])

        def singles():
            its, res, sts = 0, 0.0, []
            for k in range(nf):
                u1.zero_()
                st1, i1 = ctx.solve(k, b[k].data_ptr(), u1.data_ptr(), 2, TOL, precision=precision)
                its += i1.inner_iters
                res = max(res, i1.final_rel_res)
                sts.append(st1)
            return its, res, sts
        ts, (it_single, res1, st1) = timed(ctx, singles)
        ctx.close()
        rec = {"grid": f"{g.nx}x{g.ny}x{g.nz}", "instances": 2 * nf, "batched_s": tb,
               "batched_iters": info.inner_iters, "batched_res": info.final_rel_res, "one_at_a_time_s": ts,
               "one_at_a_time_iters": it_single, "one_at_a_time_res": res1, "status": [st] + st1}
        if with_fp64:
            ctx64 = ie.Context(g, m.layers, m.sigma_a, m.freqs, None, max_rhs=2 * nf, restart=args.restart_fp64)
            t64, (st64, info64) = timed(ctx64, lambda: batched(ctx64, ie.IE_FP64))
            ctx64.close()
            rec.update({"fp64_batched_s": t64, "fp64_iters": info64.inner_iters, "fp64_res": info64.final_rel_res,
                        "fp64_status": st64})
            t_64 += t64
        out.append(rec)
        t_b += tb
        t_s += ts
        del b, u, u1
        torch.cuda.empty_cache()
    res = {"workload": "C3: 32 instances (16 frequencies x 2 polarisations) over 4 grids",
           "metric": "solved instances/s (tol 1e-7)", "precision": {ie.IE_MIXED: "IE_MIXED",
                                                                     ie.IE_MIXED_FP64K: "IE_MIXED_FP64K",
                                                                     ie.IE_FP64: "IE_FP64"}[precision],
           "batched": 32 / t_b, "one_at_a_time": 32 / t_s, "batched_s": t_b, "one_at_a_time_s": t_s,
           "tol": TOL, "per_grid": out}
    if with_fp64:
        res.update({"fp64_batched_s": t_64, "fp64": 32 / t_64, "speedup_batched_vs_fp64": t_64 / t_b,
                    "speedup_batched_vs_one_at_a_time": t_s / t_b})
    return res


def run_batch(args):
    print(json.dumps({"mode": "batch", **c3_summary(args, PRECISIONS_BY_NAME[args.precision],
                                                    with_fp64=not args.skip_fp64)}),
          flush=True)


def run_maps(args):
    """Field recovery at sites and the MT maps of the COMMEMI3D-3-like model (Sect. 4):
    both polarisations solved in IE_MIXED_FP64K (tol 1e-7), the fields recovered at
    two profiles of sites off the cell centres (x = 1.9 km and y = 3.83 km of the model,
    a site every 100 m), the impedances and the apparent resistivity / phase; device
    time of each stage (set-up of the site kernels: host clock, synchronous)."""
    import torch
    from paper_1512_06126_gb300 import build, ie
    build.build()
    m = W.commemi3d3_like()
    g = m.grid
    ox, oy = W.COMMEMI3D3_ORIGIN
    t0 = time.perf_counter()
    ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs, None, max_rhs=2, restart=args.restart,
                     inner_tol=args.inner_tol)
    t_setup = time.perf_counter() - t0
    b = torch.empty((2, 3, g.nz, g.ny, g.nx), dtype=torch.complex128, device="cuda")
    for p in range(2):
        ctx.rhs_mt(0, p, b[p].data_ptr())
    u = torch.zeros_like(b)
    torch.cuda.synchronize()
    ext = torch.cuda.ExternalStream(ctx.stream)

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(ext):
            e0.record()
        r = fn()
        with torch.cuda.stream(ext):
            e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1), r

    ms_solve, (st, info) = timed(lambda: ctx.solve(0, b.data_ptr(), u.data_ptr(), 2, TOL,
                                                   precision=ie.IE_MIXED_FP64K))
    # profile A along y at x = 1.9 km (a cell face), profile B along x at y = 3.83 km
    ys = (np.arange(g.ny) + 0.5) * g.hy
    xs = (np.arange(g.nx) + 0.5) * g.hx
    sx = np.concatenate([np.full(g.ny, 1900.0 + ox), xs])
    sy = np.concatenate([ys, np.full(g.nx, 3830.0 + oy)])
    n_rec = sx.size
    t0 = time.perf_counter()
    ctx.set_receivers_xy(sx, sy, 0.0)
    t_sites = time.perf_counter() - t0
    f = torch.empty((2, n_rec, 4), dtype=torch.complex128, device="cuda")
    z = torch.empty((n_rec, 4), dtype=torch.complex128, device="cuda")
    c = torch.empty((2, n_rec, 4), dtype=torch.complex128, device="cuda")
    zobs = torch.zeros_like(z)
    rho = torch.empty((n_rec, 4), dtype=torch.float64, device="cuda")
    ph = torch.empty_like(rho)
    ms_fields, _ = timed(lambda: ctx.receiver_fields(0, u.data_ptr(), 2, (0, 1), f.data_ptr()))
    ms_z, _ = timed(lambda: ctx.mt_misfit(f.data_ptr(), zobs.data_ptr(), z.data_ptr(), c.data_ptr()))
    ms_maps, _ = timed(lambda: ctx.mt_apparent(0, z.data_ptr(), n_rec, rho.data_ptr(), ph.data_ptr()))
    rho_h, ph_h = rho.cpu().numpy(), ph.cpu().numpy()
    ctx.close()
    a, bb = slice(0, g.ny), slice(g.ny, n_rec)
    print(json.dumps({
        "mode": "maps", "workload": f"COMMEMI3D-3-like: {g.nx}x{g.ny}x{g.nz} cells, 7 blocks (max contrast "
                                    f"3.3e4), period 1 s, 2 polarisations, tol {TOL}",
        "setup_s": t_setup, "status": st, "inner_iters": info.inner_iters, "outer": info.outer_iters,
        "final_rel_res": info.final_rel_res, "solve_s": ms_solve / 1e3, "sites": int(n_rec),
        "site_kernels_s": t_sites, "fields_ms": ms_fields, "impedance_ms": ms_z, "maps_ms": ms_maps,
        "profile_x1.9km": {"y_km": list(np.round(ys / 1000 - oy / 1000, 3)),
                           "rho_xy": list(np.round(rho_h[a, 1], 4)), "phase_xy": list(np.round(ph_h[a, 1], 3))},
        "profile_y3.83km": {"x_km": list(np.round(xs / 1000 - ox / 1000, 3)),
                            "rho_yx": list(np.round(rho_h[bb, 2], 4)), "phase_yx": list(np.round(ph_h[bb, 2], 3))},
    }), flush=True)


def run_block_eval(args):
    """Evaluation of block GMRES across the two polarisations (one Krylov space of block
    size 2) against two independent GMRES(m), for the decision whether to build it: the
    same operator (the library's c128 product through ie_matvec on the C2 workload), the
    Arnoldi steps and least-squares problems in plain torch, and the number of block
    steps / iterations to ||b - A x|| <= 1e-7 ||b|| counted (one step of either costs one
    product of two vectors).  Not a solver of the library."""
    import torch
    from paper_1512_06126_gb300 import build, ie
    build.build()
    m = workload(args.workload)
    g = m.grid
    N = 3 * g.nz * g.ny * g.nx
    ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs[:1], None, max_rhs=2)
    b = torch.empty((2, N), dtype=torch.complex128, device="cuda")
    for p in range(2):
        ctx.rhs_mt(0, p, b[p].data_ptr())
    torch.cuda.synchronize()

    def A(X):
        Y = torch.empty_like(X)
        torch.cuda.synchronize()
        ctx.matvec(0, X.data_ptr(), Y.data_ptr(), X.shape[0], dtype=ie.IE_C128)
        if ctx.sync() != ie.IE_OK:
            raise RuntimeError("a contraction wait ran out")
        return Y

    def lstsq(H, E):
        return torch.linalg.lstsq(H.cpu(), E.cpu()).solution.to(H.device)

    def block_gmres(B, mrest, maxit):
        p = B.shape[0]
        nbB = B.norm(dim=1)
        X = torch.zeros_like(B)
        its = 0
        while its < maxit:
            R = B - A(X)
            if (R.norm(dim=1) <= TOL * nbB).all():
                return its
            Q, Rr = torch.linalg.qr(R.T)
            V = [Q.T.contiguous()]
            H = torch.zeros(((mrest + 1) * p, mrest * p), dtype=torch.complex128, device="cuda")
            E = torch.zeros(((mrest + 1) * p, p), dtype=torch.complex128, device="cuda")
            E[:p, :] = Rr
            for k in range(mrest):
                Wk = A(V[k])
                its += 1
                Vm = torch.cat(V)
                h = Vm.conj() @ Wk.T
                Wk = Wk - (Vm.T @ h).T
                h2 = Vm.conj() @ Wk.T
                Wk = Wk - (Vm.T @ h2).T
                Qk, Rk = torch.linalg.qr(Wk.T)
                H[:(k + 1) * p, k * p:(k + 1) * p] = h + h2
                H[(k + 1) * p:(k + 2) * p, k * p:(k + 1) * p] = Rk
                V.append(Qk.T.contiguous())
                Hk = H[:(k + 2) * p, :(k + 1) * p]
                Y = lstsq(Hk, E[:(k + 2) * p])
                if ((E[:(k + 2) * p] - Hk @ Y).norm(dim=0) <= TOL * nbB).all() or k == mrest - 1:
                    X = X + (torch.cat(V[:k + 1]).T @ Y).T
                    break
        return its

    out = {"mode": "block-eval", "workload": workload_desc(args.workload, m), "tol": TOL, "restarts": {}}
    for mrest in (45, 20):
        sep = [block_gmres(b[p:p + 1], mrest, 2000) for p in range(2)]
        blk = block_gmres(b, mrest, 2000)
        out["restarts"][str(mrest)] = {"separate_iterations": sep, "lockstep_iterations": max(sep),
                                       "block_steps": blk}
    ctx.close()
    print(json.dumps(out), flush=True)


def run_gradient(args):
    """MT misfit and its gradient on the 64x64x24 workload: 8 frequencies x 2
    polarisations, 16 x 16 receivers every second cell over the centre, observed
    impedances from the same model with the anomaly conductivities doubled.  Times one
    misfit evaluation (16 forward solves, FP64) and one gradient (16 adjoint solves)
    after one untimed pair."""
    import torch
    from paper_1512_06126_gb300 import build, ie, mt
    build.build()
    m = W.config4()
    g = m.grid
    sb = W.background_sigma(g, m.layers)
    base = np.broadcast_to(sb[:, None, None], m.sigma_a.shape).astype(np.complex128).copy()
    ctx = ie.Context(g, m.layers, m.sigma_a, m.freqs, None, max_rhs=2)
    idx = np.arange(16, 48, 2)
    ix, iy = np.meshgrid(idx, idx)
    n_inst = len(m.freqs)
    P = mt.MTProblem(ctx, ix.ravel(), iy.ravel(), np.zeros((n_inst, ix.size, 2, 2), dtype=np.complex128),
                     tol=1e-9, precision=ie.IE_FP64)
    truth = m.sigma_a.copy()
    an = np.abs(truth - base) > 0
    truth[an] *= 2.0
    ctx.set_sigma(truth)
    P.misfit()
    P.zobs.copy_(P.z)
    ctx.set_sigma(m.sigma_a)
    P.misfit()
    P.gradient()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    phi = P.misfit()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    grad = P.gradient()
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    gn = grad.cpu().numpy()
    print(json.dumps({"mode": "gradient", "workload": "C4: 64x64x24 cells, 8 frequencies x 2 polarisations, "
                      "16x16 receivers, FP64 solves to 1e-9", "misfit": phi, "misfit_s": t1 - t0,
                      "gradient_s": t2 - t1, "anomalous_cells": int(an.sum()),
                      "gradient_norm": float(np.linalg.norm(gn)), "gradient_nonzero": int((gn != 0).sum()),
                      "forward_iters": P.iters["forward"], "adjoint_iters": P.iters["adjoint"]}), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="C2", choices=["C1", "C2", "C4", "C5"])
    ap.add_argument("--restart", type=int, default=20)
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--restart-fp64", type=int, default=45)
    ap.add_argument("--tts-repeats", type=int, default=3)
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--threads", type=int, default=1, help=argparse.SUPPRESS)
    ap.add_argument("--iters", type=int, default=3, help=argparse.SUPPRESS)
    ap.add_argument("--mode", choices=["solve", "matvec", "batch", "gradient", "maps", "block-eval"],
                    default="solve")
    ap.add_argument("--precision", choices=list(PRECISIONS_BY_NAME), default="fp64k",
                    help="batch mode: the precision of the batched and one-at-a-time solves")
    ap.add_argument("--skip-fp64", action="store_true", help="skip the plain FP64 comparisons")
    ap.add_argument("--skip-c3", action="store_true", help="leave the batched four-grid summary out of the solve line")
    ap.add_argument("--variant", type=int, default=-1,
                    help="matvec mode: force this contraction variant (default: the autotuner's choice)")
    args = ap.parse_args()
    if args.cpu_sample:
        run_cpu_sample(args)
        return
    rank, ws = dist_setup()
    if args.mode == "matvec":
        run_matvec_only(args)
    elif args.mode == "batch":
        run_batch(args)
    elif args.mode == "gradient":
        run_gradient(args)
    elif args.mode == "maps":
        run_maps(args)
    elif args.mode == "block-eval":
        run_block_eval(args)
    elif args.impl == "reference":
        run_reference(args, rank, ws)
    else:
        run_ours(args, rank, ws)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
