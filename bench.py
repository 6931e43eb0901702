"""Benchmark: spherical Poisson solves per second on GB300, in DOF/s.

One step = one full solve (all five kernels: longitude FFTs, folded colatitude
transforms, per-k parity tridiagonal solves, inverse transforms) of the
5000 x 10000 grid (DFS 10^4 x 10^4) with a random spherical-harmonic series
l <= 2000, coefficients N(0,1)/(1+l)^2, in FP64.  DOF = n_theta * n_lambda per
solve (the paper's mn/2 convention).  Inputs (400 MB) are larger than the
129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank solves its own independent problem (weak
scaling, replicas: the single solve has no exchange step on one GPU); rank 0
prints one JSON line.  --impl reference times the CPU oracle instead (rank 0
only).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Poisson DOF/s on 1 GB300 at stated error vs FP64 oracle"
WORKLOAD = "sh2000_5000x10000"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# FP64 pipe peak if the live probe fails: 504 G DFMA/s, measured on a GB300 by
# the library's register-only FMA loop filling every SM (sphere_poisson_pipe_rates),
# = 1008 GFLOP/s counting an FMA as 2 flops.
FP64_PEAK_GFLOPS_FALLBACK = 1008.0

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of each FP64
# stage kernel, from one ncu capture of the 5000 x 5000 workload (the colatitude
# transforms of the 5000 x 10000 grid on half the longitudes; 200 MB input, larger
# than L2) on the stage-kernel sources whose hash is `csrc_sha256`, with
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum` on one solve after
# warm-up (read + write bytes below).  bench.py scales them to its own grid by the
# spectrum size n_theta * Kp (every stage streams the spectrum once or twice) and
# reports null when the sources have changed since the capture.
TRAFFIC_CAPTURE = {
    "csrc_sha256": "02e997e5d6337967",
    "n_theta": 5000, "n_lambda": 5000,
    "bytes": {"rows_forward": 200256000 + 146959616, "theta_forward": 200861184 + 159193088,
              "solve": 662352640 + 321982976, "theta_inverse": 201085696 + 164486400,
              "rows_inverse": 200748032 + 146642688},
}
# the same for the FP32 form's dominant kernel, the fused colatitude stage
# (k_theta_fused1 with two columns per CTA, its tile by TMA, at 5000 x 5000;
# `ncu --section ... --metrics dram__bytes_read.sum,dram__bytes_write.sum` on
# two launches after warm-up), over the sources it is compiled from
TRAFFIC_CAPTURE_FP32 = {
    "csrc_sha256": "825b545093ed33d5",
    "n_theta": 5000, "n_lambda": 5000,
    "bytes": {"theta_fused": 150896640 + 50061568},
}


# the sources the five stage kernels of the solve are compiled from (the
# operators of calculus.cuh and the plan code do not enter their code)
TRAFFIC_SOURCES = ("fft.cuh", "kernels.cuh", "launchers.inl")
TRAFFIC_SOURCES_FP32 = ("fft.cuh", "kernels.cuh", "launchers.inl", "fused.cuh")


def csrc_hash(sources=TRAFFIC_SOURCES) -> str:
    """First 16 hex digits of SHA-256 over the stage kernels' sources (names and bytes)."""
    import hashlib

    d = os.path.join(ROOT, "paper_1510_08094_gb300", "csrc")
    h = hashlib.sha256()
    for n in sources:
        h.update(n.encode())
        with open(os.path.join(d, n), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(stage: str, n_theta: int, n_lambda: int, precision: str):
    """(bytes per launch, note) of an FP64 stage kernel scaled from the ncu capture,
    or (None, why) when no capture of the current sources exists."""
    if precision == "fp64":
        cap, sources = TRAFFIC_CAPTURE, TRAFFIC_SOURCES
    elif precision == "fp32":
        cap, sources = TRAFFIC_CAPTURE_FP32, TRAFFIC_SOURCES_FP32
    else:
        return None, "no ncu traffic capture of the double-float kernels on these sources"
    if stage not in cap["bytes"]:
        return None, f"no ncu traffic capture of the {stage} kernel"
    if csrc_hash(sources) != cap["csrc_sha256"]:
        return None, "kernel sources changed since the ncu traffic capture"
    kp = lambda nl: (nl // 2 + 2) // 2 * 2
    ratio = (n_theta * kp(n_lambda)) / (cap["n_theta"] * kp(cap["n_lambda"]))
    note = (f"ncu dram read+write of one {cap['n_theta']}x{cap['n_lambda']} launch x {ratio:.4f} "
            f"(spectrum-size ratio); writes still dirty in L2 at kernel end are not counted")
    return int(cap["bytes"][stage] * ratio), note


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def init_ranks(backend: str):
    """(rank, world, local rank) from the launcher's environment; joins the
    process group (backend "nccl" on GPUs, "gloo" in the CPU tests) when world > 1."""
    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if world > 1:
        import torch
        import torch.distributed as dist

        kw = {"device_id": torch.device("cuda", local)} if backend == "nccl" else {}
        dist.init_process_group(backend, **kw)
    return rank, world, local


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: every rank's timed region ends at the barrier
    that follows it, so the job's time is the maximum."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(dof_per_rank: int, world: int, ms_per_step: float) -> float:
    """DOF/s of the whole job: every rank solves its own problem (weak scaling)."""
    return dof_per_rank * world / (ms_per_step * 1e-3)


def shard_lpt(sizes, world: int):
    """Split independent problems of the given (n_theta, n_lambda) sizes over
    `world` ranks by the longest-processing-time rule: largest problem first
    (ties by index), each to the rank with the least work so far (ties to the
    lowest rank), work = n_theta * n_lambda.  Returns one sorted index list per
    rank.  Deterministic, so every rank computes the same split without any
    exchange."""
    order = sorted(range(len(sizes)), key=lambda b: (-sizes[b][0] * sizes[b][1], b))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda i: (load[i], i))
        parts[r].append(b)
        load[r] += sizes[b][0] * sizes[b][1]
    return [sorted(p) for p in parts]


def algorithmic_flops(n_theta: int, n_lambda: int) -> dict:
    """Conventional FFT flop counts per stage launch: a real FFT of length n costs
    2.5 n log2 n, the folded colatitude transform of one complex column of length
    N costs 5 N log2 N (two real DCTs), the per-k eliminations 10 flops per (j, k)."""
    N, n = n_theta, n_lambda
    K = n // 2 + 1
    rows = N * 2.5 * n * math.log2(max(n, 2))
    cols = K * 5.0 * N * math.log2(max(N, 2))
    solve = 10.0 * N * K
    return {"rows_forward": rows, "theta_forward": cols, "solve": solve,
            "theta_inverse": cols, "rows_inverse": rows, "theta_fused": 2 * cols + solve}


def algorithmic_bytes(n_theta: int, n_lambda: int, spec_elem: int = 16, table_elem: int = 8) -> dict:
    """Bytes each stage must move: its input and output arrays once (plus the
    three factor tables of the eliminations).  spec_elem = bytes of one complex
    spectral value (16 in FP64 and double-float, 8 in FP32)."""
    N, n = n_theta, n_lambda
    Kp = (n // 2 + 2) // 2 * 2
    grid = 8.0 * N * n
    spec = float(spec_elem) * N * Kp
    K = n // 2 + 1
    return {"rows_forward": grid + spec, "theta_forward": 2 * spec, "solve": 2 * spec + 3.0 * table_elem * N * Kp,
            "theta_inverse": 2 * spec, "rows_inverse": spec + grid,
            # the fused colatitude stage of the FP32 form: the spectrum in and out once,
            # its per-column pivot table (K columns) once
            "theta_fused": 2 * spec + 1.0 * table_elem * N * K}


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = init_ranks("nccl")
    torch.cuda.set_device(local)
    import tempfile

    import paper_1510_08094_gb300 as sp
    from synth import sh

    if "SPHERE_POISSON_TUNE_CACHE" not in os.environ:
        os.environ["SPHERE_POISSON_TUNE_CACHE"] = os.path.join(tempfile.gettempdir(), "sphere_poisson_tune.txt")
    w = sh.workload(args.workload)
    N, n = w.n_theta, w.n_lambda
    dev = torch.device("cuda", local)
    f, u_exact = w.make(device=dev)
    tune = not args.no_autotune
    plan = sp.Plan(N, n, args.precision, args.sweeps, device=dev, autotune=tune)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream()

    # correctness at the stated error, on the solution the timed loop produces
    plan.solve(f, u, ws)
    torch.cuda.synchronize()
    err = float((u - u_exact).abs().max() / u_exact.abs().max())

    for _ in range(args.warmup):
        plan.solve(f, u, ws)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    plan.profile_begin(args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        plan.solve(f, u, ws)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stage_ms, recorded = plan.profile_end()
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, dev)
    ms_step = ms / args.steps
    dof = N * n
    value = whole_job_value(dof, world, ms_step)

    # end to end through the host-buffer C-ABI call (pinned host memory; the copies
    # of f in and u out are inside the timed region)
    f_host = f.cpu().pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    dbuf = torch.empty(plan.host_buffer_bytes(), dtype=torch.uint8, device=dev)
    for _ in range(2):
        plan.solve_host(f_host, u_host, dbuf)
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    # each call synchronises before it returns; the median of the per-call times
    # keeps host-side jitter (other processes on the shared host) out of the figure
    t_calls = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        plan.solve_host(f_host, u_host, dbuf)
        t_calls.append(time.perf_counter() - t0)
    # the slowest rank's time, as for the device-timed value
    t_e2e = max_over_ranks(statistics.median(t_calls) * 1e3, world, dev) * 1e-3
    t_e2e_mean = max_over_ranks(sum(t_calls) / len(t_calls) * 1e3, world, dev) * 1e-3
    e2e_err = float((u_host.cuda() - u_exact).abs().max() / u_exact.abs().max())

    # roofline of the dominant stage
    flops = algorithmic_flops(N, n)
    if args.precision == "fp32":
        bytes_ = algorithmic_bytes(N, n, 8, 4)
    else:
        bytes_ = algorithmic_bytes(N, n)
    dom = max(stage_ms, key=stage_ms.get)
    dom_ms = stage_ms[dom] / max(recorded, 1)
    achieved_gflops = flops[dom] / (dom_ms * 1e-3) / 1e9
    stage_share = {k: round(v / sum(stage_ms.values()), 4) for k, v in stage_ms.items()}
    dtype_name = {"fp64": "f64", "fp32": "f32", "fp32_refine": "f32+df64"}[args.precision]
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    try:
        rates = sp.pipe_rates()
        fp64_peak = 2.0 * rates["fp64_fma_gops"]
        peak_src = (f"measured live: FP64 FMA issue rate {rates['fp64_fma_gops']:.1f} G/s x 2 flops "
                    f"(sphere_poisson_pipe_rates)")
    except Exception as exc:  # keep the bench line even if the probe fails
        fp64_peak = FP64_PEAK_GFLOPS_FALLBACK
        peak_src = f"earlier probe on a GB300 (live probe failed: {exc})"
    hbm_gbs = bytes_[dom] / (dom_ms * 1e-3) / 1e9
    if args.precision == "fp32":
        # FP32 transforms are bounded by HBM traffic, not arithmetic
        roofline = {"kernel": dom, "bound": "hbm", "achieved": round(hbm_gbs, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(hbm_gbs / hbm_peak, 4),
                    "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)"}
    else:
        roofline = {"kernel": dom, "bound": "alu", "achieved": round(achieved_gflops / 1e3, 4),
                    "peak": round(fp64_peak / 1e3, 4), "unit": "TFLOP/s",
                    "frac": round(achieved_gflops / fp64_peak, 4), "peak_source": peak_src}
        if args.precision == "fp32_refine":
            roofline["note"] = ("double-float arithmetic on the FP32 pipes; achieved counts conventional "
                                "FP64-equivalent flops against the FP64 pipe peak")
    traffic, traffic_note = traffic_for(dom, N, n, args.precision)
    roofline.update({
        "traffic": traffic,
        "traffic_note": traffic_note,
        "algorithmic_bytes": int(bytes_[dom]),
        "hbm_achieved_gbs": round(hbm_gbs, 1),
        "hbm_peak_gbs": hbm_peak,
        "stage_ms_per_solve": {k: round(v / max(recorded, 1), 4) for k, v in stage_ms.items()},
        "stage_share": stage_share,
    })

    out = {
        "metric": METRIC,
        "value": value,
        "unit": "DOF/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": dtype_name,
        "data": "synthetic: seeded spherical-harmonic series (no dataset)",
        "config": {
            "precision": args.precision,
            "refine_sweeps": args.sweeps if args.precision == "fp32_refine" else None,
            "workload": f"{w.name}: {args.precision} solve, n_theta={N} x n_lambda={n} (DFS {2*N}x{n}), "
                        f"random SH series l<={w.lmax}, c~N(0,1)/(1+l)^2, seed {w.seed}",
            "dof_per_solve": dof,
            "dof_convention": "n_theta*n_lambda (= mn/2, the paper's); mn convention = 2x",
            "l2": f"inputs ({f.numel() * 8 / 1e6:.0f} MB) larger than L2 (129 MB); no flush",
            "tiles": "autotuned at plan time" if tune else "default",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "max_rel_err_vs_closed_form": err,
        },
        "clocks": clk,
        "gpu_launches": plan.launches() * args.steps,
        "e2e": {"value": dof * world / t_e2e, "unit": "DOF/s", "h2d_bytes_per_step": int(f.numel() * 8),
                "d2h_bytes_per_step": int(f.numel() * 8), "ms_per_step": t_e2e * 1e3,
                "ms_per_step_mean": t_e2e_mean * 1e3, "timing": f"median of {e2e_steps} host-timed calls",
                "max_rel_err_vs_closed_form": e2e_err},
        "roofline": roofline,
    }
    if not args.no_forms and args.precision == "fp64":
        out["forms"] = measure_forms(sp, f, u_exact, u, N, n, dev, ms_step, args)
    if not args.no_batched and args.precision == "fp64":
        del f_host, u_host, dbuf
        out["batched"] = measure_batched(sp, dev, args, rank, world)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(f.cpu().numpy(), budget_s=args.cpu_budget)
    if rank == 0 and not args.no_cpu_fast:
        out["cpu_fft_thomas"] = cpu_fft_thomas(f.cpu().numpy(), u.cpu().numpy())
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


FORM_GROUPS = ("precision", "adjoint", "inverse_fit", "transforms", "tangential_gradient", "vector_calculus",
               "lowrank", "mixed_sizes", "paper_scale", "poles")


def measure_forms(sp, f, u_exact, u64, N, n, dev, ms_fp64, args):
    """The reduced-precision forms on the same input and device, timed the same
    way, with their error against the FP64 solution and the closed form."""
    import torch

    ex = float(u_exact.abs().max())
    res = {}
    steps = max(5, min(args.steps, 50))
    want = set(args.forms.split(",")) if args.forms else set(FORM_GROUPS)
    for prec, sweeps in [("fp32", 0), ("fp32_refine", 0), ("fp32_refine", 1), ("fp32_refine", 2)]:
        if "precision" not in want:
            break
        plan = sp.Plan(N, n, prec, sweeps, device=dev, autotune=not args.no_autotune)
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
        u = torch.empty_like(f)
        for _ in range(3):
            plan.solve(f, u, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            plan.solve(f, u, ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        key = prec if prec == "fp32" else f"{prec}_sweeps{sweeps}"
        res[key] = {"value": N * n / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms,
                    "speedup_vs_fp64": ms_fp64 / ms,
                    "max_rel_err_vs_fp64": float((u - u64).abs().max()) / ex,
                    "max_rel_err_vs_closed_form": float((u - u_exact).abs().max()) / ex,
                    "gpu_launches_per_step": plan.launches()}
        del plan, ws
    # the adjoint (the transposed solve behind autograd): FP64 and FP32, checked by
    # the dot-product identity <S f, g> = <f, S^T g> with g = the exact solution
    g = u_exact
    sg64 = None
    for prec in ("fp64", "fp32"):
        if "adjoint" not in want:
            break
        plan = sp.Plan(N, n, prec, 0, device=dev, autotune=not args.no_autotune)
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
        out = torch.empty_like(f)
        for _ in range(3):
            plan.solve_adjoint(g, out, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            plan.solve_adjoint(g, out, ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        sf = plan.solve(f)
        lhs, rhs = float((sf * g).sum()), float((f * out).sum())
        entry = {"value": N * n / (ms * 1e-3), "unit": "DOF/s", "ms_per_step": ms,
                 "dot_product_identity_rel_err": abs(lhs - rhs) / max(abs(lhs), 1e-300),
                 "gpu_launches_per_step": plan.launches(adjoint=True)}
        if prec == "fp64":
            sg64 = out.clone()
        else:
            entry["max_rel_err_vs_fp64_adjoint"] = float((out - sg64).abs().max() / sg64.abs().max())
        res[f"adjoint_{prec}"] = entry
        del plan, ws, out, sf
    if "inverse_fit" in want:
        res["inverse_fit"] = measure_inverse_fit(sp, dev, steps, args)
    if "transforms" in want:
        res["transforms"] = measure_transforms(sp, f, N, n, dev, steps, args)
    if "tangential_gradient" in want:
        res["tangential_gradient"] = measure_tangential(sp, f, N, n, dev, steps, args)
    if "vector_calculus" in want:
        res["vector_calculus"] = measure_vector_calculus(sp, N, n, dev, steps, args)
    if "lowrank" in want:
        res["lowrank"] = measure_lowrank(sp, N, n, dev, steps, ms_fp64, args)
    if "mixed_sizes" in want:
        res["mixed_sizes"] = measure_mixed_sizes(sp, dev, args)
    if "paper_scale" in want and not args.no_paper_scale:
        res["paper_scale"] = measure_paper_scale(sp, dev, args)
    if "poles" in want:
        res["poles"] = measure_poles(sp, N, n, dev, steps, ms_fp64, args)
    return res


def measure_poles(sp, N, n, dev, steps, ms_fp64, args):
    """The FP64 solve on the grid with both poles (n_theta + 1 rows theta_i =
    i pi / n_theta) for the same series and grid size, against the closed form
    on every row; its colatitude transforms have length 2 n_theta."""
    import torch
    from synth import sh

    w = sh.workload(args.workload)
    c = w.coeffs()
    f = sh.synthesize(c, N, n, device=dev, grid="poles")
    ue = sh.synthesize(sh.poisson_exact(c), N, n, device=dev, grid="poles")
    plan = sp.Plan(N, n, "fp64", device=dev, autotune=not args.no_autotune, grid="poles")
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
    u = torch.empty_like(f)
    for _ in range(3):
        plan.solve(f, u, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        plan.solve(f, u, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rows = N + 1
    out = {"grid": f"{rows} x {n} (theta_i = i pi / {N}, both poles)", "value": rows * n / (ms * 1e-3),
           "unit": "DOF/s", "ms_per_step": ms, "ms_vs_pole_free_fp64": ms / ms_fp64,
           "max_rel_err_vs_closed_form": float((u - ue).abs().max() / ue.abs().max()),
           "gpu_launches_per_step": plan.launches()}
    del plan, ws, u, f, ue
    return out


def measure_lowrank(sp, N, n, dev, steps, ms_fp64, args):
    """The low-rank form on the paper's Section 5 right-hand side sin(50 xyz) at
    the bench grid: the structure-preserving GE (timed once, it synchronises per
    step) and the solve from the factors, against the dense FP64 solve of the
    same f."""
    import torch
    from synth import sh

    th = torch.tensor(sh.colatitudes(N), device=dev)[:, None]
    la = torch.tensor(sh.longitudes(n), device=dev)[None, :]
    f = torch.sin(50 * (torch.cos(la) * torch.sin(th)) * (torch.sin(la) * torch.sin(th)) * torch.cos(th))
    f = f.contiguous()
    plan = sp.Plan(N, n, device=dev, autotune=not args.no_autotune)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cols, piv, rows = plan.lowrank_ge(f, max_terms=min(256, N))
    t_ge = time.perf_counter() - t0
    rank = sum(int(abs(a + b) > 0) + int(abs(a - b) > 0) for a, b in piv.cpu().tolist())
    u = torch.empty_like(f)
    for _ in range(2):
        plan.solve_lowrank(cols, piv, rows, u)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(steps, 10))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        plan.solve_lowrank(cols, piv, rows, u)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    ud = plan.solve(f)
    return {"value": N * n / (ms * 1e-3), "unit": "DOF/s", "ms_per_solve": ms,
            "case": "f = sin(50 xyz) (the paper's Section 5 example) on the bench grid",
            "ge_terms": int(cols.shape[0]), "rank": rank, "ge_seconds": t_ge,
            "speedup_vs_dense_fp64_solve": ms_fp64 / ms,
            "max_rel_err_vs_dense_fp64_solve": float((u - ud).abs().max() / ud.abs().max()),
            "gpu_launches_per_solve": 3 + 1 + 3}


def measure_tangential(sp, f, N, n, dev, steps, args):
    """The surface gradient (Section 4, Differentiation) of the bench input, timed;
    accuracy from a polynomial with a closed-form tangential gradient on the same
    grid (grad f - (r . grad f) r)."""
    import torch
    from synth import sh

    plan = sp.Plan(N, n, device=dev, autotune=not args.no_autotune)
    ws = torch.empty(plan.gradient_workspace_bytes(), dtype=torch.uint8, device=dev)
    out = tuple(torch.empty_like(f) for _ in range(3))
    for _ in range(2):
        plan.tangential_gradient(f, out, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(3, min(steps, 10))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        plan.tangential_gradient(f, out, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    th = torch.tensor(sh.colatitudes(N), device=dev)[:, None]
    la = torch.tensor(sh.longitudes(n), device=dev)[None, :]
    x, y, z = torch.cos(la) * torch.sin(th), torch.sin(la) * torch.sin(th), torch.cos(th) + 0 * la
    p = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
    px = 1 + 2 * x * y + 4 * x ** 3 + 2 * x * (y * z) ** 2
    py = 2 * y + x ** 2 + 5 * y ** 4 + 2 * y * (x * z) ** 2
    pz = 2 * z * (x * y) ** 2
    rd = x * px + y * py + z * pz
    g = plan.tangential_gradient(p.contiguous(), out, ws)
    errs = [float((gi - (pi - rd * ri)).abs().max() / (pi - rd * ri).abs().max())
            for gi, pi, ri in zip(g, (px, py, pz), (x, y, z))]
    return {"value": N * n / (ms * 1e-3), "unit": "DOF/s", "ms_per_call": ms,
            "outputs": "d^t f/dx, d^t f/dy, d^t f/dz on the grid",
            "max_rel_err_vs_closed_form_xyz": errs,
            "closed_form_case": "1 + x + y^2 + x^2 y + x^4 + y^5 + (xyz)^2",
            "gpu_launches_per_call": 2 + 3 + 1 + 3 * 2}


def measure_transforms(sp, f, N, n, dev, steps, args):
    """The transforms alone (Section 4): coeffs2, sample and sum2 of the bench
    input, each timed; accuracy from the paper's worked example
    p = 1 + x + y^2 + x^2 y + x^4 + y^5 + (xyz)^2 on the same grid: the round trip
    sample(coeffs2(p)) = p (p is band-limited far inside the grid; the bench
    series carries ~1e-9 of synthesis rounding in its theta-Nyquist mode, which
    coeffs2 drops) and sum2(p) against its integral 216 pi/35."""
    import torch
    from synth import sh

    plan = sp.Plan(N, n, device=dev, autotune=not args.no_autotune)
    X = plan.coeffs2(f)
    calls = {"coeffs2": lambda: plan.coeffs2(f), "sample": lambda: plan.sample(X), "sum2": lambda: plan.sum2(f)}
    reps = max(3, min(steps, 10))
    out = {}
    for name, call in calls.items():
        for _ in range(2):
            call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name] = {"ms_per_call": ms, "value": N * n / (ms * 1e-3)}
    th = torch.tensor(sh.colatitudes(N), device=dev)[:, None]
    la = torch.tensor(sh.longitudes(n), device=dev)[None, :]
    x, y, z = torch.cos(la) * torch.sin(th), torch.sin(la) * torch.sin(th), torch.cos(th) + 0 * la
    p = (1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2).contiguous()
    rt = float((plan.sample(plan.coeffs2(p)) - p).abs().max() / p.abs().max())
    exact = 216 * math.pi / 35
    return {"unit": "DOF/s", "calls": out, "max_rel_err_sample_coeffs2_roundtrip": rt,
            "sum2_worked_example_abs_err": abs(plan.sum2(p) - exact),
            "gpu_launches_per_call": {"coeffs2": 2, "sample": 2, "sum2": 3}}


def measure_inverse_fit(sp, dev, steps, args):
    """The differentiation form on its workload (512 x 1024, u_obs a seeded l <= 200
    series plus N(0, 1e-3) noise): one gradient of ||u(f) - u_obs||^2 through the
    autograd function (forward solve, loss, adjoint solve), timed in FP64 and FP32;
    the FP64 gradient checked against a central difference (h = 1e-6) along a
    random direction and the FP32 one against it."""
    import numpy as np
    import torch
    from synth import sh

    w = sh.workload("sh200_512x1024_noisy")
    u_obs = w.observation(device=dev)
    f0 = torch.tensor(np.random.default_rng(55).standard_normal((w.n_theta, w.n_lambda)) * 0.1, device=dev)
    reps = max(5, min(steps, 50))
    res = {"workload": w.name, "unit": "DOF/s"}
    grads = {}
    for prec in ("fp64", "fp32"):
        def gradient():
            f = f0.clone().requires_grad_(True)
            loss = ((sp.poisson(f, prec) - u_obs) ** 2).sum()
            loss.backward()
            return f.grad
        for _ in range(3):
            gradient()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            gradient()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        grads[prec] = gradient()
        res[prec] = {"ms_per_gradient": ms, "value": w.n_theta * w.n_lambda / (ms * 1e-3)}
    plan = sp.get_plan(w.n_theta, w.n_lambda, device=dev)
    d = torch.tensor(np.random.default_rng(7).standard_normal(tuple(f0.shape)), device=dev)
    loss = lambda x: float(((plan.solve(x) - u_obs) ** 2).sum())
    h = 1e-6
    fd = (loss(f0 + h * d) - loss(f0 - h * d)) / (2 * h)
    res["fp64"]["central_difference_rel_err"] = abs(fd - float((grads["fp64"] * d).sum())) / max(1.0, abs(fd))
    res["fp32"]["max_rel_err_vs_fp64_gradient"] = float((grads["fp32"] - grads["fp64"]).abs().max()
                                                        / grads["fp64"].abs().max())
    return res


def measure_vector_calculus(sp, N, n, dev, steps, args):
    """Divergence, curl, curl of a scalar function and vorticity (Section 4) on the
    paper's Rossby-Haurwitz stream function psi = cos(theta) + sin^4(theta)
    cos(theta) cos(4 lambda) at the bench size, each timed; accuracy: the
    vorticity of curl(psi) against the Laplacian of psi, and div curl(psi) = 0."""
    import torch
    from synth import sh

    plan = sp.Plan(N, n, device=dev, autotune=not args.no_autotune)
    ws = torch.empty(plan.curl_workspace_bytes(), dtype=torch.uint8, device=dev)
    th = torch.tensor(sh.colatitudes(N), device=dev)[:, None]
    la = torch.tensor(sh.longitudes(n), device=dev)[None, :]
    x, y, z = torch.cos(la) * torch.sin(th), torch.sin(la) * torch.sin(th), torch.cos(th) + 0 * la
    q = x ** 4 - 6 * x ** 2 * y ** 2 + y ** 4
    psi = (z + z * q).contiguous()
    lap = -2 * z - 30 * z * q
    del x, y, th, la
    u = tuple(torch.empty_like(psi) for _ in range(3))
    c = tuple(torch.empty_like(psi) for _ in range(3))
    s = torch.empty_like(psi)
    calls = {
        "scalar_curl": lambda: plan.scalar_curl(psi, u, ws),
        "divergence": lambda: plan.divergence(*u, s, ws),
        "curl": lambda: plan.curl(*u, c, ws),
        "vorticity": lambda: plan.vorticity(*u, s, ws),
    }
    reps = max(3, min(steps, 5))
    out = {}
    for name, call in calls.items():
        for _ in range(2):
            call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            call()
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"ms_per_call": e0.elapsed_time(e1) / reps}
    chained = {}
    for rtol in (0.0, 1e-14):
        plan.set_chop(rtol)
        plan.scalar_curl(psi, u, ws)
        zeta = plan.vorticity(*u, s, ws)
        err_vort = float((zeta - lap).abs().max() / lap.abs().max())
        div = plan.divergence(*u, c[0], ws)
        scale = max(float(ui.abs().max()) for ui in u)
        chained[f"chop_{rtol:g}"] = {"max_rel_err_vort_u_vs_laplacian_psi": err_vort,
                                     "max_div_u_rel": float(div.abs().max()) / scale}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        plan.vorticity(*u, s, ws)
    e1.record()
    torch.cuda.synchronize()
    out["vorticity_chop_1e-14"] = {"ms_per_call": e0.elapsed_time(e1) / reps}
    plan.set_chop(0.0)
    return {"unit": "DOF/s", "calls": out,
            "value_vorticity": N * n / (out["vorticity"]["ms_per_call"] * 1e-3),
            "case": "psi = cos(theta) + sin^4(theta) cos(theta) cos(4 lambda); u = n x grad psi",
            "chained_vort_of_curl": chained,
            "gpu_launches_per_call": {"scalar_curl": 13, "divergence": 17, "curl": 24, "vorticity": 25,
                                      "extra_per_input_with_chop": 2}}


def measure_paper_scale(sp, dev, args):
    """The paper's headline size: m = n with mn/2 = 1.03e8 unknowns (7168 x 14336),
    FP64 and FP32+refinement (1 sweep), against the paper's ~1 minute on a laptop."""
    import torch
    from synth import sh

    w = sh.workload("sh2000_7168x14336")
    f, ue = w.make(device=dev)
    ex = float(ue.abs().max())
    out = {"workload": f"{w.name}: n_theta={w.n_theta} x n_lambda={w.n_lambda}, DOF (mn/2) = "
                       f"{w.n_theta * w.n_lambda}", "paper_seconds_context": 60.0}
    for prec, sweeps in [("fp64", 0), ("fp32_refine", 1)]:
        plan = sp.Plan(w.n_theta, w.n_lambda, prec, sweeps, device=dev, autotune=not args.no_autotune)
        ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
        u = torch.empty_like(f)
        for _ in range(2):
            plan.solve(f, u, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(5):
            plan.solve(f, u, ws)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        out[prec] = {"ms_per_solve": ms, "value": w.n_theta * w.n_lambda / (ms * 1e-3), "unit": "DOF/s",
                     "max_rel_err_vs_closed_form": float((u - ue).abs().max()) / ex}
        del plan, ws, u
    return out


def measure_mixed_sizes(sp, dev, args):
    """The mixed-precision workloads at 2048 x 4096 and 4096 x 8192: FP64, FP32 and
    FP32 + refinement with 1, 2 and 3 sweeps, each timed, with the error of each
    against the FP64 solution (itself within 1e-12 of the oracle) and against
    the closed form of the series, per sweep."""
    import torch
    from synth import sh

    out = {}
    for name in ("sh1024_2048x4096", "sh2048_4096x8192"):
        w = sh.workload(name)
        f, ue = w.make(device=dev)
        ex = float(ue.abs().max())
        entry = {"n_theta": w.n_theta, "n_lambda": w.n_lambda, "unit": "DOF/s"}
        u64 = None
        for prec, sweeps in [("fp64", 0), ("fp32", 0), ("fp32_refine", 1), ("fp32_refine", 2), ("fp32_refine", 3)]:
            plan = sp.Plan(w.n_theta, w.n_lambda, prec, sweeps, device=dev, autotune=not args.no_autotune)
            ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
            u = torch.empty_like(f)
            for _ in range(3):
                plan.solve(f, u, ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(10):
                plan.solve(f, u, ws)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 10
            key = prec if prec != "fp32_refine" else f"fp32_refine_sweeps{sweeps}"
            r = {"ms_per_solve": ms, "value": w.n_theta * w.n_lambda / (ms * 1e-3),
                 "max_rel_err_vs_closed_form": float((u - ue).abs().max()) / ex}
            if u64 is None:
                u64 = u.clone()
            else:
                r["max_rel_err_vs_fp64"] = float((u - u64).abs().max()) / ex
            entry[key] = r
            del plan, ws, u
        out[name] = entry
        del f, ue, u64
    return out


def measure_batched(sp, dev, args, rank: int = 0, world: int = 1):
    """4096 spheres of uneven resolution (n_theta = 16 s, s uniform in 2..32,
    n_lambda = 2 n_theta, SH series l <= n_theta/2) in persistent launches (one per radix group)
    with autotuned tiles, against the same problems solved one by one with
    single-problem FP64 plans; then the same batch in FP32 + refinement.
    With several ranks the problems are split by shard_lpt (no collective on the
    data path: each rank solves its shard in its own launch); the batch's time
    is the slowest rank's and the value counts every rank's problems."""
    import tempfile

    import torch
    from synth import sh

    if "SPHERE_POISSON_TUNE_CACHE" not in os.environ:
        os.environ["SPHERE_POISSON_TUNE_CACHE"] = os.path.join(tempfile.gettempdir(), "sphere_poisson_tune.txt")
    t0 = time.perf_counter()
    sizes, fs, us = sh.batched_workload(args.batch_count, device=dev)
    t_gen = time.perf_counter() - t0
    total_dof = sum(a * b for a, b in sizes)
    total_problems = len(sizes)
    if world > 1:
        mine = shard_lpt(sizes, world)[rank]
        sizes = [sizes[b] for b in mine]
        fs = [fs[b] for b in mine]
        us = [us[b] for b in mine]
    t0 = time.perf_counter()
    plan = sp.BatchedPlan(sizes, autotune=True, device=dev)
    t_plan = time.perf_counter() - t0
    f = plan.pack(fs)
    ue = plan.pack(us)
    del fs, us
    u = torch.empty_like(f)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device=dev)
    for _ in range(2):
        plan.solve(f, u, ws)
    reps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
    e0.record()
    for _ in range(reps):
        plan.solve(f, u, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)
    # error per problem against the closed form, worst case
    worst = 0.0
    for b in range(len(sizes)):
        a, c = plan.offsets[b], plan.offsets[b + 1]
        worst = max(worst, float((u[a:c] - ue[a:c]).abs().max() / ue[a:c].abs().max()))
    worst = max_over_ranks(worst, world, dev)
    # plain FP64: one single-problem plan per size, problems solved one by one
    singles = {sz: sp.Plan(sz[0], sz[1], device=dev, autotune=not args.no_autotune) for sz in set(sizes)}
    outs = [torch.empty(sz, dtype=torch.float64, device=dev) for sz in sizes]
    views = plan.unpack(f)
    for b, sz in enumerate(sizes[:64]):
        singles[sz].solve(views[b], outs[b])
    torch.cuda.synchronize()
    e0.record()
    for b, sz in enumerate(sizes):
        singles[sz].solve(views[b], outs[b])
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    dof = total_dof
    ms_plain = max_over_ranks(ms_plain, world, dev)
    del outs, views, singles
    out = {"value": dof / (ms * 1e-3), "unit": "DOF/s", "ms_per_batch": ms, "problems": total_problems,
           "dof_per_batch": dof, "distinct_sizes": len(set(sizes)), "gpu_launches_per_batch": plan.launches(),
           "plain_fp64_loop_ms": ms_plain, "speedup_vs_plain_fp64_loop": ms_plain / ms,
           "max_rel_err_vs_closed_form": worst, "autotuned": True, "plan_seconds": t_plan,
           "input_generation_seconds": t_gen,
           "sharding": (f"{world} ranks, longest-processing-time split by n_theta*n_lambda, no collective "
                        f"on the data path; this rank {len(sizes)} problems, {plan.offsets[-1]} DOF"
                        if world > 1 else "single GPU")}

    # the same batch in FP32 + refinement (one sweep), the same launches
    sweeps = 1
    t0 = time.perf_counter()
    rplan = sp.BatchedPlan(sizes, precision="fp32_refine", refine_sweeps=sweeps, autotune=True, device=dev)
    t_rplan = time.perf_counter() - t0
    del ws
    rws = torch.empty(rplan.workspace_bytes, dtype=torch.uint8, device=dev)
    ur = torch.empty_like(f)
    for _ in range(2):
        rplan.solve(f, ur, rws)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record()
    for _ in range(reps):
        rplan.solve(f, ur, rws)
    e1.record()
    torch.cuda.synchronize()
    ms_r = max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)
    worst_r = worst_r64 = 0.0
    for b in range(len(sizes)):
        a, c = plan.offsets[b], plan.offsets[b + 1]
        worst_r = max(worst_r, float((ur[a:c] - ue[a:c]).abs().max() / ue[a:c].abs().max()))
        worst_r64 = max(worst_r64, float((ur[a:c] - u[a:c]).abs().max() / u[a:c].abs().max()))
    worst_r = max_over_ranks(worst_r, world, dev)
    worst_r64 = max_over_ranks(worst_r64, world, dev)
    out["fp32_refine"] = {"value": dof / (ms_r * 1e-3), "unit": "DOF/s", "ms_per_batch": ms_r,
                          "refine_sweeps": sweeps, "speedup_vs_batched_fp64": ms / ms_r,
                          "max_rel_err_vs_batched_fp64": worst_r64, "max_rel_err_vs_closed_form": worst_r,
                          "gpu_launches_per_batch": rplan.launches(), "autotuned": True,
                          "plan_seconds": t_rplan}
    return out


def _host_threads() -> int:
    """Threads the oracle's numpy / LAPACK calls run on: the BLAS pool's size
    where threadpoolctl can read it, else the CPUs this process may run on."""
    try:
        from threadpoolctl import threadpool_info

        n = [i["num_threads"] for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_sample(f_np, ks):
    """Time the oracle's sampled-column solve on wavenumbers ks of the full input."""
    from oracle import sphere_oracle as O

    t0 = time.perf_counter()
    O.sampled_columns(f_np, ks)
    return time.perf_counter() - t0


def cpu_baseline(f_np, budget_s: float = 20.0, ks=None) -> dict:
    """The CPU oracle as it stands, on the host cores, on a bounded sample of the
    same workload: its sampled-column mode solves a few wavenumbers k of the
    full-size input (each needs the full DFT of the input at that k, the full
    colatitude DFT, a banded solve and the inverse); the time per wavenumber,
    times the n_lambda wavenumbers the oracle's full solve computes, gives DOF/s."""
    nt, nl = f_np.shape
    if ks is None:
        ks = [0, 1, 2, 7, 50, 333, 1001, 2500]
    t_warm = _oracle_sample(f_np, [5])          # builds the oracle's cached phase matrix
    t = 0.0
    used = []
    for k in ks:
        t += _oracle_sample(f_np, [k])
        used.append(k)
        if t > budget_s:
            break
    per_k = t / len(used)
    full = per_k * nl
    return {"value": nt * nl / full, "unit": "DOF/s", "cores": _host_threads(), "kind": "oracle",
            "sample": f"oracle.sampled_columns on {len(used)} of the {nl} wavenumbers of the "
                      f"{nt}x{nl} input, one call each ({t:.1f} s; a first call building the cached "
                      f"colatitude phase matrix took {t_warm:.1f} s and is not counted), "
                      f"scaled by {nl}/{len(used)}"}


def cpu_fft_thomas(f_np, u_gpu) -> dict:
    """A full CPU solve of the same input by the paper's algorithm as a plain
    CPU program (baseline/fft_thomas.py: scipy.fft transforms, numpy Thomas
    eliminations), timed once on one core and once with the FFTs on every host
    core: measured whole solves, not extrapolated."""
    from baseline import fft_thomas

    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    nt, nl = f_np.shape
    times = {}
    u = None
    for workers in (1, cores):
        t0 = time.perf_counter()
        u = fft_thomas.solve(f_np, workers=workers)
        times[workers] = time.perf_counter() - t0
    diff = float(abs(u - u_gpu).max() / abs(u_gpu).max())
    return {"kind": "fft+thomas", "unit": "DOF/s", "dof_per_solve": nt * nl,
            "value_1_core": nt * nl / times[1], "seconds_1_core": times[1],
            "value_all_cores": nt * nl / times[cores], "seconds_all_cores": times[cores], "cores": cores,
            "sample": f"one full {nt}x{nl} solve per core count (scipy.fft with workers=1 and "
                      f"workers={cores}; the eliminations run on one thread in both)",
            "max_rel_diff_vs_gpu_solution": diff}


def run_reference(args):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    import torch  # noqa: F401
    from synth import sh

    w = sh.workload(args.workload)
    f, _ = w.make(device="cuda" if _cuda_ok() else "cpu")
    f_np = f.cpu().numpy()
    ks_all = list(range(0, w.n_lambda // 2))
    for s in range(args.warmup):
        _oracle_sample(f_np, [ks_all[(7 * s) % len(ks_all)]])
    times = []
    for s in range(args.steps):
        k = ks_all[(131 * s + 3) % len(ks_all)]
        times.append(_oracle_sample(f_np, [k]))
    per_k = sum(times) / len(times)
    full = per_k * w.n_lambda
    value = w.n_theta * w.n_lambda / full
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "DOF/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": full * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic: seeded spherical-harmonic series (no dataset)",
        "config": {"workload": f"{w.name}: CPU FP64 oracle on the same input",
                   "dof_per_solve": w.n_theta * w.n_lambda},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": _host_threads(), "kind": "oracle",
                         "sample": f"each step: oracle.sampled_columns on 1 of the {w.n_lambda} "
                                   f"wavenumbers, scaled by {w.n_lambda}"},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def _cuda_ok():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-fast", action="store_true", help="skip the full CPU FFT + Thomas solves")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--forms", default="",
                    help="comma-separated subset of the forms to measure: " + ",".join(FORM_GROUPS))
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-paper-scale", action="store_true")
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32_refine"])
    ap.add_argument("--sweeps", type=int, default=1)
    ap.add_argument("--no-autotune", action="store_true", help="plan-time tile tuning off (default tiles)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
