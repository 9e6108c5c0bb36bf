"""Benchmark of the GMCP contact pass on one B300 (or N independent replicas).

A step is one full contact pass (ipc_contact_pass) through the C ABI on the
gel-on-terrain workload (256x256-quad gel pad, 131,072 slave triangles x 16 face samples =
2,097,152 samples, against a 199,712-triangle Perlin terrain, dhat = 5e-5 m),
mixed precision (FP32 barrier, FP64 distance anchors and CCD):
  broad phase, samples, energy, gradient, BSR Hessian (as ipc_barrier_eval)
  linearised-gap bound and additive CCD for a step dx (as ipc_ccd_max_step)
The pad state is the terrain pressed 0.15 mm deep (scenes.drape_on_master);
dx is a seeded downward press of 5 um x U[0.5, 1.5] per vertex plus 1 um
tangential noise.  Inputs stay resident in HBM; L2 (126 MB) is flushed by
writing a 256 MB buffer between timed steps, outside the timed region.

metric = contact samples per second, samples per pass = face samples
(n_slave_tris x 16) + 2 x edge candidates + point candidates.

``--impl reference`` times the FP64 CPU oracle (the correctness reference,
single-threaded) on a bounded window of the same workload (half-width 2 mm
around the highest terrain peak) with the same metric.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "contact samples/s (barrier E+grad+H+CCD)"
UNIT = "samples/s"
WORKLOAD = "gel_on_terrain 256x256 pad (131,072 slave tris x 16 samples) vs 199,712-tri Perlin terrain, pressed 0.15 mm"
CROP_HALF_WIDTH = 2.0e-3
CLOCK_WINDOW_S = 1.5      # sustained run of the same step that the clock record also covers


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def make_workload(seed=11):
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain()
    x = S.drape_on_master(sc, 0.15e-3)
    rng = np.random.default_rng(seed)
    dx = np.zeros_like(x)
    dx[:, 2] = -5e-6 * (0.5 + rng.random(x.shape[0]))
    dx[:, :2] = 1e-6 * rng.normal(size=(x.shape[0], 2))
    return sc, x, dx


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n_gpus, backend="nccl"):
    """One process per GPU (torchrun sets RANK / WORLD_SIZE / MASTER_*):
    every rank runs an independent replica of the workload (the benchmark
    workload is one environment and does not shard); only the timing is
    reduced across ranks.  backend "gloo" serves the CPU tests."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend=backend)
        return rank, world, dist
    return 0, 1, None


def max_over_ranks(v, dist):
    """The slowest rank's value (the whole job ends with it)."""
    if dist is None:
        return v
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step, steps, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank has the same per-step work)."""
    return units_per_step * steps * world / seconds


def barrier(dist):
    if dist is not None:
        dist.barrier()


def samples_per_pass(ctx, x, xm, nk):
    c = ctx.candidates(x, xm)
    return ctx.ns * nk + 2 * c["edge"] + c["point"], c


def measure_alu_peaks(dev):
    """FP32 and FP64 FMA rates of this GPU (ipc_alu_peak: chains of fused
    multiply-adds on every SM, CUDA events), TFLOP/s; the best of three."""
    from paper_2605_24339_b300 import binding
    return {"fp32_tflops": max(binding.alu_peak(0, dev) for _ in range(3)),
            "fp64_tflops": max(binding.alu_peak(1, dev) for _ in range(3)),
            "how": "ipc_alu_peak: 16 independent FMA chains per thread, 8 blocks of 256 per SM, "
                   "CUDA events, best of 3 (1 FMA = 2 flops)"}


def pass_bytes(sc, ctx, nnzb):
    """Algorithmic bytes of one contact pass, per unit of work (what the
    method must move; each read or written once):
      slave surface vertices: current and rest positions (FP64, 48 B) and the
        step's displacement (FP64, 24 B); gradient row written (FP32, 12 B)
      slave triangles: indices (12 B)
      master vertices: current and rest positions (FP64, 48 B)
      master triangles: indices (12 B)
      surface Hessian blocks of the BSR written (FP32 3x3, 36 B)."""
    n_sv = ctx.slave_vertices().shape[0]
    parts = {"slave_verts": n_sv * (48 + 24 + 12), "slave_tris": sc.stris.shape[0] * 12,
             "master_verts": sc.Y0.shape[0] * 48, "master_tris": sc.mtris.shape[0] * 12,
             "bsr_blocks": int(nnzb) * 36}
    return sum(parts.values()), parts


def time_steps(step, stream, steps, flush):
    """CUDA-event time of each step on the launching stream, L2 flushed
    (a 256 MB write) before every step, outside the events."""
    import torch
    ms = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        info = step()
        ev1.record(stream)
        ev1.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    return ms, info


def sustain(step, flush, seconds):
    """The same step, flush included, repeated for about ``seconds`` (the
    clock sampler's window beside the short timed region)."""
    import torch
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds:
        flush.zero_()
        step()
        n += 1
        if n % 64 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    return n


def sections(ctx, step, flush, n):
    """Per-section device times (ipc_profile: CUDA events around each group
    of launches; the profiled passes run without the CUDA graph)."""
    import torch
    ctx.profile_start()
    for _ in range(n):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.profile_stop()
    prof = ctx.profile_read()
    return {k: v["ms"] / max(v["calls"], 1) for k, v in prof.items()}


def run_ours(args):
    import torch
    from paper_2605_24339_b300 import binding
    rank, world, dist = dist_setup(args.gpus)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    alu = measure_alu_peaks(dev)
    sc, x_np, dx_np = make_workload(seed=11 + rank)
    nk = 4 ** sc.params["face_rule_level"]
    stream = torch.cuda.current_stream()
    ctx = binding.Context(sc, precision=args.precision, device=dev, stream=stream)
    x = torch.as_tensor(x_np, device="cuda")
    dx = torch.as_tensor(dx_np, device="cuda")
    xm = torch.as_tensor(sc.Y0, device="cuda")
    grad = torch.empty((sc.X.shape[0], 3), device="cuda",
                       dtype=torch.float32 if args.precision == "mixed" else torch.float64)
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    units, cand = samples_per_pass(ctx, x, xm, nk)
    first = ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=True)
    counts_once, nnzb = first["counts"], first["hess"].nnzb
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        return ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=False, energy_dev=e_dev,
                                grad_out=grad)

    # launch shapes by the autotuner (results do not depend on them)
    tune_s, tune_q, tune_ms = ctx.autotune(x, xm, dx, reps=3)
    for _ in range(args.warmup):
        info = step()
    torch.cuda.synchronize()
    kernels_per_pass = ctx.pass_kernels()
    clocks = ClockSampler(dev)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    step_ms, info = time_steps(step, stream, args.steps, flush)
    torch.cuda.synchronize()
    barrier(dist)
    n_sustain = sustain(step, flush, CLOCK_WINDOW_S)
    clk = clocks.stop()
    clk["window"] = (f"the {args.steps} timed steps and {n_sustain} more of the same step "
                     f"({CLOCK_WINDOW_S} s)")
    sec_ms = sections(ctx, step, flush, min(max(args.steps, 20), 100))
    total_ms = max_over_ranks(sum(step_ms), dist)
    ms_step = total_ms / args.steps
    value = job_throughput(units, args.steps, world, total_ms / 1e3)

    # end to end: the pass's per-step inputs from the pad, the positions and
    # displacements of the slave surface vertices (the only pad vertices the
    # pass reads), in pinned host memory, through ipc_contact_pass_host (it
    # copies them in, the displacements behind the broad phase, and scatters
    # them into the device arrays); energy and alpha read back; every step
    svert = ctx.slave_vertices()
    xs_host = torch.as_tensor(np.ascontiguousarray(x_np[svert])).pin_memory()
    dxs_host = torch.as_tensor(np.ascontiguousarray(dx_np[svert])).pin_memory()
    out_host = np.zeros(2)   # the step's results on the host
    x_e2e = torch.zeros_like(x)
    dx_e2e = torch.zeros_like(dx)

    def e2e_step():   # energy and alpha come back in the call's own synchronisation
        info = ctx.contact_pass_host(xs_host, dxs_host, x_e2e, dx_e2e, xm, grad=True, hess="view", counts=False,
                                     grad_out=grad)
        out_host[0] = info["energy"]
        out_host[1] = info["alpha"]

    for _ in range(max(1, args.warmup)):   # the first call captures the pass with its copies
        e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
    e2e_value = job_throughput(units, args.steps, world, e2e_s)
    e2e_h2d = int(xs_host.numel() * 8 + dxs_host.numel() * 8)

    if rank != 0:
        return
    peaks, peak_kind = load_peaks()
    alg_b, alg_parts = pass_bytes(sc, ctx, nnzb)
    ctx.close()
    dominant = max(sec_ms, key=sec_ms.get)
    gbs = alg_b / (ms_step * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.precision, "samples_per_pass": int(units),
                   "face_samples": int(sc.stris.shape[0] * nk), "edge_candidates": cand["edge"],
                   "point_candidates": cand["point"], "face_candidates": cand["face"],
                   "active_samples": {k: int(counts_once[k]) for k in ("face", "edge", "point")},
                   "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}",
                   "cuda_graph": True, "autotuned_blocks_per_sm": {"samples": tune_s, "query": tune_q}},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_h2d,
                "d2h_bytes_per_step": 16},
        "gpu_launches": kernels_per_pass * args.steps if kernels_per_pass > 0 else None,
        "kernels_per_pass": kernels_per_pass,
        "roofline": {"bound": "hbm", "kernel": f"contact pass (one CUDA graph of {kernels_per_pass} kernels)",
                     "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                     "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)",
                     "algorithmic_bytes_per_pass": alg_b, "bytes_by_part": alg_parts,
                     "launch_ms": ms_step,
                     "dominant_section": {"name": dominant, "ms": sec_ms[dominant],
                                          "share": sec_ms[dominant] / sum(sec_ms.values())},
                     "note": "the pass is latency-bound at this size (its algorithmic bytes are L2-resident); "
                             "the contact-dense line (key dense) and the batch carry the HBM-scale cases"},
        "alu_peaks": alu,
        "sections_ms": {k: round(v, 4) for k, v in sec_ms.items()},
        "alpha": info["alpha"],
        "clocks": clk,
    }
    if not args.no_dense:
        line["dense"] = dense_measurement(dev, alu, steps=max(args.steps, 10))
    if not args.no_batch:
        line["batched"] = batched_measurement(dev, n_env=args.batch_envs)
    if not args.no_newton:
        line["newton_step"] = newton_measurement(dev)
        line["config1_indent"] = config1_measurement(dev)
        line["ccd_stress"] = ccd_stress_measurement(dev)
        line["batched_step"] = batched_step_measurement(dev, n_env=args.step_envs, steps=10)
        if args.big_step_envs > 0:
            # the batched workload's full environment count, stepped: one tet layer per pad, since
            # two layers need ~320 GB at 512 environments (42.8 GB measured at 64)
            import torch
            torch.cuda.empty_cache()
            free_gb = torch.cuda.mem_get_info()[0] / 1e9
            if free_gb >= 230:
                line["batched_step_full"] = batched_step_measurement(dev, n_env=args.big_step_envs, steps=10,
                                                                     layers=1)
            else:
                line["batched_step_full"] = {"skipped": f"{free_gb:.0f} GB free, 230 GB wanted"}
        line["warm_start"] = warm_start_measurement(dev)
    if not args.no_newton:
        line["patch_test"] = patch_measurement(dev)
    if not args.no_dual_map:
        line["dual_mesh"] = dual_mesh_measurement(dev)
        line["face_clip"] = face_clip_measurement(dev)
        line["master_rows"] = master_grad_measurement(dev)
    line["precision_vs_fp64"] = precision_measurement(dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


def dense_measurement(dev, alu, steps=20):
    """Contact-dense pass: the gel pad (131,072 slave triangles x 16 samples)
    pressed fully onto a low Perlin plate (390,728 triangles), so that every
    face sample is active (scenes.gel_dense); mixed precision, one pass per
    step as in the headline (broad phase, E, gradient, BSR Hessian, step
    bound), CUDA graph, L2 flushed between steps.  Rooflines: the pass's
    algorithmic bytes (pass_bytes) against the measured HBM copy bandwidth,
    and the sample evaluation's FP32 model -- 160 flops per evaluated
    (sample, candidate) item -- against the measured FP32 FMA rate."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc, x_np = S.gel_dense(with_tets=False)
    nk = 4 ** sc.params["face_rule_level"]
    rng = np.random.default_rng(13)
    dx_np = np.zeros_like(x_np)
    dx_np[:, 2] = -2e-6 * (0.5 + rng.random(x_np.shape[0]))
    dx_np[:, :2] = 5e-7 * rng.normal(size=(x_np.shape[0], 2))
    ctx = binding.Context(sc, precision="mixed", device=dev)
    x = torch.as_tensor(x_np, device="cuda")
    dx = torch.as_tensor(dx_np, device="cuda")
    xm = torch.as_tensor(sc.Y0, device="cuda")
    units, cand = samples_per_pass(ctx, x, xm, nk)
    first = ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=True)
    cnt, nnzb = first["counts"], first["hess"].nnzb
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((sc.X.shape[0], 3), device="cuda", dtype=torch.float32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=False, energy_dev=e_dev,
                                grad_out=grad)
    tune_s, tune_q, _ = ctx.autotune(x, xm, dx, reps=2)
    for _ in range(3):
        info = step()
    torch.cuda.synchronize()
    ms, info = time_steps(step, stream, steps, flush)
    ms_pass = statistics.median(ms)
    sec = sections(ctx, step, flush, steps)
    kern = ctx.pass_kernels()
    alg_b, parts = pass_bytes(sc, ctx, nnzb)
    ctx.close()
    peaks, kind = load_peaks()
    evals = int(cnt["face_evaluated"]) + 2 * int(cand["edge"]) + int(cand["point"])
    item_ms = sec.get("items", 0.0) + sec.get("samples", 0.0)
    gbs = alg_b / (ms_pass * 1e-3) / 1e9
    tf = 160.0 * evals / (item_ms * 1e-3) / 1e12 if item_ms > 0 else None
    return {"workload": "gel_dense: 256x256 gel pad (131,072 slave tris x 16 samples) pressed fully onto a "
                        "442x442-quad Perlin plate (390,728 tris, amplitude 0.1 mm), dhat 5e-5",
            "samples_per_pass": int(units), "active": {k: int(cnt[k]) for k in ("face", "edge", "point")},
            "evaluated_items": evals, "ms_per_pass": ms_pass, "samples_per_s": units / (ms_pass * 1e-3),
            "kernels_per_pass": kern, "sections_ms": {k: round(v, 4) for k, v in sec.items()},
            "autotuned_blocks_per_sm": {"samples": tune_s, "query": tune_q},
            "roofline_hbm": {"achieved_gbs": gbs, "peak_gbs": peaks["hbm_gbs"], "frac": gbs / peaks["hbm_gbs"],
                             "target_frac": 0.6, "algorithmic_bytes_per_pass": alg_b, "bytes_by_part": parts,
                             "peak_source": kind},
            "roofline_fp32_model": {"flops_per_item": 160, "section_ms": item_ms, "achieved_tflops": tf,
                                    "peak_tflops": alu["fp32_tflops"],
                                    "frac": tf / alu["fp32_tflops"] if tf else None,
                                    "sections": "samples (frames, pre-tests) + items (exact FP64 cast)"},
            "alpha": info["alpha"], "l2": "flushed (256 MB write) between passes"}


def precision_measurement(dev):
    """What the mixed path's FP32 barrier, gradient and Hessian cost in
    accuracy against the all-FP64 path, on a pressed 24x24-quad indent (the
    FP64 path matches the FP64 CPU oracle to 1e-12, tests/test_gpu_contact.py),
    and what the FP64 anchors keep: the additive-CCD step (FP64 in both),
    the linearised step bound, and one implicit-Euler step (its line-search
    energy sum and PCG dot products are FP64 in both precisions)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc = S.tactile_indent(n_quads=24, side=12e-3, nz=2, thick=1e-3, sphere_subdiv=3, radius=5e-3,
                          face_rule_level=2)
    x = S.drape_on_master(sc, 0.12e-3)
    rng = np.random.default_rng(3)
    dx = np.zeros_like(x)
    dx[:, 2] = -(1e-5 + 2e-5 * rng.random(x.shape[0]))
    out = {}
    res = {}
    for prec in ("fp64", "mixed"):
        ctx = binding.Context(sc, precision=prec, device=dev)
        r = ctx.contact_pass(x, sc.Y0, dx, grad=True, hess=True, counts=True)
        rp, ci, vals = (t.cpu().numpy() for t in r["hess"])
        blocks = {}
        for i in range(rp.shape[0] - 1):
            for k in range(rp[i], rp[i + 1]):
                blocks[(i, int(ci[k]))] = vals[k].astype(np.float64)
        res[prec] = (r["energy"], r["grad"].double().cpu().numpy(), blocks, r["alpha_lin"], r["alpha_accd"],
                     r["counts"])
        ctx.close()
    e64, g64, b64, al64, aa64, c64 = res["fp64"]
    e32, g32, b32, al32, aa32, c32 = res["mixed"]
    big = max(np.linalg.norm(b) for b in b64.values())
    worst = 0.0
    for k, b in b64.items():
        nb = np.linalg.norm(b)
        if nb > 1e-9 * big:
            worst = max(worst, np.linalg.norm(b32.get(k, 0.0) - b) / nb)
    out["contact_pass"] = {
        "energy_rel": abs(e32 - e64) / abs(e64), "grad_rel_l2": float(np.linalg.norm(g32 - g64) / np.linalg.norm(g64)),
        "hess_block_max_rel": worst, "alpha_lin_rel": abs(al32 - al64) / al64 if np.isfinite(al64) else 0.0,
        "alpha_accd_equal": aa32 == aa64,
        "same_active_samples": all(c32[k] == c64[k] for k in ("face", "edge", "point")),
        "gap_and_decisions": "FP64 in both paths, or FP32 certified to decide as FP64 (same active samples)"}
    # one implicit-Euler step of the same pad pressed onto the sphere from the
    # draped state: the FP64 anchors (line-search energy sum, PCG dot products,
    # step bounds) are FP64 in both precisions
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    steps = {}
    for prec in ("fp64", "mixed"):
        ctx = binding.Context(sc, precision=prec, device=dev, params={"pcg_rel_tol": 1e-6})
        xs = torch.as_tensor(x.copy(), device="cuda")
        vs = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
        r = ctx.newton_step(xs, vs)
        steps[prec] = (xs.cpu().numpy(), r)
        ctx.close()
    (x64, r64), (x32, r32) = steps["fp64"], steps["mixed"]
    disp = np.linalg.norm(x64 - x)
    out["time_step"] = {
        "status": [r64["status"], r32["status"]], "newton_iters": [r64["newton_iters"], r32["newton_iters"]],
        "pcg_iters": [r64["pcg_iters"], r32["pcg_iters"]],
        "position_rel_to_displacement": float(np.linalg.norm(x32 - x64) / disp) if disp > 0 else 0.0,
        "incremental_potential_rel": abs(r32["energy"] - r64["energy"]) / abs(r64["energy"]),
        "residual": [r64["residual"], r32["residual"]],
        "note": "mixed (FP32 barrier, gradient, Hessian, PCG vectors and matrix; double-float elastic energy and gradient) against FP64, same start state"}
    return out


def face_clip_measurement(dev, n_pairs=2_000_000, reps=20):
    """Paper-exact face samples (Sec. 4.1, ipc_face_clip_samples) on
    n_pairs seeded (slave, master) triangle pairs of unit size: slaves near
    z = 0, masters 0.05-0.3 above with random tilt and offset (about half of
    the pairs overlap in projection).  Throughput of the sampler in pairs/s
    and samples/s (CUDA events, L2 flushed between launches)."""
    import torch
    from paper_2605_24339_b300 import binding
    rng = np.random.default_rng(12)
    xs = np.c_[rng.uniform(0, 1, (3 * n_pairs, 2)), rng.uniform(-0.05, 0.05, 3 * n_pairs)]
    xm = np.c_[rng.uniform(0, 1, (3 * n_pairs, 2)), rng.uniform(0.05, 0.3, 3 * n_pairs)]
    T = np.arange(3 * n_pairs, dtype=np.int32).reshape(n_pairs, 3)
    pairs = np.c_[np.arange(n_pairs), np.arange(n_pairs)].astype(np.int32)
    a = [torch.as_tensor(v, device=dev) for v in (xs, T, xm, T, pairs)]
    smp, cnt = binding.face_clip_samples(*a)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    times = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        smp, cnt = binding.face_clip_samples(*a)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    s = statistics.median(times)
    n_samples = int(cnt.sum().item())
    return {"workload": f"{n_pairs} seeded unit-size triangle pairs (slave near z = 0, tilted masters above)",
            "ms_per_call": round(s * 1e3, 3), "pairs_per_s": n_pairs / s, "samples_per_call": n_samples,
            "samples_per_s": n_samples / s, "overlapping_pairs": int((cnt > 0).sum().item()),
            "note": "wall time of the call and a synchronisation"}


def master_grad_measurement(dev, reps=50):
    """Master rows of two-sided GMCP (Sec. 4.3 with Eq. gap, ipc_master_grad)
    on the pressed gel_on_terrain state: the broad phase plus the
    item-parallel FP64 sample kernels, which add kappa w gamma B'(g) bm_j n_s
    to each master vertex (ipc_master_hess: the blocks with master vertices,
    wall time of the synchronising call).  CUDA events on the context's stream, L2 flushed between calls.
    The balance check (net master force + net slave force, relative to the
    total slave force) holds at any size."""
    import torch
    from paper_2605_24339_b300 import binding
    sc, x, _ = make_workload()
    ctx = binding.Context(sc, precision="mixed", device=dev)
    xd = torch.as_tensor(x, device="cuda")
    xm = torch.as_tensor(sc.Y0, device="cuda")
    out = torch.empty((sc.Y0.shape[0], 3), dtype=torch.float64, device="cuda")
    for _ in range(3):
        ctx.master_grad(xd, xm, out)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        ctx.master_grad(xd, xm, out)
        e1.record()
    torch.cuda.synchronize()
    ms = statistics.median([e0.elapsed_time(e1) for e0, e1 in ev])
    # the Hessian blocks with master vertices (synchronising call: wall time)
    ij, blk = ctx.master_hess(xd, xm)
    cap = ij.shape[0]
    ij = torch.empty((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    blk = torch.empty((max(cap, 1), 9), dtype=torch.float64, device="cuda")
    n = ctypes.c_int64()
    hts = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = binding.lib().ipc_master_hess(ctx.h, binding._ptr(xd), binding._ptr(xm), cap, binding._ptr(ij),
                                           binding._ptr(blk), ctypes.byref(n))
        hts.append(time.perf_counter() - t0)
        assert st == 0
    ctx64 = binding.Context(sc, precision="fp64", device=dev)
    gm = ctx64.master_grad(xd, xm).cpu().numpy()
    gs = ctx64.barrier_eval(xd, xm, hess=False, counts=False)["grad"].cpu().numpy()
    bal = float(np.abs(gm.sum(axis=0) + gs.sum(axis=0)).max() / np.abs(gs).sum())
    rows = int(np.any(gm != 0, axis=1).sum())
    ctx.close()
    ctx64.close()
    return {"workload": "gel_on_terrain pad draped 0.15 mm onto the terrain (master rows of every active sample)",
            "ms_per_call": round(ms, 4), "master_rows": rows, "balance_rel": bal,
            "hess_ms_per_call": round(statistics.median(hts) * 1e3, 4), "hess_blocks": int(n.value),
            "l2": "flushed (256 MB write) between calls",
            "note": "broad phase + item-parallel FP64 sample kernels (k_items_pre, k_items); the rows' entries sorted by master vertex and summed in a fixed order (two host synchronisations)"}


def dual_mesh_measurement(dev, n_points=2_000_000, reps=50):
    """Dual-mesh mapper (Sec. 3.2): a visual mesh of n_points seeded points
    near the gel pad's 131,072-triangle tactile surface (random barycentrics
    on random surface triangles, offsets of +-0.2 mm along the normal),
    embedded once (ipc_dual_map_build, wall time) and updated per frame from
    deformed simulation vertices (ipc_dual_map_apply, CUDA events, L2
    flushed between frames).  Roofline of the update: HBM bytes (per point
    tri 4 B + uvwd 32 B + output 24 B, plus the simulation vertices and
    triangles once) against the measured copy bandwidth, and its FP64
    operations against the FP64 pipe."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain()
    V = np.ascontiguousarray(sc.X, dtype=np.float64)
    T = np.ascontiguousarray(sc.stris, dtype=np.int32)
    rng = np.random.default_rng(11)
    k = rng.integers(0, len(T), n_points)
    b = rng.dirichlet([1.0, 1.0, 1.0], n_points)
    A, Bv, Cv = V[T[k, 0]], V[T[k, 1]], V[T[k, 2]]
    nrm = np.cross(Bv - A, Cv - A)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    P = b[:, :1] * A + b[:, 1:2] * Bv + b[:, 2:] * Cv + rng.uniform(-2e-4, 2e-4, (n_points, 1)) * nrm
    Vd = torch.as_tensor(V, device=dev)
    Td = torch.as_tensor(T, device=dev)
    Pd = torch.as_tensor(P, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tri, uvwd, d2 = binding.dual_map_build(Vd, Td, Pd)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    # deformed simulation vertices: a smooth bend of the pad
    W = V.copy()
    W[:, 2] += 0.05 * (W[:, 0] - W[:, 0].mean()) ** 2
    Wd = torch.as_tensor(W, device=dev)
    out = torch.empty((n_points, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(3):
        binding.dual_map_apply(Wd, Td, tri, uvwd, out)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for e0, e1 in ev:
        flush.zero_()
        e0.record()
        binding.dual_map_apply(Wd, Td, tri, uvwd, out)
        e1.record()
    torch.cuda.synchronize()
    ms = statistics.median([e0.elapsed_time(e1) for e0, e1 in ev])
    err = float(torch.abs(binding.dual_map_apply(Vd, Td, tri, uvwd) - Pd).max())
    peaks, src = load_peaks()
    byts = n_points * (4 + 32 + 24) + V.nbytes + T.nbytes
    gbs = byts / (ms * 1e-3) / 1e9
    fp64_ops = 32 * n_points
    fp64_peak = 148 * 2 * 2032e6
    return {"workload": f"{n_points} visual points near the 131,072-triangle tactile surface of gel_on_terrain",
            "build_s": round(build_s, 3), "apply_ms": round(ms, 4),
            "points_per_s": n_points / (ms * 1e-3),
            "undeformed_max_err_m": err, "max_dist_m": float(np.sqrt(d2.max().item())),
            "roofline": {"hbm_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_frac": gbs / peaks["hbm_gbs"],
                         "peak_source": src, "bytes_per_apply": byts, "fp64_ops_per_point": 32,
                         "fp64_frac": fp64_ops / (ms * 1e-3) / fp64_peak,
                         "fp64_peak_note": "148 SMs x 2 FP64 lanes/clock x 2032 MHz"},
            "l2": "flushed (256 MB write) between frames"}


def batched_measurement(dev, n_env=512, steps=20):
    """Batched contact pass: n_env fingertip environments (5 pads of 16-128
    quads of 0.25 mm, 4 samples per slave triangle, around a perturbed convex
    object of 2k-80k triangles), every pad pressed 1.5 dhat toward its
    object, in one pass per step (one grid per environment, persistent
    kernels over all of them, captured CUDA graph, autotuned launch shapes).
    L2 is flushed between steps.  The environments are generated in worker
    processes (spawn) and without tetrahedra: the contact pass reads the
    surfaces only."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    t0 = time.perf_counter()
    dhat = 1e-4
    sc, x_np = S.fingertip_batch(n_env=n_env, dhat=dhat, pressed=1.5 * dhat, with_tets=False,
                                 workers=max(1, min(32, os.cpu_count() or 1)))
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(5)
    dx_np = np.zeros_like(x_np)
    dx_np[:, :] = -1e-6 * (x_np - x_np.mean(axis=0)) / np.linalg.norm(x_np - x_np.mean(axis=0), axis=1)[:, None]
    t1 = time.perf_counter()
    ctx = binding.Context(sc, precision="mixed", device=dev)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t1
    x = torch.as_tensor(x_np, device="cuda")
    dx = torch.as_tensor(dx_np, device="cuda")
    xm = torch.as_tensor(sc.Y0, device="cuda")
    nk = 4 ** sc.params["face_rule_level"]
    c = ctx.candidates(x, xm)
    units = ctx.ns * nk + 2 * c["edge"] + c["point"]
    tune_s, tune_q, _ = ctx.autotune(x, xm, dx, reps=2)
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.empty((sc.X.shape[0], 3), device="cuda", dtype=torch.float32)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        return ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=False, energy_dev=e_dev,
                                grad_out=grad)
    for _ in range(3):
        info = step()
    full = ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=True)
    cnt = full["counts"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        ev0.record(stream)
        info = step()
        ev1.record(stream)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    # per-section device times, as for the single-environment pass
    ctx.profile_start()
    for _ in range(steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    ctx.profile_stop()
    prof = ctx.profile_read()
    free_b, total_b = torch.cuda.mem_get_info()
    ctx.close()
    ms = total / steps
    return {"workload": f"fingertip_batch {n_env} envs x 5 pads (16-128 quads, 4 samples/tri) vs "
                        f"2k-80k-tri objects, pads pressed 1.5 dhat",
            "n_env": n_env, "slave_tris": int(sc.stris.shape[0]), "master_tris": int(sc.mtris.shape[0]),
            "samples_per_pass": int(units), "active_face_samples": int(cnt["face"]),
            "candidates": {k: int(c[k]) for k in ("face", "edge", "point")},
            "face_evaluated": int(cnt["face_evaluated"]), "query_tris": int(cnt["query_tris"]),
            "swept_tris": int(full["swept_tris"]), "ccd_pairs": [int(full["n_pt"]), int(full["n_ee"])],
            "ms_per_pass": ms, "samples_per_s": units / (ms / 1e3),
            "autotuned_blocks_per_sm": {"samples": tune_s, "query": tune_q},
            "sections_ms": {k: round(v["ms"] / max(v["calls"], 1), 4) for k, v in prof.items()},
            "alpha": info["alpha"], "scene_build_s": round(gen_s, 1), "context_create_s": round(create_s, 1),
            "gpu_mem_used_gb": round((total_b - free_b) / 1e9, 1)}


def newton_measurement(dev, start_step=20, n_states=4):
    """Second half of the metric: wall time of one implicit-Euler step solved
    to a 1e-6 residual (ipc_newton_step), mixed precision against plain FP64.
    States: the gel_on_terrain press run from rest in mixed precision; steps
    ``start_step`` .. ``start_step + n_states - 1`` (contact starts at step 10)
    are recorded as (x^t, v^t).  Each precision then solves the step from
    every recorded state (after one untimed step that builds its time-stepper
    state); the median wall time is reported."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain()
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    gen = binding.Context(sc, precision="mixed", device=dev)
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = vd.clone()
    states = []
    for k in range(start_step + n_states):
        if k >= start_step:
            states.append((x.clone(), v.clone()))
        r = gen.newton_step(x, v)
        v[top] = vd[top]
        if r["status"] != 0:
            break
    gen.close()
    out = {"workload": f"gel_on_terrain press from rest, steps {start_step}..{start_step + len(states) - 1} "
                       f"(top face at -0.5 mm/s, h = 10 ms, in contact from step 10)",
           "n_vert": int(sc.X.shape[0]), "n_tet": int(sc.tets.shape[0]),
           "newton_tol": sc.params["newton_tol"], "pcg_rel_tol": sc.params["pcg_rel_tol"]}
    for prec in ("fp64", "mixed"):
        ctx = binding.Context(sc, precision=prec, device=dev)
        ctx.newton_step(states[0][0].clone(), states[0][1].clone())
        times, iters, pcg, ok = [], [], [], True
        for xs0, vs0 in states:
            xs, vs = xs0.clone(), vs0.clone()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ctx.newton_step(xs, vs)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
            iters.append(st["newton_iters"])
            pcg.append(st["pcg_iters"])
            ok = ok and st["status"] == 0 and st["residual"] <= sc.params["newton_tol"]
        out[prec] = {"ms_per_step_median": statistics.median(times), "ms_per_step": [round(t, 1) for t in times],
                     "newton_iters": iters, "pcg_iters": pcg, "all_converged": ok,
                     "newton_iters_per_s": sum(iters) / (sum(times) / 1e3)}
        ctx.close()
    out["speedup_mixed_vs_fp64"] = out["fp64"]["ms_per_step_median"] / out["mixed"]["ms_per_step_median"]
    return out


def config1_measurement(dev):
    """The single-environment indent as specified (32x32-quad pad, 2 mm Neo-Hookean slab pressed
    0.3 mm in 10 steps onto the rigid subdivision-3 icosphere, dhat 1e-4, kappa 1e5, h 1 ms,
    vertex jitter 1e-5 m, seed 1), stepped on the GPU in plain FP64 and in mixed precision up
    to the first step that fails.  Reported per step: status (0 converged to the 1e-6 residual;
    4 infeasible, the state kept; 6 not converged within max_newton iterations), Newton and PCG
    iterations, the final residual and the wall time.  The fifth step fails in both: a slave
    edge closes on a master edge near the indenter's tip where no sample measures the gap, and
    the additive CCD stops each iterate short of it (with such pairs ~1e-13 m apart, later
    steps take tens of seconds in FP64, so the run stops at the first failure)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc = S.tactile_indent()
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    out = {"workload": "tactile_indent: 32x32-quad pad (1,089 surface verts, 2,048 slave tris x 4 samples), "
                       "2 mm slab (4 tet layers) pressed 0.3 mm in 10 steps onto a subdivision-3 icosphere "
                       "(1,280 tris, radius 5 mm); dhat 1e-4, kappa 1e5, h 1 ms, jitter 1e-5 m",
           "n_vert": int(sc.X.shape[0]), "n_tet": int(sc.tets.shape[0]), "max_newton": sc.params["max_newton"]}
    for prec in ("fp64", "mixed"):
        ctx = binding.Context(sc, precision=prec, device=dev)
        x = torch.as_tensor(sc.X.copy(), device="cuda")
        v = vd.clone()
        rows = []
        for _ in range(sc.n_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ctx.newton_step(x, v)
            torch.cuda.synchronize()
            rows.append({"status": r["status"], "newton_iters": r["newton_iters"], "pcg_iters": r["pcg_iters"],
                         "residual": r["residual"], "ms": round((time.perf_counter() - t0) * 1e3, 2)})
            v[top] = vd[top]
            if r["status"] != 0:
                break
        ctx.close()
        out[prec] = {"steps": rows, "converged_steps": sum(q["status"] == 0 for q in rows),
                     "first_failed_step": next((k for k, q in enumerate(rows) if q["status"] != 0), None)}
    return out


def ccd_stress_measurement(dev, calls=10):
    """The step bound on the CCD / line-search stress workload at its specified size: 64
    environments, each a free 128x128-quad pad (0.25 mm, 4 tet layers) moving at U[0.5, 2] m/s
    toward a closed 30x30x1 mm thin shell (100x100 quads a face) from 1 mm away, at a seeded
    random rotation; h = 1 ms, so a step moves a pad 0.5-2 mm, up to twice the shell's thickness.
    Times ipc_ccd_max_step for the whole batch on the first step's displacement h v (broad phase
    of the swept boxes, Eq. (ccd)/(global_ccd) over the samples, additive CCD over the swept
    primitive pairs), inputs resident, after one untimed call."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    t0 = time.perf_counter()
    sc, v0 = S.ccd_stress()
    gen_s = time.perf_counter() - t0
    ctx = binding.Context(sc, precision="mixed", device=dev)
    x = torch.as_tensor(sc.X, device="cuda")
    dx = torch.as_tensor(sc.params["h"] * v0, device="cuda")
    y0 = torch.as_tensor(sc.Y0, device="cuda")
    r = ctx.ccd_max_step(x, dx, y0)
    torch.cuda.synchronize()
    times = []
    for _ in range(calls):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = ctx.ccd_max_step(x, dx, y0)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t1) * 1e3)
    ctx.close()
    ms = statistics.median(times)
    pairs = int(r["n_pt"]) + int(r["n_ee"])
    return {"workload": "ccd_stress: 64 envs, 128x128-quad free pads at 0.5-2 m/s toward closed 1 mm shells "
                        "(100x100 quads a face), random rotations, h = 1 ms",
            "n_env": 64, "slave_tris": int(sc.stris.shape[0]), "master_tris": int(sc.mtris.shape[0]),
            "scene_build_s": round(gen_s, 1), "ms_per_call": ms, "ms_per_call_all": [round(t, 2) for t in times],
            "alpha": r["alpha"], "alpha_lin": r["alpha_lin"], "alpha_accd": r["alpha_accd"],
            "accd_pairs": {"point_triangle": int(r["n_pt"]), "edge_edge": int(r["n_ee"])},
            "accd_pairs_per_s": pairs / (ms / 1e3), "swept_tris": int(r["swept_tris"]),
            "iter_cap_hit": r["iter_cap_hit"]}


def fingertip_step_scene(n_env, layers=2):
    """The batched time-step workload: n_env fingertip environments with
    tets (5 pads of 16-128 quads of 0.25 mm, ``layers`` tet layers, around a perturbed
    convex object of 2k-80k triangles, each pad 1.5 dhat pressed toward it,
    top faces driven at 0.5 mm/s), generated in spawn worker processes past
    16 environments.  Returns (parts [(scene, x0) per env], the concatenated
    scene, its x0)."""
    from paper_2605_24339_b300 import scenes as S
    dhat = 1e-4
    args = (5, (16, 128), 0.25e-3, layers, 0.5e-3, (2000, 80000), 15e-3, dhat, 1e5, 1e-3, 0.5e-3, 100, 3, 1,
            1.5 * dhat, True)
    workers = max(1, min(32, os.cpu_count() or 1))
    if n_env > 16 and workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(S._fingertip_env, range(n_env), *[[a] * n_env for a in args],
                                chunksize=max(1, n_env // (4 * workers))))
    else:
        parts = [S._fingertip_env(e, *args) for e in range(n_env)]
    sc = S.concat_envs([p[0] for p in parts], name="fingertip_batch")
    return parts, sc, np.concatenate([p[1] for p in parts])


def batched_step_measurement(dev, n_env=16, steps=3, alone_envs=16, layers=2):
    """Batched time steps (ipc_newton_step_envs): n_env fingertip environments
    of the batched workload's recipe with their tetrahedra (5 pads of 16-128
    quads of 0.25 mm, ``layers`` tet layers through their 0.5 mm, around a perturbed convex object of
    2k-80k triangles), every pad starting 1.5 dhat pressed toward its object
    (in contact from the first step) with its top face driven at 0.5 mm/s.
    Each environment has its own Newton iteration, solve, step bound and
    stopping; one call steps them all.  Timed: ``steps`` batched steps after
    one untimed step (which builds the time-stepper state), and the same
    steps taken one environment at a time with a context per environment
    (the batch's results are bit for bit those), for the first
    ``alone_envs`` environments; the comparison is in environment-steps
    per second."""
    import torch
    from paper_2605_24339_b300 import binding
    t0 = time.perf_counter()
    parts, sc, x0 = fingertip_step_scene(n_env, layers)
    gen_s = time.perf_counter() - t0
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    out = {"workload": f"fingertip_batch {n_env} envs x 5 pads (16-128 quads, {layers} tet layers, 4 samples/tri) vs "
                       f"2k-80k-tri objects, pads 1.5 dhat pressed, top faces at 0.5 mm/s, h = 1 ms",
           "n_env": n_env, "n_vert": int(sc.X.shape[0]), "n_tet": int(sc.tets.shape[0]),
           "slave_tris": int(sc.stris.shape[0]), "master_tris": int(sc.mtris.shape[0]),
           "newton_tol": sc.params["newton_tol"], "scene_build_s": round(gen_s, 1)}
    t0 = time.perf_counter()
    ctx = binding.Context(sc, precision="mixed", device=dev)
    x = torch.as_tensor(x0, device="cuda")
    v = vd.clone()
    torch.cuda.synchronize()
    out["context_create_s"] = round(time.perf_counter() - t0, 2)
    t0 = time.perf_counter()
    ctx.newton_step_envs(x, v)
    torch.cuda.synchronize()
    out["first_step_s_with_setup"] = round(time.perf_counter() - t0, 2)
    v[top] = vd[top]
    times, iters, statuses = [], [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r, per = ctx.newton_step_envs(x, v)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
        v[top] = vd[top]
        iters.append([q["newton_iters"] for q in per])
        statuses.append(sorted(set(q["status"] for q in per)))
    free_b, total_b = torch.cuda.mem_get_info()
    out["gpu_mem_used_gb"] = round((total_b - free_b) / 1e9, 1)
    ctx.close()
    ms = statistics.median(times)
    out["batched"] = {"ms_per_step_median": ms, "ms_per_step": [round(t, 1) for t in times],
                      "env_steps_per_s": n_env / (ms / 1e3),
                      "env_newton_iters_per_s": float(sum(sum(i) for i in iters)) / (sum(times) / 1e3),
                      "newton_iters_max": [max(i) for i in iters], "newton_iters_mean": [float(np.mean(i)) for i in iters],
                      "statuses": statuses}
    # the same states stepped one environment at a time
    seq = []
    for e, (pe, xe) in enumerate(parts[:alone_envs]):
        c = binding.Context(pe, precision="mixed", device=dev, params=sc.params)
        xg = torch.as_tensor(xe, device="cuda")
        tp = torch.as_tensor(pe.dirichlet.astype(bool), device="cuda")
        vde = torch.as_tensor(pe.v_dirichlet, device="cuda")
        vg = vde.clone()
        c.newton_step(xg, vg)
        vg[tp] = vde[tp]
        tt = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.newton_step(xg, vg)
            torch.cuda.synchronize()
            tt.append((time.perf_counter() - t0) * 1e3)
            vg[tp] = vde[tp]
        c.close()
        seq.append(tt)
    na = len(seq)
    seq_ms = [sum(t[k] for t in seq) for k in range(steps)]
    rate = na / (statistics.median(seq_ms) / 1e3)
    out["one_env_at_a_time"] = {"envs": na, "ms_for_these_envs_median": statistics.median(seq_ms),
                                "env_steps_per_s": rate}
    out["env_steps_per_s_batched_over_one_at_a_time"] = out["batched"]["env_steps_per_s"] / rate
    return out


def patch_measurement(dev, steps=12):
    """Contact patch test with a deformable master (Sec. 5.1, Table
    patch_test): two 1 x 1 x 0.5 blocks on non-matching structured tet
    meshes (5x5x2 and 4x4x2 cells), E = 1000, nu = 0, a pressure of 10 on the
    upper block's top, the lower block's bottom held, h = 0.05 s, FP64 (the
    free lateral mode of the upper block makes the system too ill-conditioned
    for the FP32 matrix to reach the 1e-6 residual at rest); ``steps`` joint
    time steps (ipc_newton_step_joint) per kappa.
    Reported per kappa: sigma_zz mean and largest relative error per block,
    the largest other stress component, statuses, Newton iterations and the
    median wall time of a step.  The exact state is sigma_zz = -10."""
    import torch
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "tests"))
    from helpers import patch_report
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    out = {"workload": "patch_test 5x5x2 over 4x4x2 cells, E 1000, nu 0, pressure 10, h 0.05 s, "
                       f"{steps} steps", "paper_table": {"1e4": [8.00e-4, 6.00e-3], "1e6": [4.66e-5, 2.48e-4],
                                                          "1e8": [4.66e-5, 2.48e-4]}}
    for kappa in (1e4, 1e6, 1e8):
        sc, f = S.patch_test(kappa=kappa, h=0.05, density=1.0)
        ctx = binding.Context(sc, precision="fp64", device=dev)
        x = torch.as_tensor(np.concatenate([sc.X, sc.Y0]), device="cuda")
        v = torch.zeros_like(x)
        ft = torch.as_tensor(f, device="cuda")
        times, st = [], []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = ctx.newton_step_joint(x, v, f_ext=ft)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
            st.append((r["status"], r["newton_iters"]))
        ctx.close()
        rep = patch_report(sc, x.cpu().numpy())
        out[f"kappa_{kappa:.0e}"] = {"report": rep, "status_iters": st,
                                     "ms_per_step_median": statistics.median(times)}
    return out


def warm_start_measurement(dev, train_iters=1500, timed_iters=50):
    """Learned warm start on the terrain press: tensor-core training
    throughput (one Adam step = forward + backward over all 594,441
    vertices) and what the trained network gains on held-out steps (start
    fraction alpha0, Newton iterations, wall time), against the plain
    predictor from the same states."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    from paper_2605_24339_b300 import warmstart as WS
    sc = S.gel_on_terrain()
    sc.params.update(max_newton=60)
    ctx = binding.Context(sc, precision="mixed", device=dev)
    p0 = WS.init_params(0)
    p0[-3 - 3 * 256:] = 0.0
    ctx.ws_create(p0, lr=3e-4, **WS.default_scales(sc))
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
    WS.rollout(ctx, sc, x, v, 8, record=False)
    ro = WS.rollout(ctx, sc, x, v, 20, record=True)
    for smp in ro.samples:
        big = (smp.target.abs().amax(dim=1) > 0.02).float()
        smp.mask = (smp.mask * (0.01 + big + smp.feats[:, 14].float())).contiguous()
    WS.train(ctx, ro.samples[:14], train_iters, seed=1)
    s0 = ro.samples[0]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(timed_iters):
        ctx.ws_train_step(s0.feats, s0.target, s0.mask)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / timed_iters
    n = sc.X.shape[0]
    macs = 32 * 256 + 2 * 256 * 256 + 256 * 3
    # forward 2 n macs; backward: activation gradients of layers 2-3 and all
    # weight gradients, 2 n (macs - 32*256) + 2 n macs
    flops = 2.0 * n * macs + 2.0 * n * (macs - 32 * 256) + 2.0 * n * macs
    res = WS.compare_starts(ctx, sc, ro.states[14:20])
    held = ro.samples[14:20]
    net = [ctx.ws_grads(sm.feats, sm.target, sm.mask)[0] for sm in held]
    zero = [float((sm.mask[:, None] * sm.target ** 2).sum() / (3 * sm.mask.sum())) for sm in held]
    ctx.close()
    peaks, _ = load_peaks()
    tf = flops / (ms / 1e3) / 1e12
    return {
        "workload": "gel_on_terrain press, train on steps 8-21, held out 22-27",
        "train_ms_per_step": ms, "train_tflops": tf, "train_flops_per_step": flops,
        "train_frac_of_bf16_peak": tf / peaks.get("bf16_tflops", 1800.0),
        "held_out_loss": {"network": net, "plain_predictor": zero},
        "plain": {"newton_iters": [r["newton_iters"] for r in res["plain"]],
                  "alpha0": [r["alpha0"] for r in res["plain"]],
                  "wall_ms": [round(r["wall_ms"], 1) for r in res["plain"]]},
        "learned": {"newton_iters": [r["newton_iters"] for r in res["learned"]],
                    "alpha0": [r["alpha0"] for r in res["learned"]],
                    "pred_used": [r["pred_used"] for r in res["learned"]],
                    "wall_ms": [round(r["wall_ms"], 1) for r in res["learned"]]},
    }


def _oracle_windows(n):
    """n windows (4 mm squares) of the benchmark state, spread over the pad
    in a grid, each a contact-only sub-scene with its own seeded step dx."""
    from paper_2605_24339_b300 import scenes as S
    sc, x, _ = make_workload()
    k = int(np.ceil(np.sqrt(n)))
    lo, hi = x[:, 0].min() + CROP_HALF_WIDTH, x[:, 0].max() - CROP_HALF_WIDTH
    cs = np.linspace(lo, hi, k)
    out = []
    for i in range(n):
        c = (cs[i % k], cs[(i // k) % k])
        sub, xs = S.crop(sc, x, c, CROP_HALF_WIDTH, 4 * sc.params["dhat"])
        rng = np.random.default_rng(11 + i)
        dxs = np.zeros_like(xs)
        dxs[:, 2] = -5e-6 * (0.5 + rng.random(xs.shape[0]))
        dxs[:, :2] = 1e-6 * rng.normal(size=(xs.shape[0], 2))
        out.append((sub, xs, dxs))
    return out


def _oracle_worker(win, passes, start, q):
    """One host core: the FP64 oracle, as it stands, over one window -- an
    untimed pass, then ``passes`` timed passes (energy, gradient, Hessian and
    step bound), started together with the other workers."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    sub, xs, dxs = win
    Os = O.Scene(sub)
    nk = 4 ** sub.params["face_rule_level"]
    units = (sub.stris.shape[0] * nk + 2 * Os.candidates(1, xs, sub.Y0).shape[0]
             + Os.candidates(2, xs, sub.Y0).shape[0])
    Os.contact(xs, sub.Y0)
    Os.ccd_max_step(xs, dxs, sub.Y0)
    start.wait()
    t0 = time.perf_counter()
    for _ in range(passes):
        Os.contact(xs, sub.Y0)
        Os.ccd_max_step(xs, dxs, sub.Y0)
    q.put((units * passes, t0, time.perf_counter()))


def oracle_all_cores(passes=1, procs=None, windows=None):
    """The oracle on every host core: one spawned process per core, each on
    its own window of the workload; throughput = all samples over the span
    from the first start to the last finish."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    procs = procs or len(os.sched_getaffinity(0))
    windows = windows or _oracle_windows(procs)
    ctx = mp.get_context("spawn")
    start = ctx.Barrier(procs)
    q = ctx.Queue()
    ps = [ctx.Process(target=_oracle_worker, args=(windows[i], passes, start, q)) for i in range(procs)]
    for p in ps:
        p.start()
    res = [q.get() for _ in ps]
    for p in ps:
        p.join()
    units = sum(r[0] for r in res)
    span = max(r[2] for r in res) - min(r[1] for r in res)
    return units / span, span, procs, windows


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline():
    """The FP64 oracle, as it stands, on all host cores (one window of the
    workload per core, bounded: one timed pass each)."""
    v, span, procs, wins = oracle_all_cores(passes=1)
    n_tris = sum(w[0].stris.shape[0] for w in wins)
    return {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "cpu": _cpu_model(),
            "sample": f"{procs} processes, one per core, each one pass over its own "
                      f"{2 * CROP_HALF_WIDTH * 1e3:.0f} mm window of the workload ({n_tris} slave tris in all)",
            "seconds": span}


def run_passes(args):
    """A few contact passes on the benchmark workload with no timing: the
    command line used for ncu captures of single kernels."""
    import torch
    from paper_2605_24339_b300 import binding
    sc, x_np, dx_np = make_workload()
    ctx = binding.Context(sc, precision=args.precision)
    x = torch.as_tensor(x_np, device="cuda")
    dx = torch.as_tensor(dx_np, device="cuda")
    xm = torch.as_tensor(sc.Y0, device="cuda")
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        info = ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=False, energy_dev=e_dev)
    torch.cuda.synchronize()
    print(json.dumps({"passes": args.steps, "alpha": info["alpha"], "ccd_pairs_pt": info["n_pt"],
                      "ccd_pairs_ee": info["n_ee"]}))


def run_dense_passes(args):
    """--steps contact passes on the contact-dense workload with no timing
    (the command line for ncu captures of its kernels); --dense-quads sets the
    pad's quads per side (256 in the measured workload; the plate scales with
    it, keeping its 0.063 mm triangles)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    q = args.dense_quads
    sc, x_np = S.gel_dense(n_quads=q, plate_quads=max(8, (442 * q) // 256), plate_size=28e-3 * q / 256,
                           with_tets=False)
    ctx = binding.Context(sc, precision=args.precision)
    x = torch.as_tensor(x_np, device="cuda")
    dx = torch.zeros_like(x)
    dx[:, 2] = -2e-6
    xm = torch.as_tensor(sc.Y0, device="cuda")
    e_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(args.steps):
        info = ctx.contact_pass(x, xm, dx, grad=True, hess="view", counts=False, energy_dev=e_dev)
    torch.cuda.synchronize()
    print(json.dumps({"passes": args.steps, "alpha": info["alpha"]}))


def run_mlp(args):
    """--steps training steps of the warm-start network on a 594,441-vertex
    batch of seeded features and targets (the command line for profiling
    the tensor-core kernels)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    from paper_2605_24339_b300 import warmstart as WS
    sc = S.gel_on_terrain()
    ctx = binding.Context(sc, precision="mixed")
    ctx.ws_create(WS.init_params(0), lr=1e-3, **WS.default_scales(sc))
    n = sc.X.shape[0]
    g = torch.Generator(device="cuda").manual_seed(3)
    f = torch.randn((n, 32), device="cuda", generator=g).to(torch.bfloat16)
    t = torch.randn((n, 3), device="cuda", generator=g)
    m = torch.ones(n, device="cuda")
    loss = ctx.ws_train_step(f, t, m)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        loss = ctx.ws_train_step(f, t, m)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / max(1, args.steps) * 1e3
    print(json.dumps({"mlp_train_steps": args.steps, "ms_per_step": ms, "loss": loss}))


def run_newton(args):
    """--steps time steps of the gel_on_terrain press from rest (the command
    line for profiling the time-stepper kernels); --newton-quads sets the
    pad's quads per side (256 in the measured workload)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    sc = S.gel_on_terrain(n_quads=args.newton_quads)
    ctx = binding.Context(sc, precision=args.precision)
    x = torch.as_tensor(sc.X.copy(), device="cuda")
    v = torch.as_tensor(sc.v_dirichlet.copy(), device="cuda")
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    for _ in range(args.steps):
        st = ctx.newton_step(x, v)
        v[top] = vd[top]
    torch.cuda.synchronize()
    print(json.dumps({"newton_steps": args.steps, "last": {k: st[k] for k in ("status", "newton_iters", "pcg_iters")}}))


def run_profile_step(args):
    """One time step between cudaProfilerStart and cudaProfilerStop, for a
    launch list of that step alone (ncu --profile-from-start off): with
    --prof-workload batch the batched time-step workload (--step-envs
    environments, three steps first), with gel the gel_on_terrain press in
    mixed precision (21 steps first, in contact from step 10)."""
    import torch
    from paper_2605_24339_b300 import binding
    from paper_2605_24339_b300 import scenes as S
    if args.prof_workload == "batch":
        _, sc, x0 = fingertip_step_scene(args.step_envs)
        warm = 3
    else:
        sc = S.gel_on_terrain(n_quads=args.newton_quads)
        x0 = sc.X.copy()
        warm = 21
    ctx = binding.Context(sc, precision=args.precision)
    x = torch.as_tensor(x0, device="cuda")
    vd = torch.as_tensor(sc.v_dirichlet, device="cuda")
    top = torch.as_tensor(sc.dirichlet.astype(bool), device="cuda")
    v = vd.clone()
    step = (lambda: ctx.newton_step_envs(x, v)[1]) if args.prof_workload == "batch" else \
        (lambda: [ctx.newton_step(x, v)])
    for _ in range(warm):
        step()
        v[top] = vd[top]
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    per = step()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"workload": args.prof_workload, "newton_iters_max": max(q["newton_iters"] for q in per),
                      "pcg_iters_max": max(q["pcg_iters"] for q in per),
                      "statuses": sorted(set(q["status"] for q in per))}))


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (the paper ships no code) on all
    host cores; each step one pass over a window of the workload per core."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    procs = len(os.sched_getaffinity(0))
    wins = _oracle_windows(procs)
    if args.warmup > 0:
        oracle_all_cores(passes=1, procs=procs, windows=wins)
    v, span, _, _ = oracle_all_cores(passes=args.steps, procs=procs, windows=wins)
    n_tris = sum(w[0].stris.shape[0] for w in wins)
    sample = (f"each step: {procs} processes, one per core, each one pass over its own "
              f"{2 * CROP_HALF_WIDTH * 1e3:.0f} mm window ({n_tris} slave tris in all)")
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": span / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "window": sample}, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle", "cpu": _cpu_model(),
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-envs measurement")
    ap.add_argument("--no-dense", action="store_true", help="skip the contact-dense measurement")
    ap.add_argument("--no-dual-map", action="store_true", help="skip the dual-mesh mapper, face-clip and master-row measurements")
    ap.add_argument("--dual-points", type=int, default=2_000_000,
                    help="--mode dualmap: visual points of the dual-mesh measurement")
    ap.add_argument("--no-newton", action="store_true",
                    help="skip the time-step measurement (newton_step key)")
    ap.add_argument("--batch-envs", type=int, default=512,
                    help="environments in the batched measurement")
    ap.add_argument("--step-layers", type=int, default=2,
                    help="--mode batchstep: tet layers through each pad's 0.5 mm thickness")
    ap.add_argument("--big-step-envs", type=int, default=512,
                    help="environments of the one-layer batched time-step measurement (0 skips it)")
    ap.add_argument("--step-envs", type=int, default=64,
                    help="environments in the batched time-step measurement")
    ap.add_argument("--dense-quads", type=int, default=256,
                    help="--mode dense_passes: gel pad quads per side (256 = the measured workload)")
    ap.add_argument("--prof-workload", default="gel", choices=["gel", "batch"],
                    help="--mode profstep: the time step captured (gel_on_terrain press, or the batched step)")
    ap.add_argument("--newton-quads", type=int, default=256,
                    help="--mode newton: gel pad quads per side (256 = the measured workload)")
    ap.add_argument("--mode", default="bench", choices=["bench", "passes", "mlp", "newton", "config1", "ccd", "batch", "batchstep", "patch",
                                                       "dualmap", "faceclip",
                                                       "mastergrad", "dense", "dense_passes", "peaks", "profstep"],
                    help="passes / mlp / newton: run --steps untimed contact passes, network "
                         "training steps or time steps (command lines for profilers); batch: "
                         "the batched measurement alone, --steps timed passes")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.mode == "passes":
        run_passes(args)
    elif args.mode == "mlp":
        run_mlp(args)
    elif args.mode == "newton":
        run_newton(args)
    elif args.mode == "dualmap":
        import torch
        print(json.dumps(dual_mesh_measurement("cuda", n_points=args.dual_points, reps=max(3, args.steps))))
    elif args.mode == "faceclip":
        import torch
        print(json.dumps(face_clip_measurement("cuda", reps=max(3, args.steps))))
    elif args.mode == "mastergrad":
        import torch
        print(json.dumps(master_grad_measurement(0, reps=max(3, args.steps))))
    elif args.mode == "dense":
        print(json.dumps(dense_measurement(0, measure_alu_peaks(0), steps=max(3, args.steps))), flush=True)
    elif args.mode == "dense_passes":
        run_dense_passes(args)
    elif args.mode == "peaks":
        print(json.dumps(measure_alu_peaks(0)), flush=True)
    elif args.mode == "patch":
        print(json.dumps(patch_measurement(0)), flush=True)
    elif args.mode == "profstep":
        run_profile_step(args)
    elif args.mode == "config1":
        print(json.dumps(config1_measurement(0)), flush=True)
    elif args.mode == "ccd":
        print(json.dumps(ccd_stress_measurement(0)), flush=True)
    elif args.mode == "batchstep":
        print(json.dumps(batched_step_measurement(0, n_env=args.step_envs, steps=max(1, args.steps),
                                                  layers=args.step_layers)), flush=True)
    elif args.mode == "batch":
        print(json.dumps(batched_measurement(0, n_env=args.batch_envs,
                                             steps=args.steps)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
