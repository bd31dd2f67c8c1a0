#!/usr/bin/env python3
"""Benchmark of the GSW-MTP hologram loop on GB300.

One step = one hologram job of the 1024^2-pupil / 1000-focus workload
(Poisson-disk foci, targets U[0.5, 1]): 100 iterations of forward MTP at the
foci, generalized weight update and inverse MTP with phase projection.
Metric: GSW-MTP iterations per second (whole job, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Our arm times K steps with CUDA events on the plan's stream, the L2 flushed
(256 MiB write) before every step; N > 1 (torchrun) runs one independent
replica per GPU (weak scaling, no collective on the data path) and reports the
max over ranks.  The reference arm times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GSW-MTP iterations/s at 1024² pupil, 1000 foci; % roofline; err vs FP64"
UNIT = "iterations/s"
WORKLOAD = "pupil1024_poisson1000"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP32 FMA peak of the CUDA cores by arithmetic (152 SMs x 128 lanes x 2 flop x 2.07 GHz),
# reported for context; the roofline uses the measured SGEMM rate (measure_gemm_peaks).
FP32_SIMT_PEAK_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu --set full
# capture of the kernel as it stands (cold caches, 1024^2 pupil, 1000 foci); an entry
# is removed whenever that kernel changes.
NCU_TRAFFIC_BYTES = {("f16x3", "forward"): 33632000, ("f16x3", "inverse"): 29405952}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def measure_gemm_peaks(torch, n: int = 8192, reps: int = 5) -> dict:
    """Dense GEMM rates measured live with cuBLAS (best of `reps`, CUDA events): FP32
    with TF32 off (the CUDA cores' FFMA rate, the peak of the plain FP32 form) and FP32
    with TF32 tensor cores on (the peak of the TF32 form).  2 n^3 flop per product."""
    a = torch.randn(n, n, device="cuda")
    b = torch.randn(n, n, device="cuda")
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    for key, tf32 in (("fp32_simt_tflops", False), ("tf32_tflops", True)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        torch.matmul(a, b)
        best = 1e30
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[key] = 2.0 * n ** 3 / (best * 1e-3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = old
    out["how"] = (f"torch.matmul fp32 {n}^3 (cuBLAS), TF32 off and on, best of {reps}, "
                  "CUDA events; 2 n^3 flop")
    return out


# ---------------------------------------------------------------- oracle legs
def oracle_leg(name: str, iters: int) -> dict:
    """Time the FP64 oracle (as it stands) for `iters` iterations of the workload."""
    import oracle as O
    from paper_2206_12661_gb300 import inputs as I
    w = I.named(name)
    fx, fy = O.plan_matrices(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length,
                             w.focus_xy)
    t0 = time.perf_counter()
    O.gsw(w.amplitude, w.phi0, fx, fy, w.target, iters)
    return {"seconds": time.perf_counter() - t0, "iters": iters}


def spawn_oracle(name: str, iters: int, cores: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-leg", name,
                        "--oracle-iters", str(iters)], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError(f"oracle leg failed: {r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(name: str, target_s: float = 15.0, max_iters: int = 100) -> dict:
    cores = os.cpu_count() or 1
    probe = spawn_oracle(name, 1, cores)
    iters = int(max(1, min(max_iters, target_s / max(probe["seconds"], 1e-3))))
    leg = spawn_oracle(name, iters, cores)
    return {"value": leg["iters"] / leg["seconds"], "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{leg['iters']} iterations of the {name} workload in FP64 numpy "
                      f"(complex128 BLAS products, {cores} threads), DFT rows built untimed"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.fh = None

    def start(self):
        try:
            self.fh = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "50", "-i", str(self.gpu)], stdout=self.fh, stderr=subprocess.DEVNULL)
            self.t0 = time.time()
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.flush()
        self.fh.seek(0)
        rows = [r.split(",") for r in self.fh.read().strip().splitlines() if r.strip()]
        self.fh.close()
        os.unlink(self.fh.name)
        sm, mx, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- distributed
def bench_config(ofa, I, torch, stream, flush, name: str, precisions, reps: int = 3) -> dict:
    """Iterations/s of each precision form on a named workload, and each form's error
    against the FP32 form on the GPU: relative L2 of |Theta| from the same phi0, and
    the differences of the final xi and uniformity after the workload's iterations."""
    w = I.named(name)
    n_iter = w.n_iter
    phi0 = torch.from_numpy(w.phi0).cuda()
    out = {"workload": name, "nx": w.nx, "ny": w.ny, "n_foci": w.n_foci,
           "iterations": n_iter, "forms": {}}
    ref = None
    for prec in precisions:
        with torch.cuda.stream(stream):
            p = ofa.Plan.from_workload(w, precision=prec, stream=stream.cuda_stream)
            th = torch.zeros(w.n_foci, 2, device="cuda")
            ofa.ofa_forward(p.handle, phi0, th, None)
            p.iterate(n_iter)
            st = p.stats()
            amp = torch.linalg.vector_norm(th.double(), dim=1).cpu().numpy()
            ms = 0.0
            for _ in range(reps):
                torch.cuda.synchronize()
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                p.iterate(n_iter)
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
            p.close()
        rec = {"iterations_per_s": reps * n_iter / (ms / 1000.0), "xi": st.xi,
               "uniformity": st.uniformity}
        if prec == "fp32":
            ref = (amp, st.xi, st.uniformity)
        if ref is not None:
            rec["amp_rel_l2_vs_fp32"] = float(np.linalg.norm(amp - ref[0]) /
                                              np.linalg.norm(ref[0]))
            rec["d_xi_vs_fp32"] = abs(st.xi - ref[1])
            rec["d_uniformity_vs_fp32"] = abs(st.uniformity - ref[2])
        out["forms"][prec] = rec
    return out


SEPARABLE_GRIDS = ("table1_grid9x9", "table1_grid45x47", "table1_random66")


def bench_separable(ofa, I, torch, stream, flush, reps: int = 3, grids=SEPARABLE_GRIDS) -> dict:
    """Table 1 geometry (1000^2 pupil) with regular 9 x 9 and 45 x 47 grids and the
    paper's 66 random spots on a 45 x 47 sampling grid: the separable grid form
    (products through the distinct focus coordinates) with FP32 products on the CUDA
    cores and with F16X3 products on the tensor cores, against the general tensor-core
    form (F16X3), iterations/s."""
    out = {}
    for name in grids:
        w = I.named(name)
        rec = {"n_foci": w.n_foci}
        for label, kw in (("separable_fp32", {"separable": 1, "precision": "fp32"}),
                          ("separable_f16x3_tc", {"separable": 1, "precision": "f16x3",
                                                  "separable_tc": 1}),
                          ("general_f16x3", {"separable": 0, "precision": "f16x3"})):
            with torch.cuda.stream(stream):
                p = ofa.Plan.from_workload(w, stream=stream.cuda_stream, **kw)
                p.iterate(w.n_iter)
                ms = 0.0
                for _ in range(reps):
                    torch.cuda.synchronize()
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    p.iterate(w.n_iter)
                    e1.record(stream)
                    e1.synchronize()
                    ms += e0.elapsed_time(e1)
                rec[label] = {"iterations_per_s": reps * w.n_iter / (ms / 1000.0),
                              "form": ofa.ofa_plan_form(p.handle), "xi": p.stats().xi}
                p.close()
        out[name] = rec
    return out


def bench_differentiation(ofa, I, torch, stream, flush, precision: str = "f16x3",
                          steps: int = 200) -> dict:
    """Adam on the focal-intensity loss (1024^2 pupil, 20x20 grid, random targets).

    One step = the library's forward (field planes, forward product, focal output),
    loss adjoint (loss and dL/dI, c_k = g_k Theta_k, inverse left operand, inverse
    product with the gradient epilogue) and Adam update: library kernels only,
    captured once as a CUDA graph and replayed.  Timed with CUDA events on the plan's
    stream after 10 warm-up steps."""
    from paper_2206_12661_gb300 import autograd as AG
    w = I.named("pupil1024_grid400_adam")
    with torch.cuda.stream(stream):
        plan = ofa.Plan.from_workload(w, precision=precision, stream=stream.cuda_stream)
        phi0 = torch.from_numpy(w.phi0).cuda()
        tgt = torch.from_numpy(w.target).cuda()
        loop = AG.AdamLoop(plan, phi0, tgt, steps + 10, lr=0.05, stream=stream, graph=True)
        loop.run(10)                                           # warm-up
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        loop.run(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        losses = loop.losses[:steps + 10].cpu().numpy()
        plan.close()
    ms = e0.elapsed_time(e1)
    flop = 2 * 8.0 * w.nx * w.ny * w.n_foci
    return {"workload": "pupil1024_grid400_adam", "precision": precision, "steps": steps,
            "adam_steps_per_s": steps / (ms / 1000.0), "ms_per_step": ms / steps,
            "tflops_products": flop * steps / (ms / 1000.0) / 1e12,
            "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
            "cuda_graph": True, "library_launches_per_step": 8,
            "step": "ofa_forward (field planes, forward, focal output), ofa_loss_adjoint (loss and dL/dI, operand build, inverse with the gradient epilogue), ofa_adam_step (update, step counter): library kernels only"}


def bench_batch(ofa, I, torch, stream, flush, n_iter: int = 50) -> dict:
    """256 holograms, pupils 512^2 / 768^2 / 1024^2, 16..4096 foci (log-uniform),
    jittered grids, 50 iterations: the grouped batch (f16x3), the same plans run
    plan after plan, each hologram as one persistent fused-loop launch (plan after
    plan), and the plain FP32 form plan after plan.  Unit: hologram
    iterations per second.  Timed with CUDA events on one stream after a warm-up."""
    ws = I.batch_workloads(count=256, n_iter=n_iter, seed=5)
    flop = sum(16.0 * w.nx * w.ny * w.n_foci for w in ws) * n_iter
    units = len(ws) * n_iter
    out = {"workload": "256 holograms, N in {512, 768, 1024}, K log-uniform 16..4096, "
                       f"{n_iter} iterations each, seed 5", "holograms": len(ws),
           "iterations": n_iter, "unit": "hologram-iterations/s",
           "flop_per_run": flop}

    def timed(fn):
        torch.cuda.synchronize()
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0

    plans = [ofa.Plan.from_workload(w, precision="f16x3", stream=stream.cuda_stream,
                                    autotune=False) for w in ws]
    b = ofa.ofa_batch_create([p.handle for p in plans], stream.cuda_stream)
    out["grouped"] = ofa.ofa_batch_info(b)
    ofa.ofa_batch_iterate(b, 2)                        # warm-up (graph for 2)
    ofa.ofa_batch_iterate(b, n_iter)                   # builds the n-iteration graph
    t = timed(lambda: ofa.ofa_batch_iterate(b, n_iter))
    ofa.ofa_batch_destroy(b)
    out["batched_f16x3"] = units / t
    out["batched_tflops"] = flop / t / 1e12
    for p in plans:
        p.iterate(1)
    t = timed(lambda: [p.iterate(n_iter) for p in plans])
    out["plan_after_plan_f16x3"] = units / t
    for p in plans:
        p.close()
    # the persistent form: each hologram's iterations in one cooperative launch of the
    # fused loop kernel (grid barriers between the phases), hologram after hologram
    loops = [ofa.Plan.from_workload(w, precision="f16x3", stream=stream.cuda_stream,
                                    autotune=False, fused_loop=1) for w in ws]
    out["persistent_loop_holograms"] = sum(
        ofa.ofa_plan_config(p.handle)["fused_loop"] == 1 for p in loops)
    for p in loops:
        p.iterate(1)
    t = timed(lambda: [p.iterate(n_iter) for p in loops])
    out["persistent_loop_plan_after_plan_f16x3"] = units / t
    for p in loops:
        p.close()
    fp32 = [ofa.Plan.from_workload(w, precision="fp32", stream=stream.cuda_stream)
            for w in ws]
    for p in fp32:
        p.iterate(1)
    t = timed(lambda: [p.iterate(n_iter) for p in fp32])
    out["plain_fp32_plan_after_plan"] = units / t
    for p in fp32:
        p.close()
    return out


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks (every rank gets it); x itself without a group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world: int, steps: int, iters_per_step: int, slowest_ms: float) -> float:
    """Whole-job iterations/s: every rank's iterations over the slowest rank's time."""
    return world * steps * iters_per_step / (slowest_ms / 1000.0)


def run_reference(args, world, rank):
    """FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    probe = spawn_oracle(WORKLOAD, 1, cores)
    # each step: a bounded sample of the job, about 1-2 s of CPU work
    per_step = int(max(1, min(100, 1.5 / max(probe["seconds"], 1e-3))))
    for _ in range(args.warmup):
        spawn_oracle(WORKLOAD, 1, cores)
    total_s, total_it = 0.0, 0
    for _ in range(args.steps):
        leg = spawn_oracle(WORKLOAD, per_step, cores)
        total_s += leg["seconds"]
        total_it += leg["iters"]
    value = total_it / total_s
    sample = (f"{per_step} iterations per step of the {WORKLOAD} workload in FP64 numpy "
              f"({cores} threads; one 100-iteration job per step is the GPU arm's unit)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nx": 1024, "ny": 1024, "n_foci": 1000,
                       "iterations_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16x3")
    ap.add_argument("--iters-per-step", type=int, default=100)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel-config", default=None,
                    help="force the tensor-core tiles: fwd_bn,fwd_split,fwd_cg,inv_bn,inv_cg "
                         "(as ofa_options.kernel_config; default: the plan's autotuner)")
    ap.add_argument("--separable-grid", default=None, choices=list(SEPARABLE_GRIDS),
                    help="with --only separable: time this Table 1 grid alone")
    ap.add_argument("--only", default=None,
                    choices=["differentiation", "batch", "separable", "configs"],
                    help="run one of the extra sections alone and print its JSON (for "
                         "profiling runs; no timed loop, not a bench line)")
    ap.add_argument("--oracle-leg", default=None)
    ap.add_argument("--oracle-iters", type=int, default=1)
    args = ap.parse_args()

    if args.oracle_leg:
        print(json.dumps(oracle_leg(args.oracle_leg, args.oracle_iters)), flush=True)
        return 0

    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    from paper_2206_12661_gb300 import _build
    _build.build()
    from paper_2206_12661_gb300 import inputs as I
    from paper_2206_12661_gb300 import ofa

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    w = I.named(WORKLOAD)
    n_iter = args.iters_per_step
    stream = torch.cuda.Stream()
    if args.only:
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        sections = {
            "differentiation": lambda: bench_differentiation(ofa, I, torch, stream, flush),
            "batch": lambda: bench_batch(ofa, I, torch, stream, flush),
            "separable": lambda: bench_separable(
                ofa, I, torch, stream, flush,
                grids=(args.separable_grid,) if args.separable_grid else SEPARABLE_GRIDS),
            "configs": lambda: [bench_config(ofa, I, torch, stream, flush,
                                             "pupil256_grid100_uniform", ("fp32", "f16x3"))]}
        print(json.dumps({"section": args.only, args.only: sections[args.only]()}),
              flush=True)
        return 0
    forced = ([int(x) for x in args.kernel_config.split(",")] if args.kernel_config
              else None)
    plan = ofa.Plan.from_workload(w, precision=args.precision, stream=stream.cuda_stream,
                                  kernel_config=forced)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        plan.iterate(n_iter)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for e0, e1 in ev:
            flush.zero_()             # write > L2 so every step starts from a cold L2
            e0.record(stream)
            plan.iterate(n_iter)
            e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), pg, device="cuda")
    value = job_value(world, args.steps, n_iter, total_ms)

    # live per-kernel timing (CUDA events on the plan's stream) for the roofline
    kms = ofa.ofa_profile_kernels(plan.handle, reps=50)
    kernel_config = ofa.ofa_plan_config(plan.handle)
    peaks, peak_src = load_peaks()
    live = measure_gemm_peaks(torch)
    flops_per_product = 8.0 * w.nx * w.ny * w.n_foci
    dom = int(np.argmax([kms[0], kms[3]]))
    dom_ms = kms[0] if dom == 0 else kms[3]
    achieved = flops_per_product / (dom_ms * 1e-3) / 1e12
    if args.precision == "fp32":
        roof = {"bound": "alu", "peak": live["fp32_simt_tflops"],
                "peak_source": "measured in this run: cuBLAS SGEMM 8192^3 (TF32 off); "
                               f"derived FFMA peak {FP32_SIMT_PEAK_DERIVED_TFLOPS:.1f} TFLOP/s"}
    elif args.precision == "tf32":
        roof = {"bound": "tensor", "peak": live["tf32_tflops"],
                "peak_source": "measured in this run: cuBLAS TF32 8192^3"}
    else:
        roof = {"bound": "tensor", "peak": peaks["bf16_tflops"],
                "peak_source": f"{peak_src} bf16 dense burst (kernel timed alone)"}
    roofline = {"bound": roof["bound"], "achieved": achieved, "peak": roof["peak"],
                "unit": "TFLOP/s", "frac": achieved / roof["peak"],
                "traffic": NCU_TRAFFIC_BYTES.get((args.precision,
                                                  "forward" if dom == 0 else "inverse")),
                "kernel": "forward product + per-focus dot" if dom == 0
                else "inverse product + phase projection",
                "algorithmic_flop_per_launch": flops_per_product,
                "kernel_ms": {"forward": kms[0], "focal": kms[1], "p_build": kms[2],
                              "inverse": kms[3]},
                "peak_source": roof["peak_source"],
                "passes": 3 if args.precision in ("f16x3", "bf16x3") else 1}

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup,
              "ms_per_step": total_ms / args.steps, "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
              "data": "synthetic",
              "config": {"workload": WORKLOAD, "nx": w.nx, "ny": w.ny, "n_foci": w.n_foci,
                         "iterations_per_step": n_iter, "precision": args.precision,
                         "foci": "Poisson disk, 3-spot min spacing, 2.0 mm ROI",
                         "l2": "flushed (256 MiB write) before every step; inputs "
                               "(about 45 MB) stay L2-resident within a step",
                         "parallelism": f"replicas x{world}",
                         "kernels": kernel_config},
              "roofline": roofline, "clocks": clocks,
              "peaks": {"bf16_tflops": peaks["bf16_tflops"], "bf16_source": peak_src,
                        **{k: v for k, v in live.items()}}}
    # forward (+ the focal step in its last block: up to 2048 foci in the FP32 form,
    # 4096 in the tensor-core forms; else a separate focal kernel), inverse operand
    # build, inverse
    fused_limit = 2048 if args.precision == "fp32" else 4096
    kernels_per_iter = 3 if w.n_foci <= fused_limit else 4
    result["gpu_launches"] = args.steps * (n_iter * kernels_per_iter + 1)

    if rank == 0 and not args.no_e2e:
        # end to end through the C ABI with host buffers: create (H2D of foci, targets,
        # A, phi0), iterate, read phi back (D2H), destroy.  The host inputs and the
        # result buffer are pinned (allocated once, before the timed region).
        def pinned(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        xy_h = pinned(w.focus_xy.astype(np.float64))
        t_h = pinned(w.target.astype(np.float32))
        amp_h = pinned(w.amplitude.astype(np.float32))
        phi0_h = pinned(w.phi0.astype(np.float32))
        phi = torch.empty((w.ny, w.nx), dtype=torch.float32).pin_memory().numpy()

        def job():
            p = ofa.Plan(w.nx, w.ny, w.pitch_x, w.pitch_y, w.wavelength, w.focal_length, xy_h,
                         t_h, precision=args.precision, amplitude=amp_h, phi0=phi0_h)
            p.iterate(n_iter)
            ofa.ofa_get_phase(p.handle, phi, ofa.OFA_MEM_HOST)
            p.close()

        reps = max(1, min(5, args.steps))
        job()  # warm
        t = 0.0
        for _ in range(reps):
            t0 = time.perf_counter()
            job()
            t += time.perf_counter() - t0
        h2d = xy_h.nbytes + t_h.nbytes + amp_h.nbytes + phi0_h.nbytes
        d2h = phi.nbytes
        result["e2e"] = {"value": reps * n_iter / t, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h,
                         "step": "one hologram job: plan create from pinned host arrays, "
                                 f"{n_iter} iterations, phase read back to pinned host "
                                 "memory, destroy"}

    if rank == 0 and not args.no_forms:
        forms = {}
        for prec in ("fp32", "tf32", "bf16", "bf16x3", "f16x3"):
            p = ofa.Plan.from_workload(w, precision=prec, stream=stream.cuda_stream)
            reps = 2 if prec == "fp32" else 10
            p.iterate(n_iter)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = 0.0
            for _ in range(reps):
                flush.zero_()
                e0.record(stream)
                p.iterate(n_iter)
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
            k = ofa.ofa_profile_kernels(p.handle, reps=10 if prec == "fp32" else 50)
            its = reps * n_iter / (ms / 1000.0)
            # each form against the peak of the pipe it runs on (measured); the split
            # forms' extra products are overhead, not credit
            pk = {"fp32": live["fp32_simt_tflops"], "tf32": live["tf32_tflops"]}.get(
                prec, peaks["bf16_tflops"])
            loop_tflops = 2 * flops_per_product * its / 1e12
            forms[prec] = {"iterations_per_s": its,
                           "kernel_ms": [round(x, 5) for x in k],
                           "loop_tflops": loop_tflops,
                           "peak_tflops": pk,
                           "loop_frac_of_own_peak": loop_tflops / pk,
                           "kernels": ofa.ofa_plan_config(p.handle)}
            p.close()
        result["forms"] = forms
        # the opt-in fused loop (one persistent launch per call) on the same workload
        fl = {}
        for prec in ("f16x3", "bf16"):
            p = ofa.Plan.from_workload(w, precision=prec, stream=stream.cuda_stream,
                                       fused_loop=1)
            p.iterate(n_iter)
            ms_it, ph = ofa.ofa_profile_loop(p.handle, n_iter=n_iter, reps=3, phases=True)
            fl[prec] = {"iterations_per_s": 1.0 / (ms_it * 1e-3),
                        "phase_us_cta0": {k2: round(v, 2) for k2, v in ph.items()},
                        "config": {k2: v for k2, v in ofa.ofa_plan_config(p.handle).items()
                                   if k2.startswith("loop") or k2 == "fused_loop"}}
            p.close()
        result["fused_loop"] = fl
        result["differentiation"] = bench_differentiation(ofa, I, torch, stream, flush)
        all_forms = ("fp32", "tf32", "bf16", "bf16x3", "f16x3")
        result["configs"] = [
            bench_config(ofa, I, torch, stream, flush, "pupil256_grid100_uniform",
                         ("fp32", "f16x3")),
            bench_config(ofa, I, torch, stream, flush, WORKLOAD, all_forms, reps=1),
            bench_config(ofa, I, torch, stream, flush, "pupil1920x1152_grid2500", all_forms),
        ]
        result["batch"] = bench_batch(ofa, I, torch, stream, flush)
        result["separable"] = bench_separable(ofa, I, torch, stream, flush)

    plan.close()
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(WORKLOAD)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
