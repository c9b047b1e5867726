"""Benchmark: WMG-preconditioned Krylov reconstructions per second to a 1e-4
relative normal-equation residual on the 256x256 parallel-beam workload
(180 angles, 363 detector bins, seeded 20-ellipse phantoms, 1% Gaussian
noise, 5 WMG levels), solved by restarted GMRES(20) with right
preconditioning by the paper's WMG cycle (hybrid residual update at depth 0,
no smoothing sweeps), FP32 operator with FP64 Krylov vectors and reductions.
Further legs of the same run (the smoothed cycle, BiCGStab, Joseph's kernel,
the semi-convergence study, 1024^2, an uneven batch, a request stream, the
stored-matrix comparator) are reported beside the headline.

One step = one batch of `--batch` independent reconstructions (distinct
phantoms and noise), all iterated together until each reaches the tolerance.
The plan (geometry, smoother diagonal, leaf inverses) is built once for the
geometry and reused by every step; its setup time is reported separately.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B]
                       [--impl ours|reference]
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (one reconstruction, setup excluded) and prints the same JSON line.
Under torchrun (N > 1) every rank solves its own batch (replicas, no
communication); the value is the total over ranks divided by the slowest
rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synthetic as S  # noqa: E402

METRIC = "WMG-Krylov recon/s to 1e-4 residual"
RTOL = 1e-4
MAX_ITER = 200
RESTART = 20
# WMG cycle of the measured runs: the paper's cycle (Section 3.1.2: no
# smoothing sweeps, nu1 = nu2 = 0) with the hybrid residual update at depth 0.
# The smoothed cycle (one l1-Jacobi pre- and post-sweep) is measured beside it.
LEVELS, NU1, NU2, HYB = 5, 0, 0, 1
NU_SMOOTHED = 1
# Tikhonov parameters of the semi-convergence leg's sweep, relative to m / n
LAMBDA_SWEEP = (0.0, 1e-4, 1e-3, 1e-2, 1e-1)
# problems of the plain FP64 one-problem-per-launch comparison arms
FP64_SAMPLE = 8
# serving stream: Tikhonov parameter relative to m / n, the scale of the
# spectral radius of W^T W in unit-square units (noisy, often underdetermined
# requests; regularised normal equations as in the paper's noisy experiments)
SERVING_EPS = 1e-3
# arrival rate of the full-size request stream (requests/s): 0.7 x the
# saturated throughput measured once with --serving-burst, then fixed
SERVING_RATE_FULL = 0.7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256,
                    help="reconstructions per step and GPU (throughput grows with the batch: 704 / 753 / 782 "
                         "recon/s at 64 / 128 / 256 on GB300)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving leg (request stream through the continuous-batching server)")
    ap.add_argument("--serving-requests", type=int, default=40,
                    help="requests of the full-size stream (n 128 .. 2048, m 90 .. 720)")
    ap.add_argument("--serving-rate", type=float, default=SERVING_RATE_FULL,
                    help="mean arrivals per second (Poisson) of the full-size stream: 0.7 x its saturated "
                         "throughput measured once")
    ap.add_argument("--serving-max-n", type=int, default=2048,
                    help="largest image side of the stream (sizes 128 .. 2048 in the configured stream)")
    ap.add_argument("--serving-small-requests", type=int, default=48,
                    help="requests of the second stream, restricted to n <= 512 (0: skip it)")
    ap.add_argument("--serving-small-rate", type=float, default=8.0,
                    help="mean arrivals per second of the n <= 512 stream (0.7 x its saturated throughput)")
    ap.add_argument("--serving-only", action="store_true", help="run the serving leg alone and print its JSON")
    ap.add_argument("--serving-burst", action="store_true",
                    help="serving leg with every request arriving at t = 0 (saturated throughput)")
    ap.add_argument("--no-batched", action="store_true", help="skip the uneven-batch leg")
    ap.add_argument("--no-comparator", action="store_true", help="skip the stored-W (CSR) comparator leg")
    ap.add_argument("--no-fp64-single", action="store_true",
                    help="skip the plain FP64 one-problem-per-launch arm of the main workload")
    ap.add_argument("--no-variant", action="store_true",
                    help="skip the smoothed-cycle variant (nu1 = nu2 = 1) of the main workload")
    ap.add_argument("--no-joseph", action="store_true",
                    help="skip the leg with Joseph's kernel as W (same batch and solver)")
    ap.add_argument("--no-semiconv", action="store_true",
                    help="skip the semi-convergence leg (160^2, 400 angles, Joseph's kernel, noisy data)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 1024x1024 / 1024-angle leg (mixed FP32 path vs the FP64 GPU path)")
    ap.add_argument("--solve-case", action="store_true",
                    help="run three solves of the workload batch and exit: the case for ncu captures of the "
                         "solve's secondary kernels (Gram-Schmidt, leaf solves, Haar packets)")
    ap.add_argument("--setup-case", default=None, metavar="N:M",
                    help="create one FP32 plan of an N x N image and M angles (detectors and levels by the "
                         "uneven-batch rule, hybrid depth 1), print its setup time and exit: the case for "
                         "ncu launch lists of the leaf setup")
    ap.add_argument("--batched-case", action="store_true",
                    help="solve the uneven batch four times (one warm-up) and exit: the case for ncu launch lists")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run 3 projector and 3 backprojector launches on a batch of --kernel-images images "
                         "of the workload geometry (FP32) and exit: the small case for ncu captures")
    ap.add_argument("--kernel-images", type=int, default=16,
                    help="images of the --kernel-case batch (16: 2 group tiles per angle and ray block)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_problems(batch: int, rank: int):
    """Rank `rank`'s shard: problems batch*rank .. batch*(rank+1)-1 of the
    workload's seeded problem sequence (disjoint across ranks)."""
    return S.workload_mid(batch * (rank + 1)).problems[batch * rank: batch * (rank + 1)]


def max_over_ranks(t: float, world: int, device=None) -> float:
    """The largest of the ranks' values, on every rank (the job is as slow as
    its slowest replica)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_value(batch: int, world: int, steps: int, t_total: float) -> float:
    """Reconstructions per second of the whole job: every rank solved `steps`
    batches of `batch` problems in at most t_total seconds."""
    return batch * world * steps / t_total


# ---------------------------------------------------------------------------
# CPU oracle baseline (one reconstruction of the workload, FP64, 1 thread)
# ---------------------------------------------------------------------------
def host_cpu() -> dict:
    """The host's CPU model, logical core count and the cores this process
    may run on."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "processor name"):
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
    try:
        allowed = len(os.sched_getaffinity(0))
    except AttributeError:
        allowed = os.cpu_count()
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count(), "cores_allowed": allowed}


_ORACLE_BARRIER = None


def _oracle_worker_init(barrier):
    global _ORACLE_BARRIER
    _ORACLE_BARRIER = barrier


def _oracle_solve(seed_index: int, cpu: int) -> dict:
    """One oracle reconstruction of problem `seed_index` of the workload,
    pinned to host core `cpu`: plan setup, then (after every worker of the
    pool has finished its setup) the timed WMG-GMRES(20) solve."""
    import oracle
    try:
        os.sched_setaffinity(0, {cpu})
        pinned = True
    except (AttributeError, OSError):
        pinned = False
    problem = workload_problems(seed_index + 1, 0)[seed_index]
    op = oracle.Op(problem.n, problem.m, problem.D)
    b0 = op.project(problem.image())
    b = b0 + problem.noise * np.abs(b0).max() * problem.noise_unit()
    t0 = time.perf_counter()
    M = oracle.Wmg(op, LEVELS, NU1, NU2, 1.0, 0.0, oracle.CYCLE_HYBRID, HYB)
    setup = time.perf_counter() - t0
    if _ORACLE_BARRIER is not None:
        _ORACLE_BARRIER.wait()
    t_start = time.time()
    t0 = time.perf_counter()
    x, k, hist = oracle.gmres(op, b, MAX_ITER, RESTART, RTOL, 0.0, M)
    solve = time.perf_counter() - t0
    return {"solve_s": solve, "setup_s": setup, "iters": int(k), "seed": problem.seed, "pinned": pinned,
            "start": t_start, "end": time.time()}


def cpu_baseline(problem, all_cores: bool = True) -> dict:
    """The oracle timed on the host: one reconstruction pinned to one core,
    and (all_cores) one reconstruction per allowed core run at once, each
    pinned to its core (independent problems; recon/s = reconstructions /
    the span from the first solve's start to the last one's end). Plan setup
    is excluded like the GPU plan's. Runs in spawned processes (the calling
    process holds a CUDA context)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    info = host_cpu()
    try:
        cores = sorted(os.sched_getaffinity(0))
    except AttributeError:
        cores = list(range(os.cpu_count() or 1))
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(1, mp_context=ctx) as ex:
        one = ex.submit(_oracle_solve, 0, cores[0]).result()
    line = {"value": 1.0 / one["solve_s"], "unit": "recon/s", "cores": 1, "kind": "oracle",
            "sample": (f"1 reconstruction of the workload (problem seed {one['seed']}): WMG-GMRES(20) "
                       f"to {RTOL:g} in {one['iters']} iterations, {one['solve_s']:.1f} s on one core"
                       f"{' (pinned)' if one['pinned'] else ''}; plan setup {one['setup_s']:.1f} s excluded "
                       "like the GPU plan's"),
            "iters": one["iters"], "setup_s": one["setup_s"], **info}
    if all_cores and len(cores) > 1:
        n = len(cores)
        barrier = ctx.Barrier(n)
        with cf.ProcessPoolExecutor(n, mp_context=ctx, initializer=_oracle_worker_init,
                                    initargs=(barrier,)) as ex:
            rs = list(ex.map(_oracle_solve, range(n), cores))
        span = max(r["end"] for r in rs) - min(r["start"] for r in rs)
        line["all_cores"] = {"value": n / span, "unit": "recon/s", "cores": n,
                             "sample": f"{n} independent reconstructions (problems 0..{n - 1}), one per core, "
                                       f"solved at once; mean {np.mean([r['solve_s'] for r in rs]):.1f} s each"}
    return line


def run_reference(args, rank, world):
    if rank != 0:
        return
    P = workload_problems(1, 0)[0]
    per = []
    base = None
    for _ in range(max(1, args.warmup and 0) + args.steps):
        base = cpu_baseline(P, all_cores=False)
        per.append(1.0 / base["value"])
    t = float(np.mean(per))
    val = 1.0 / t
    line = {"metric": METRIC, "value": val, "unit": "recon/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "256x256_180ang_363det_noise1pct", "batch": 1, "solver": "WMG-GMRES(20)",
                       "levels": LEVELS, "precision": "fp64 oracle (CPU)"},
            "cpu_baseline": {"value": val, "unit": "recon/s", "cores": 1, "kind": "oracle",
                             "sample": base["sample"], **host_cpu()},
            "e2e": {"value": val, "unit": "recon/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU run
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # raw samples go to $WMG_BENCH_OUT (default bench_out/ beside this file)
        out_dir = os.environ.get("WMG_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args, rank, world, local):
    import torch
    import paper_1310_0956_gb300 as wmg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    probs = workload_problems(args.batch, rank)
    P0 = probs[0]
    B = len(probs)
    N, M = P0.N, P0.M

    # plan: built once for the geometry (timed separately)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = wmg.Plan(P0.n, P0.m, P0.D, levels=LEVELS, nu1=NU1, nu2=NU2, hybrid_depth=HYB,
                    cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0

    # synthetic inputs, resident in HBM: b = W x_phantom (FP64 library
    # projector) + sigma * N(0,1), sigma = 1% of max|W x|
    plan64 = wmg.Plan(P0.n, P0.m, P0.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE,
                      precision=wmg.PREC_F64)
    imgs = torch.tensor(np.stack([p.image() for p in probs]).reshape(-1), dtype=torch.float64, device=dev)
    b64 = plan64.project(imgs).view(B, M)
    noise = torch.tensor(np.stack([p.noise_unit() for p in probs]), dtype=torch.float64, device=dev)
    sigma = torch.tensor([p.noise for p in probs], dtype=torch.float64, device=dev)[:, None] * \
        b64.abs().amax(dim=1, keepdim=True)
    b = (b64 + sigma * noise).to(torch.float32).contiguous().view(-1)
    plan64.close()
    del imgs, b64, noise
    x = torch.empty(B * N, dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step():
        _, info, _, rc = plan.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=x)
        return info, rc

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wmg.wmg_launch_count(True)
    sampler.start()
    times, iters, statuses = [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)                              # evict L2 between steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info, rc = step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
        iters.extend(i[0] for i in info)
        statuses.extend(i[1] for i in info)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    launches = wmg.wmg_launch_count(False)
    t_step = float(np.mean(times))
    t_total = float(np.sum(times))
    if world > 1:
        t_total = max_over_ranks(t_total, world, dev)
        torch.distributed.barrier()
    value = whole_job_value(B, world, args.steps, t_total)

    # the smoothed cycle on the same batch (one l1-Jacobi pre- and post-sweep:
    # two more A-pairs per iteration, fewer iterations)
    variant = None
    if not args.no_variant:
        plan_s = wmg.Plan(P0.n, P0.m, P0.D, levels=LEVELS, nu1=NU_SMOOTHED, nu2=NU_SMOOTHED, hybrid_depth=HYB,
                          cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
        xs_ = torch.empty_like(x)
        for _ in range(2):
            plan_s.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=xs_)
        vt, vit = [], []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, vinfo, _, _ = plan_s.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=xs_)
            e1.record(stream)
            torch.cuda.synchronize()
            vt.append(e0.elapsed_time(e1) / 1e3)
            vit.extend(i[0] for i in vinfo)
        plan_s.close()
        variant = {"cycle": f"hybrid depth {HYB}, nu1=nu2={NU_SMOOTHED} (l1-Jacobi)",
                   "recon_per_s": B / float(np.mean(vt)), "iters_mean": float(np.mean(vit)),
                   "ms_per_step": float(np.mean(vt)) * 1e3}
        # the paper's own Krylov solver on the same batch and cycle
        xb_ = torch.empty_like(x)
        plan.solve(b, wmg.SOLVER_BICGSTAB, True, MAX_ITER, RTOL, RESTART, out=xb_)
        bt_, bit_, bst_ = [], [], []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, binfo, _, _ = plan.solve(b, wmg.SOLVER_BICGSTAB, True, MAX_ITER, RTOL, RESTART, out=xb_)
            e1.record(stream)
            torch.cuda.synchronize()
            bt_.append(e0.elapsed_time(e1) / 1e3)
            bit_.extend(i[0] for i in binfo)
            bst_.extend(i[1] for i in binfo)
        # the fully multiplicative WTG (eq. wmg) at the root: three band-local
        # residual updates per cycle instead of the hybrid rule's one
        plan_m = wmg.Plan(P0.n, P0.m, P0.D, levels=LEVELS, nu1=NU1, nu2=NU2, hybrid_depth=HYB,
                          cycle=wmg.CYCLE_MULTIPLICATIVE, precision=wmg.PREC_F32)
        plan_m.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=xs_)
        mt, mit, mst = [], [], []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, minfo, _, _ = plan_m.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=xs_)
            e1.record(stream)
            torch.cuda.synchronize()
            mt.append(e0.elapsed_time(e1) / 1e3)
            mit.extend(i[0] for i in minfo)
            mst.extend(i[1] for i in minfo)
        plan_m.close()
        variant["multiplicative"] = {"cycle": f"fully multiplicative WTG (eq. wmg) at depth < {HYB}, nu1=nu2={NU1}",
                                     "recon_per_s": B / float(np.mean(mt)), "iters_mean": float(np.mean(mit)),
                                     "all_converged": bool(all(s_ == 0 for s_ in mst))}
        variant["bicgstab"] = {"solver": "WMG-BiCGStab (right preconditioning), the paper's cycle",
                               "recon_per_s": B / float(np.mean(bt_)), "iters_mean": float(np.mean(bit_)),
                               "all_converged": bool(all(s_ == 0 for s_ in bst_))}

    # end-to-end: the same solve through the C ABI with HOST (pinned) buffers,
    # host->device copy of the sinograms and device->host copy of the images
    # inside the timed region
    b_host = b.cpu().pin_memory()
    x_host = torch.empty(B * N, dtype=torch.float32).pin_memory()
    b_dev = torch.empty_like(b)
    e2e_times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b_dev.copy_(b_host, non_blocking=True)
        plan.solve(b_dev, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=x)
        x_host.copy_(x, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_times.append(e0.elapsed_time(e1) / 1e3)
    e2e_val = B * world / float(np.mean(e2e_times))

    # the plain form: FP64, one problem per launch, the same cycle and solver
    single = None
    if rank == 0 and not args.no_fp64_single:
        try:
            ns = min(FP64_SAMPLE, B)
            single = fp64_single_leg([dict(n=P0.n, m=P0.m, D=P0.D, levels=LEVELS)] * ns,
                                     [b.view(B, M)[i].double().contiguous() for i in range(ns)],
                                     wmg.SOLVER_GMRES, HYB, wmg.CYCLE_HYBRID,
                                     [x.view(B, N)[i].double() for i in range(ns)], dev)
            single["mixed_batched_over_fp64_single"] = value / world / single["recon_per_s"]
        except Exception as e:
            single = {"unavailable": f"{type(e).__name__}: {e}"}

    # dominant-kernel timing: projector and backprojector launches of one
    # profiled step (CUDA events around every launch on the plan's stream)
    prof = plan.profile_step(b, x, MAX_ITER, RTOL, RESTART)
    roofline = None
    if prof:
        peaks = {name: wmg.wmg_measure_peak(kind) for name, kind in
                 (("fp32_fma", wmg.PEAK_FP32_FMA), ("fp32_fma_paired", wmg.PEAK_FP32_FMA2),
                  ("fp64_fma", wmg.PEAK_FP64_FMA))}
        prof["fp32_fma_tflops_measured"] = max(peaks["fp32_fma"], peaks["fp32_fma_paired"])
        roofline = roofline_entry(prof, P0, B)
        roofline["measured_peaks_tflops"] = peaks
        roofline["operator_launches"] = {k: {"launches": prof[k]["launches"], "mean_ms": prof[k]["mean_ms"],
                                             "images_per_launch": prof[k]["images_per_launch"]}
                                         for k in ("project", "backproject", "project_2h")}
    comparator = None
    if not args.no_comparator and rank == 0:
        try:
            comparator = comparator_leg(plan, P0, x, b, flush, dev)
            if roofline is not None:
                roofline["fp32_sgemm_tflops_measured"] = comparator["fp32_sgemm_tflops_measured"]
        except Exception as e:
            comparator = {"unavailable": f"{type(e).__name__}: {e}"}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            try:
                cpu = cpu_baseline(P0)
                cpu.pop("iters", None)
                cpu.pop("setup_s", None)
            except Exception as e:  # the oracle is a baseline, never the product path
                cpu = {"value": None, "unit": "recon/s", "cores": 1, "kind": "oracle",
                       "sample": f"unavailable: {e}"}
        line = {
            "metric": METRIC, "value": value, "unit": "recon/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "256x256_180ang_363det_noise1pct", "batch_per_gpu": B,
                       "solver": f"WMG-GMRES(20), hybrid cycle depth {HYB}, nu1=nu2={NU1} (the paper's WMG: "
                                 "no smoothing)", "levels": LEVELS,
                       "precision": "fp32 operator and leaf solves, fp64 Krylov vectors/reductions/Gram-Schmidt",
                       "rtol": RTOL, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "iters_mean": float(np.mean(iters)), "iters_max": int(np.max(iters)),
                       "all_converged": bool(all(s == 0 for s in statuses)),
                       "plan_setup_s": setup_s,
                       "launch_shapes_ctas_per_sm": dict(zip(("project", "backproject"), plan.tuning()))},
            "clocks": clocks,
            "e2e": {"value": e2e_val, "unit": "recon/s", "h2d_bytes_per_step": int(B * M * 4),
                    "d2h_bytes_per_step": int(B * N * 4)},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "stored_w_comparator": comparator,
            "smoothed_cycle_variant": variant,
            "fp64_one_problem_per_launch": single,
        }
        if not args.no_joseph and world == 1:
            try:
                line["joseph_kernel"] = joseph_leg(args, dev, probs, flush)
            except Exception as e:
                line["joseph_kernel"] = {"unavailable": f"{type(e).__name__}: {e}"}
        if not args.no_semiconv and world == 1:
            try:
                line["semiconvergence"] = semiconvergence_leg(dev)
            except Exception as e:
                line["semiconvergence"] = {"unavailable": f"{type(e).__name__}: {e}"}
        if not args.no_large and world == 1:
            try:
                line["large"] = large_leg(dev)
            except Exception as e:
                line["large"] = {"unavailable": f"{type(e).__name__}: {e}"}
        if not args.no_batched and world == 1:
            try:
                line["batched"] = batched_leg(args, dev)
            except Exception as e:
                line["batched"] = {"unavailable": f"{type(e).__name__}: {e}"}
        if not args.no_serving and world == 1:
            try:
                line["serving"] = serving_leg(args, dev)
                line["serving"]["setup_s_per_geometry"] = setup_times(((1024, 405), (2048, 405)))
            except Exception as e:
                line["serving"] = {"unavailable": f"{type(e).__name__}: {e}"}
            if args.serving_small_requests > 0:
                try:
                    line["serving_n_le_512"] = serving_leg(args, dev, args.serving_small_requests, 512,
                                                           args.serving_small_rate)
                except Exception as e:
                    line["serving_n_le_512"] = {"unavailable": f"{type(e).__name__}: {e}"}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# Joseph leg: the same batch and solver with W = Joseph's interpolating kernel
# (the paper's projector, Section 2.1) in place of exact intersection lengths
# ---------------------------------------------------------------------------
def joseph_leg(args, dev, probs, flush) -> dict:
    import torch
    import paper_1310_0956_gb300 as wmg
    P0 = probs[0]
    B, N, M = len(probs), P0.N, P0.M
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = wmg.Plan(P0.n, P0.m, P0.D, levels=LEVELS, nu1=NU1, nu2=NU2, hybrid_depth=HYB,
                    cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32, kernel=wmg.KERNEL_JOSEPH)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    plan64 = wmg.Plan(P0.n, P0.m, P0.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE,
                      precision=wmg.PREC_F64, kernel=wmg.KERNEL_JOSEPH)
    imgs = torch.tensor(np.stack([p.image() for p in probs]).reshape(-1), dtype=torch.float64, device=dev)
    b64 = plan64.project(imgs).view(B, M)
    noise = torch.tensor(np.stack([p.noise_unit() for p in probs]), dtype=torch.float64, device=dev)
    sigma = torch.tensor([p.noise for p in probs], dtype=torch.float64, device=dev)[:, None] * \
        b64.abs().amax(dim=1, keepdim=True)
    b = (b64 + sigma * noise).to(torch.float32).contiguous().view(-1)
    plan64.close()
    del imgs, b64, noise
    x = torch.empty(B * N, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        plan.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=x)
    ts, its, sts = [], [], []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, info, _, _ = plan.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=x)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
        its.extend(i[0] for i in info)
        sts.extend(i[1] for i in info)
    prof = plan.profile_step(b, x, MAX_ITER, RTOL, RESTART)
    out = {"workload": "256x256_180ang_363det_noise1pct, W = Joseph's kernel", "problems": B,
           "solver": f"WMG-GMRES(20), hybrid cycle depth {HYB}, nu1=nu2={NU1}", "recon_per_s": B / float(np.mean(ts)),
           "ms_per_step": float(np.mean(ts)) * 1e3, "iters_mean": float(np.mean(its)),
           "all_converged": bool(all(s_ == 0 for s_ in sts)), "plan_setup_s": setup_s,
           "nnz_per_image": prof["nnz_per_image"],
           "project_ms_per_launch": prof["project"]["mean_ms"],
           "backproject_ms_per_launch": prof["backproject"]["mean_ms"]}
    plan.close()
    return out


# ---------------------------------------------------------------------------
# Semi-convergence leg (Section 4.2): the error of the k-th iterate against the
# exact phantom for SIRT, BiCGStab and WMG-BiCGStab, without and with Tikhonov
# regularisation, on the paper's noisy model problem sizes
# ---------------------------------------------------------------------------
def semiconvergence_leg(dev) -> dict:
    import torch
    import paper_1310_0956_gb300 as wmg
    from paper_1310_0956_gb300 import study
    n, m, D, levels = 160, 400, 160, 5
    x = S.phantom(n, 12, S.seed_for(6, 0))
    xd = torch.tensor(x.reshape(-1), dtype=torch.float32, device=dev)
    p64 = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64,
                   kernel=wmg.KERNEL_JOSEPH)
    b = p64.project(xd.double())
    b = b + 0.01 * b.abs().max() * torch.tensor(S.uniform_noise_draws(m * D, S.seed_for(6, 0)),
                                                dtype=torch.float64, device=dev)
    b = b.to(torch.float32).contiguous()
    p64.close()
    out = {"workload": f"{n}x{n}_{m}ang_{D}det, W = Joseph's kernel, 1% uniform white noise (eq. noise_term)",
           "levels": levels, "cycle": f"hybrid at every depth ({levels - 1}), nu1=nu2=0",
           "error": "||x_k - x_ex|| / ||x_ex|| (L2, Linf); x_k from a solve of exactly k iterations",
           "lambda_regularised": 1e-3 * m / n}
    stream = torch.cuda.current_stream()
    for tag, lam in (("noisy", 0.0), ("regularised", 1e-3 * m / n)):
        # the paper's cycle: the hybrid residual update at every depth
        plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, lam=lam, hybrid_depth=levels - 1,
                        cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32, kernel=wmg.KERNEL_JOSEPH)
        res = {}
        for name, solver, pre, kmax in (("SIRT", wmg.SOLVER_SIRT, False, 3000),
                                        ("BiCGStab", wmg.SOLVER_BICGSTAB, False, 300),
                                        ("WMG-BiCGStab", wmg.SOLVER_BICGSTAB, True, 100)):
            curve = study.error_curve(plan, b, xd, solver, pre, study.log_ks(kmax, 6))
            ko, row = study.k_opt(curve)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.solve(b, solver, pre, ko, 0.0, 20)
            e1.record(stream)
            torch.cuda.synchronize()
            res[name] = {"k_opt": ko, "error_l2": row[2], "error_linf": row[3],
                         "error_l2_at_kmax": curve[-1][2], "kmax": kmax,
                         "ms_to_k_opt": e0.elapsed_time(e1)}
        out[tag] = res
        plan.close()
    # Tikhonov sweep (eq. sys_reg, Tables 2-3): for each lambda the k_opt and
    # the error at k_opt and at k_max of the Krylov solvers, plain and WMG
    sweep = []
    for rel in LAMBDA_SWEEP:
        lam = rel * m / n
        plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, lam=lam, hybrid_depth=levels - 1,
                        cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32, kernel=wmg.KERNEL_JOSEPH)
        row = {"lambda_over_m_per_n": rel, "lambda": lam}
        for name, solver, pre, kmax in (("BiCGStab", wmg.SOLVER_BICGSTAB, False, 300),
                                        ("WMG-BiCGStab", wmg.SOLVER_BICGSTAB, True, 100)):
            curve = study.error_curve(plan, b, xd, solver, pre, study.log_ks(kmax, 6))
            ko, best = study.k_opt(curve)
            row[name] = {"k_opt": ko, "error_l2": best[2], "error_l2_at_kmax": curve[-1][2], "kmax": kmax}
        sweep.append(row)
        plan.close()
    out["lambda_sweep"] = sweep
    return out


# ---------------------------------------------------------------------------
# Serving leg: a seeded Poisson stream of reconstruction requests of mixed
# image sizes and angle counts through the continuous-batching server
# ---------------------------------------------------------------------------
def serving_leg(args, dev, requests=None, max_n=None, rate=None) -> dict:
    """A seeded Poisson stream through the continuous-batching server: the
    first `requests` requests of the configured stream with n <= max_n,
    arriving at `rate` per second (all at t = 0 with --serving-burst)."""
    import torch
    import paper_1310_0956_gb300 as wmg

    requests = args.serving_requests if requests is None else requests
    max_n = args.serving_max_n if max_n is None else max_n
    rate = args.serving_rate if rate is None else rate
    wl, gaps = S.workload_serving(max(2000, requests))
    picked = [(p, g) for p, g in zip(wl.problems, gaps) if p.n <= max_n][:requests]
    probs = [p for p, _ in picked]
    arrivals = np.cumsum([g for _, g in picked]) / rate
    arrivals -= arrivals[0]
    if args.serving_burst:
        arrivals[:] = 0.0
    # sinograms b = W x + 1% noise (FP64 library projector), resident on the device
    bs = []
    for p in probs:
        op = wmg.Plan(p.n, p.m, p.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
        b64 = op.project(torch.tensor(p.image().reshape(-1), dtype=torch.float64, device=dev))
        b64 = b64 + p.noise * b64.abs().max() * torch.tensor(p.noise_unit(), dtype=torch.float64, device=dev)
        bs.append(b64.to(torch.float32).contiguous())
        op.close()
    torch.cuda.synchronize()
    # device memory for the server: 160 GB (2048^2 geometries hold 4.3 GB of
    # FP32 leaf inverses each and their setups ~9 GB of transient FP64 Gram
    # blocks), 48 GB of it for request state
    srv = wmg.Server(160 << 30, max_slots=64, state_bytes=48 << 30, sino_ratio=4.0, preconditioned=True,
                     max_iter=MAX_ITER, rtol=RTOL, restart=RESTART, levels=1, nu1=NU1, nu2=NU2, hybrid_depth=HYB,
                     cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
    launches0 = wmg.wmg_launch_count(False)
    t0 = time.perf_counter()
    nxt, live, done = 0, {}, {}
    peak = 0
    while len(done) < len(probs):
        now = time.perf_counter() - t0
        while nxt < len(probs) and arrivals[nxt] <= now:
            p = probs[nxt]
            t = srv.submit({"n": p.n, "m": p.m, "D": p.D, "levels": S.levels_for(p.n),
                            "lam": SERVING_EPS * p.m / p.n}, bs[nxt])
            live[t] = nxt
            nxt += 1
        if live:
            srv.step()
            peak = max(peak, srv.stats()["running"])
            now = time.perf_counter() - t0
            for t in list(live):
                r = srv.poll(t)
                if r is not None:
                    done[live.pop(t)] = (now, r[1])
        elif nxt < len(probs):
            time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
    wall = max(d[0] for d in done.values())
    st = srv.stats()
    srv.close()
    lat = np.array([(done[i][0] - arrivals[i]) * 1e3 for i in range(len(probs))])
    infos = [done[i][1] for i in range(len(probs))]
    sizes = sorted({p.n for p in probs})
    by_size = {}
    for nn in sizes:
        ls = np.array([lat[i] for i, p in enumerate(probs) if p.n == nn])
        by_size[str(nn)] = {"requests": int(ls.size), "p50_latency_ms": float(np.percentile(ls, 50)),
                            "p99_latency_ms": float(np.percentile(ls, 99))}
    return {
        "latency_by_image_side": by_size,
        "workload": ("burst" if args.serving_burst else f"poisson_rate{rate:g}") +
                    f"_{len(probs)}req_n" + "-".join(map(str, sizes)) + "_m90-720",
        "requests": len(probs), "recon_per_s": len(probs) / wall, "wall_s": wall,
        "p50_latency_ms": float(np.percentile(lat, 50)), "p99_latency_ms": float(np.percentile(lat, 99)),
        "mean_latency_ms": float(lat.mean()),
        "latency_from": "scheduled arrival to retirement seen by the host",
        "all_converged": bool(all(i[1] == 0 for i in infos)),
        "status_counts": {str(k): int(v) for k, v in zip(*np.unique([i[1] for i in infos], return_counts=True))},
        "not_converged": [{"n": probs[i].n, "m": probs[i].m, "iters": infos[i][0], "status": infos[i][1],
                           "rel_res": infos[i][2]} for i in range(len(probs)) if infos[i][1] != 0][:8],
        "iters_mean": float(np.mean([i[0] for i in infos])),
        "max_running": peak, "ticks": st["ticks"], "geometry_setups": st["geometry_setups"],
        "gpu_launches": wmg.wmg_launch_count(False) - launches0,
        "solver": "WMG-GMRES(20) hybrid depth 1, FP32 operator / FP64 Krylov, rtol 1e-4",
        "lambda": f"Tikhonov (W^T W + lambda) x = W^T b, lambda = {SERVING_EPS:g} * m / n",
        "note": "geometry setups (leaf Gram + inverses) run on a worker stream, overlapping the steps",
    }


# ---------------------------------------------------------------------------
# Uneven-batch leg: 64 problems of different sizes and angle counts solved
# together (one launch per operator application over all of them)
# ---------------------------------------------------------------------------
def fp64_single_leg(geoms, bs64, solver, hybrid_depth, cycle, x_mixed, dev) -> dict:
    """The plain form the mixed batched one is compared with: FP64 plans (FP64
    operator, leaf solves and Krylov), one problem per solve call, so every
    operator application is a launch over one problem; the same cycle,
    solver and tolerance. Plan setup excluded (as for the batched form);
    solve time by the host clock around each synchronising solve.
    x_mixed: the mixed batched solutions of the same problems, for the
    relative image difference of the two forms at equal tolerance."""
    import torch
    import paper_1310_0956_gb300 as wmg
    times, iters, statuses, diffs = [], [], [], []
    for g, b64, xm in zip(geoms, bs64, x_mixed):
        pl = wmg.Plan(g["n"], g["m"], g["D"], levels=g["levels"], nu1=NU1, nu2=NU2, lam=g.get("lam", 0.0),
                      hybrid_depth=hybrid_depth, cycle=cycle, precision=wmg.PREC_F64)
        out = torch.empty(g["n"] * g["n"], dtype=torch.float64, device=dev)
        pl.solve(b64, solver, True, MAX_ITER, RTOL, RESTART, out=out)          # warm-up (graphs, tuning)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info, _, _ = pl.solve(b64, solver, True, MAX_ITER, RTOL, RESTART, out=out)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        iters.append(info[0][0])
        statuses.append(info[0][1])
        diffs.append(float(torch.linalg.norm(out - xm) / torch.linalg.norm(out)))
        pl.close()
    return {"precision": "fp64 operator, leaf solves and Krylov", "problems_timed": len(times),
            "recon_per_s": len(times) / float(np.sum(times)), "ms_per_recon": 1e3 * float(np.mean(times)),
            "iters_mean": float(np.mean(iters)), "all_converged": bool(all(s_ == 0 for s_ in statuses)),
            "rel_image_diff_vs_mixed_max": float(np.max(diffs)),
            "timing": "host clock around each synchronising one-problem solve, setup excluded"}


def batched_inputs(dev):
    """The uneven batch of 64 problems and their noisy FP32 sinograms
    (projected by FP64 plans)."""
    import torch
    import paper_1310_0956_gb300 as wmg

    probs = S.workload_batched(64).problems
    bs = []
    for p in probs:
        op = wmg.Plan(p.n, p.m, p.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
        b64 = op.project(torch.tensor(p.image().reshape(-1), dtype=torch.float64, device=dev))
        b64 = b64 + p.noise * b64.abs().max() * torch.tensor(p.noise_unit(), dtype=torch.float64, device=dev)
        bs.append(b64.to(torch.float32).contiguous())
        op.close()
    torch.cuda.synchronize()
    return probs, bs


def batched_plans(probs):
    import paper_1310_0956_gb300 as wmg
    return wmg.Batch([dict(n=p.n, m=p.m, D=p.D, levels=p.levels, lam=SERVING_EPS * p.m / p.n) for p in probs],
                     nu1=NU1, nu2=NU2, hybrid_depth=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)


def batched_leg(args, dev) -> dict:
    import torch
    import paper_1310_0956_gb300 as wmg

    probs, bs = batched_inputs(dev)
    t0 = time.perf_counter()
    bt = batched_plans(probs)
    torch.cuda.synchronize()
    setup = time.perf_counter() - t0
    outs = [torch.empty(p.N, dtype=torch.float32, device=dev) for p in probs]
    bt.solve(bs, wmg.SOLVER_CGLS, True, MAX_ITER, RTOL, outs=outs)          # warm-up
    times, infos = [], None
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, infos, _ = bt.solve(bs, wmg.SOLVER_CGLS, True, MAX_ITER, RTOL, outs=outs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    bt.close()
    t = float(np.mean(times))
    single = fp64_single_leg(
        [dict(n=p.n, m=p.m, D=p.D, levels=p.levels, lam=SERVING_EPS * p.m / p.n) for p in probs[:FP64_SAMPLE]],
        [b_.to(torch.float64) for b_ in bs[:FP64_SAMPLE]], wmg.SOLVER_CGLS, 0, wmg.CYCLE_ADDITIVE,
        [o.double() for o in outs[:FP64_SAMPLE]], dev)
    single["mixed_batched_over_fp64_single"] = (len(probs) / t) / single["recon_per_s"]
    return {
        "workload": "batched64_n128-512_m60-360_noise1pct", "problems": len(probs),
        "fp64_one_problem_per_launch": single,
        "recon_per_s": len(probs) / t, "ms_per_batch": t * 1e3,
        "solver": f"WMG-CGLS (PCG on the normal equations), additive cycle, nu1=nu2={NU1}, rtol {RTOL:g}",
        "lambda": f"lambda = {SERVING_EPS:g} * m / n",
        "precision": "fp32 operator and leaf solves, fp64 Krylov",
        "iters_mean": float(np.mean([i[0] for i in infos])), "iters_max": int(max(i[0] for i in infos)),
        "all_converged": bool(all(i[1] == 0 for i in infos)),
        "setup_s": setup, "timing": "host clock around the synchronising batch solve, mean of 3",
    }


# ---------------------------------------------------------------------------
# Stored-W comparator: the workload's W and W^T as CSR (wmg_csr_*), applied
# to the same 64-image batch as the matrix-free operators; its bandwidth is
# where an HBM roofline fraction means something. Also the measured FP32
# peak (cuBLAS SGEMM, no TF32) as context for the ALU-bound projector.
# ---------------------------------------------------------------------------
def _event_time(fn, stream, flush, reps=5):
    """Median device time of fn() between CUDA events, L2 flushed before each
    call; a ~0.2 ms spin kernel ahead of the start event keeps the GPU busy
    while the host issues fn(), so host launch latency is not timed."""
    import torch
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        torch.cuda._sleep(400_000)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    return float(np.median(ts))


def comparator_leg(plan, P0, x_batch, b_batch, flush, dev) -> dict:
    import torch
    stream = torch.cuda.current_stream()
    B = x_batch.numel() // P0.N
    out = {"workload": f"{P0.n}x{P0.n}_{P0.m}ang_{P0.D}det, batch {B}, fp32"}
    Wc, WTc = plan.csr(False), plan.csr(True)
    hbm = load_peaks().get("hbm_gbs")
    y_b = torch.empty_like(b_batch)
    y_x = torch.empty_like(x_batch)
    for name, csr, fn_free, inp, res in (("W", Wc, lambda: plan.project(x_batch, out=y_b), x_batch, y_b),
                                        ("WT", WTc, lambda: plan.backproject(b_batch, out=y_x), b_batch, y_x)):
        for cnt in (1, B):
            xi = inp[: cnt * csr.cols]
            yo = res[: cnt * csr.rows]
            t_csr = _event_time(lambda: csr.apply(xi, out=yo), stream, flush)
            bytes_ = csr.nnz * 8 + (csr.rows + 1) * 8 + cnt * (csr.rows + csr.cols) * 4
            out[f"{name}_csr_x{cnt}_ms"] = t_csr * 1e3
            out[f"{name}_csr_x{cnt}_gbs"] = bytes_ / t_csr / 1e9
            if hbm:
                out[f"{name}_csr_x{cnt}_hbm_frac"] = bytes_ / t_csr / 1e9 / hbm
        if name == "W":
            t_free = _event_time(lambda: plan.project(x_batch, out=y_b), stream, flush)
        else:
            t_free = _event_time(lambda: plan.backproject(b_batch, out=y_x), stream, flush)
        out[f"{name}_matrix_free_x{B}_ms"] = t_free * 1e3
        out[f"{name}_speedup_vs_csr_x{B}"] = out[f"{name}_csr_x{B}_ms"] / (t_free * 1e3)
    out["nnz"] = Wc.nnz
    out["csr_bytes"] = int(Wc.nnz * 8 + (Wc.rows + 1) * 8)
    Wc.close()
    WTc.close()
    # FP32 arithmetic peak, measured: cuBLAS SGEMM with TF32 off
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    a = torch.randn(8192, 8192, device=dev)
    bm = torch.randn(8192, 8192, device=dev)
    c = torch.empty(8192, 8192, device=dev)
    for _ in range(2):
        torch.matmul(a, bm, out=c)
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(a, bm, out=c)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    torch.backends.cuda.matmul.allow_tf32 = prev
    out["fp32_sgemm_tflops_measured"] = 2 * 8192 ** 3 / min(ts) / 1e12
    del a, bm, c
    return out


# ---------------------------------------------------------------------------
# 1024 x 1024 leg: one reconstruction of the large workload by WMG-CGLS
# (additive cycle) to 1e-4, mixed path (FP32 operator, FP64 Krylov / leaf
# solves) next to the all-FP64 GPU path
# ---------------------------------------------------------------------------
def large_leg(dev) -> dict:
    import torch
    import paper_1310_0956_gb300 as wmg

    p = S.workload_large().problems[0]
    lam = SERVING_EPS * p.m / p.n
    op = wmg.Plan(p.n, p.m, p.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    xt = torch.tensor(p.image().reshape(-1), dtype=torch.float64, device=dev)
    b = op.project(xt)
    b = b + p.noise * b.abs().max() * torch.tensor(p.noise_unit(), dtype=torch.float64, device=dev)
    op.close()
    out = {"workload": "1024x1024_1024ang_1449det_50ell_tex0.05_noise0.5pct", "levels": p.levels,
           "solver": f"WMG-CGLS additive cycle, nu1=nu2={NU1}, rtol {RTOL:g}",
           "lambda": f"lambda = {SERVING_EPS:g} * m / n"}
    xs = {}
    for prec, tag in ((wmg.PREC_F32, "mixed_fp32"), (wmg.PREC_F64, "fp64")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl = wmg.Plan(p.n, p.m, p.D, levels=p.levels, nu1=NU1, nu2=NU2, lam=lam, hybrid_depth=0,
                      cycle=wmg.CYCLE_ADDITIVE, precision=prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bb = b.float().contiguous() if prec == wmg.PREC_F32 else b
        x, info, _, _ = pl.solve(bb, wmg.SOLVER_CGLS, True, MAX_ITER, RTOL, RESTART)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        pl.close()
        xs[tag] = x.double()
        out[tag] = {"setup_s": t1 - t0, "solve_s": t2 - t1, "recon_per_s": 1.0 / (t2 - t1),
                    "iters": info[0][0], "status": info[0][1], "rel_res": info[0][2],
                    "image_err_vs_phantom": (torch.norm(x.double() - xt) / torch.norm(xt)).item()}
    out["rel_diff_mixed_vs_fp64"] = (torch.norm(xs["mixed_fp32"] - xs["fp64"]) / torch.norm(xs["fp64"])).item()
    out["solve_speedup_mixed_vs_fp64"] = out["fp64"]["solve_s"] / out["mixed_fp32"]["solve_s"]
    # WMG-GMRES(20), the paper's cycle (hybrid update at depth 0): FP32
    # operator, BF16 operator storage in the Arnoldi steps with FP32 true
    # residuals at the restarts, and the FP64 path; one warm-up solve each
    gm = {"solver": f"WMG-GMRES({RESTART}) hybrid depth {HYB}, nu1=nu2={NU1}, rtol {RTOL:g}"}
    gx = {}
    for prec, tag in ((wmg.PREC_F32, "mixed_fp32"), (wmg.PREC_F32_BF16STORE, "bf16_storage"),
                      (wmg.PREC_F64, "fp64")):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pl = wmg.Plan(p.n, p.m, p.D, levels=p.levels, nu1=NU1, nu2=NU2, lam=lam, hybrid_depth=HYB,
                      cycle=wmg.CYCLE_HYBRID, precision=prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bb = b if prec == wmg.PREC_F64 else b.float().contiguous()
        pl.solve(bb, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        x, info, _, _ = pl.solve(bb, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        pl.close()
        gx[tag] = x.double()
        gm[tag] = {"setup_s": t1 - t0, "solve_s": t3 - t2, "recon_per_s": 1.0 / (t3 - t2), "iters": info[0][0],
                   "status": info[0][1], "rel_res": info[0][2],
                   "image_err_vs_phantom": (torch.norm(x.double() - xt) / torch.norm(xt)).item()}
    for tag in ("mixed_fp32", "bf16_storage"):
        gm[tag]["rel_diff_vs_fp64"] = (torch.norm(gx[tag] - gx["fp64"]) / torch.norm(gx["fp64"])).item()
        gm[tag]["solve_speedup_vs_fp64"] = gm["fp64"]["solve_s"] / gm[tag]["solve_s"]
    out["gmres"] = gm
    return out


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# DRAM traffic of the FP32 projector (8-image TMA group tiles) and
# backprojector (8-image group tiles) measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum, 64-image launches of the workload geometry;
# profiles/dram_traffic_k_project_backproject_256x256.md), per image; each
# valid while its kernel's source is the one measured (hash), else null.
KERNEL_TRAFFIC = {
    "project": {"source": "paper_1310_0956_gb300/csrc/projector_tma.cu", "sha256_16": "ae0bdc1d96090fc7",
                "bytes_per_image": (33875712 + 11776 + 33876992 + 33878272) / 3 / 64.0},
    "backproject": {"source": "paper_1310_0956_gb300/csrc/projector_f32.cu", "sha256_16": "944267f066ebc531",
                    "bytes_per_image": (16432384 + 16489984 + 16479232) / 3 / 64.0},
}


def _kernel_traffic(name: str, images: float):
    import hashlib
    rec = KERNEL_TRAFFIC[name]
    try:
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != rec["sha256_16"]:
                return None
    except OSError:
        return None
    return rec["bytes_per_image"] * images


def roofline_entry(prof: dict, P0, B: int) -> dict:
    """Dominant kernel: the projector or the backprojector, whichever has the
    larger total time, the projector's launches on the 2h grid (band updates
    whose input lies in the first split's LL band: the same kernel) counted
    with it. It is bound by FP32 arithmetic, not memory: the algorithmic work
    is one multiply-add (2 FLOP) per nonzero of W, against the FP32 FMA peak
    of 152 SMs x 128 lanes x 2 FLOP at the maximum SM clock. Algorithmic nnz
    per launch = nnz(W) of the geometry x images in the launch; the rate is
    taken over the launches on W's grid (the 2h grid's nonzeros are those of
    W^{2h}), and the note gives the 2h launches' count and mean time."""
    p2h = prof.get("project_2h") or {"launches": 0, "total_ms": 0.0}
    total = {"project": prof["project"]["total_ms"] + p2h["total_ms"], "backproject": prof["backproject"]["total_ms"]}
    name = max(("project", "backproject"), key=lambda k: total[k])
    p = prof[name]
    nnz_per_image = prof["nnz_per_image"]
    flops_per_launch = 2.0 * nnz_per_image * p["images_per_launch"]
    achieved = flops_per_launch / (p["mean_ms"] * 1e-3) / 1e12
    peaks = load_peaks()
    clk = peaks.get("sm_max_mhz", 2070.0)
    derived = 152 * 128 * 2 * clk * 1e6 / 1e12
    # measured FP32 multiply-add peak (the better of one and two multiply-adds
    # per instruction) when given, else unit counts x the maximum clock
    measured = prof.get("fp32_fma_tflops_measured")
    peak = measured if measured else derived
    # the same launch as an HBM client: algorithmic bytes = s (N + M), the
    # FP32 input read once and the output written once
    n_in = P0.N if name == "project" else P0.M
    n_out = P0.M if name == "project" else P0.N
    gbs = p["images_per_launch"] * (n_in + n_out) * 4 / (p["mean_ms"] * 1e-3) / 1e9
    hbm = peaks.get("hbm_gbs")
    return {"kernel": f"k_{name}", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": _kernel_traffic(name, p["images_per_launch"]),
            "traffic_unit": "bytes per launch (DRAM read + write)",
            "algorithmic_gbs": gbs, "hbm_frac_of_measured": (gbs / hbm) if hbm else None,
            "note": (f"{p['launches']} launches, mean {p['mean_ms']:.3f} ms, "
                     f"{nnz_per_image * p['images_per_launch'] / (p['mean_ms'] * 1e-3) / 1e9:.0f} Gnnz/s; "
                     + (f"and {p2h['launches']} launches on the 2h grid (band updates), mean "
                        f"{p2h['mean_ms']:.3f} ms, not in the rate; "
                        if name == "project" and p2h["launches"] else "")
                     + (f"peak measured (FP32 multiply-add chains, best of scalar and paired); derived "
                        f"152 SMs x 128 FP32 lanes x 2 FLOP x {clk:.0f} MHz = {derived:.1f}; " if measured else
                        f"peak derived: 152 SMs x 128 FP32 lanes x 2 FLOP x {clk:.0f} MHz; ")
                     + "as an HBM client "
                     f"{gbs:.0f} GB/s of algorithmic bytes"
                     + (f" = {gbs / hbm:.3f} of the measured {hbm:.0f} GB/s" if hbm else ""))}


def solve_case(batch: int):
    """Three solves of the workload batch (the bench's inputs and solver) and
    exit: the case for ncu captures of the solve's secondary kernels."""
    import torch
    import paper_1310_0956_gb300 as wmg
    probs = workload_problems(batch, 0)
    P0 = probs[0]
    plan = wmg.Plan(P0.n, P0.m, P0.D, levels=LEVELS, nu1=NU1, nu2=NU2, hybrid_depth=HYB,
                    cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
    p64 = wmg.Plan(P0.n, P0.m, P0.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    imgs = torch.tensor(np.stack([p.image() for p in probs]).reshape(-1), dtype=torch.float64, device="cuda")
    b64 = p64.project(imgs).view(len(probs), P0.M)
    noise = torch.tensor(np.stack([p.noise_unit() for p in probs]), dtype=torch.float64, device="cuda")
    sigma = torch.tensor([p.noise for p in probs], dtype=torch.float64, device="cuda")[:, None] * \
        b64.abs().amax(dim=1, keepdim=True)
    b = (b64 + sigma * noise).to(torch.float32).contiguous().view(-1)
    x = torch.empty(len(probs) * P0.N, dtype=torch.float32, device="cuda")
    its = []
    for _ in range(3):
        _, info, _, _ = plan.solve(b, wmg.SOLVER_GMRES, True, MAX_ITER, RTOL, RESTART, out=x)
        its.append(float(np.mean([i[0] for i in info])))
    torch.cuda.synchronize()
    print(json.dumps({"solve_case": "ok", "iters_mean": its}))


def batched_case():
    """Three solves of the uneven batch (the batched leg's inputs and solver)
    after one warm-up, and exit: the case for ncu launch lists of that leg."""
    import torch
    import paper_1310_0956_gb300 as wmg
    dev = torch.device("cuda", 0)
    probs, bs = batched_inputs(dev)
    bt = batched_plans(probs)
    outs = [torch.empty(p.N, dtype=torch.float32, device=dev) for p in probs]
    its = []
    for _ in range(4):
        _, infos, _ = bt.solve(bs, wmg.SOLVER_CGLS, True, MAX_ITER, RTOL, outs=outs)
        its.append(float(np.mean([i[0] for i in infos])))
    torch.cuda.synchronize()
    bt.close()
    print(json.dumps({"batched_case": "ok", "iters_mean": its}))


def kernel_case(images: int = 16):
    import torch
    import paper_1310_0956_gb300 as wmg
    P0 = workload_problems(1, 0)[0]
    plan = wmg.Plan(P0.n, P0.m, P0.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE,
                    precision=wmg.PREC_F32)
    x = torch.rand(images * P0.N, dtype=torch.float32, device="cuda")
    b = torch.empty(images * P0.M, dtype=torch.float32, device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        plan.project(x, out=b)
    for _ in range(3):
        plan.backproject(b, out=y)
    torch.cuda.synchronize()
    print(json.dumps({"kernel_case": "ok", "nnz_per_image": plan.nnz()}))


def setup_times(cases) -> dict:
    """Plan creation (geometry, smoother diagonal, leaf Galerkin setup and
    inverses) of the serving configuration, FP32, per (n, m): seconds."""
    import torch
    import paper_1310_0956_gb300 as wmg
    out = {}
    for n, m in cases:
        D, levels = S.detectors_for(n), S.levels_for(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan = wmg.Plan(n, m, D, levels=levels, nu1=NU1, nu2=NU2, lam=SERVING_EPS * m / n, hybrid_depth=HYB,
                        cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
        torch.cuda.synchronize()
        out[f"{n}x{n}_{m}ang_{D}det_levels{levels}"] = time.perf_counter() - t0
        plan.close()
    return out


def setup_case(spec: str):
    import torch
    import paper_1310_0956_gb300 as wmg
    n, m = (int(v) for v in spec.split(":"))
    D, levels = S.detectors_for(n), S.levels_for(n)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=wmg.PREC_F32)
    torch.cuda.synchronize()
    print(json.dumps({"setup_case": f"{n}x{n}_{m}ang_{D}det", "levels": levels,
                      "setup_s": time.perf_counter() - t0}))
    plan.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.setup_case:
        setup_case(args.setup_case)
        return
    if args.kernel_case:
        kernel_case(args.kernel_images)
        return
    if args.solve_case:
        solve_case(args.batch)
        return
    if args.batched_case:
        batched_case()
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.serving_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(serving_leg(args, torch.device("cuda", local))), flush=True)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
