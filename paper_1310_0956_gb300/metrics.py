"""Metrics of reconstruction runs as JSON lines.

A solve record holds, per problem, the iteration count, status and final
relative normal-equation residual |W^T (b - W x) - lambda x| / |W^T b|
(with its history when asked), and for the whole call the A-pairs per
problem, the plan's setup time, the solve time and what the operator
launches achieved: intersections (nonzeros of W applied) per second and
algorithmic operator bytes per second. A serving record holds the
server's counters, queue depth, p50 / p99 request latency and completed
requests per second. Records are plain dicts; JsonlLog appends them to a
file, one JSON object per line."""
from __future__ import annotations

import json

from . import (PREC_F64, SOLVER_BICGSTAB, SOLVER_CGLS, SOLVER_GMRES, SOLVER_SIRT, STATUS_NAMES, Plan,
               wmg_profile_begin, wmg_profile_end)

SOLVER_NAMES = {SOLVER_SIRT: "SIRT", SOLVER_CGLS: "CGLS", SOLVER_GMRES: "GMRES", SOLVER_BICGSTAB: "BiCGStab"}


class JsonlLog:
    """Appends records to `path`, one compact JSON object per line."""

    def __init__(self, path: str):
        self.path = path

    def write(self, record: dict) -> None:
        with open(self.path, "a") as f:
            f.write(json.dumps(record, separators=(",", ":")) + "\n")


def solve_metrics(n: int, m: int, D: int, precision: int, solver: int, preconditioned: bool, infos, hists,
                  prof: dict, solve_s: float, setup_s: float | None = None) -> dict:
    """The record of one solve call. infos: (iterations, status, rel_res)
    per problem; hists: residual histories or None; prof: the library's
    launch profile of the call (wmg_profile_stats fields). Every A-pair
    projects each problem once, on W's grid or, in the hybrid cycle's band
    updates whose input lies in the first split's LL band, on the 2h grid;
    so A-pairs per problem = projected images of both kinds / problems.
    Intersections and operator bytes count the launches on W's grid alone
    (their time only). Operator bytes are algorithmic: the projector reads
    an image and its transposed copy and writes a sinogram, the
    backprojector reads a sinogram and writes an image."""
    cnt = len(infos)
    N, M = n * n, m * D
    esz = 8 if precision == PREC_F64 else 4
    pj_img, bp_img = prof["project_images"], prof["backproject_images"]
    pj2_img = prof.get("project_2h_images", 0.0)
    op_s = (prof["project_ms"] + prof["backproject_ms"]) / 1e3
    inter = prof["nnz_per_image"] * (pj_img + bp_img)
    nbytes = (pj_img * (2 * N + M) + bp_img * (M + N)) * esz
    rec = {
        "event": "solve", "solver": SOLVER_NAMES.get(solver, str(solver)), "preconditioned": bool(preconditioned),
        "n": n, "m": m, "D": D, "precision": "f64" if precision == PREC_F64 else "f32", "problems": cnt,
        "iterations": [int(i[0]) for i in infos],
        "status": [STATUS_NAMES.get(int(i[1]), str(i[1])) for i in infos],
        "rel_res": [float(i[2]) for i in infos],
        "a_pairs_per_problem": (pj_img + pj2_img) / cnt if cnt else 0.0,
        "setup_s": setup_s, "solve_s": solve_s,
        "project": {"launches": prof["project_launches"], "ms": prof["project_ms"], "images": pj_img},
        "backproject": {"launches": prof["backproject_launches"], "ms": prof["backproject_ms"], "images": bp_img},
        "project_2h": {"launches": prof.get("project_2h_launches", 0), "ms": prof.get("project_2h_ms", 0.0),
                       "images": pj2_img},
        "intersections_per_s": inter / op_s if op_s > 0 else None,
        "operator_gb_per_s": nbytes / op_s / 1e9 if op_s > 0 else None,
    }
    if hists is not None:
        rec["residual_history"] = [[float(v) for v in h] for h in hists]
    return rec


def profiled_solve(plan: Plan, b, solver: int, preconditioned: bool = True, max_iter: int = 100,
                   rtol: float = 1e-4, restart: int = 20, history: bool = False, x0=None, log: JsonlLog | None = None):
    """Plan.solve with the library's per-launch device timing of the
    projector and backprojector (wmg_profile_begin / end: the iterations run
    without CUDA graphs while it is on). Returns (x, infos, hists, rc,
    record) and appends the record to `log` if given."""
    torch = plan._torch
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    wmg_profile_begin(plan.handle)
    try:
        e0.record(stream)
        x, infos, hists, rc = plan.solve(b, solver, preconditioned, max_iter, rtol, restart, history=history, x0=x0)
        e1.record(stream)
    finally:
        st = wmg_profile_end(plan.handle, plan._stream())
    torch.cuda.synchronize()
    prof = {k: getattr(st, k) for k in ("project_launches", "project_ms", "project_images", "backproject_launches",
                                        "backproject_ms", "backproject_images", "nnz_per_image",
                                        "project_2h_launches", "project_2h_ms", "project_2h_images")}
    rec = solve_metrics(plan.n, plan.m, plan.D, plan.opts.precision, solver, preconditioned, infos, hists, prof,
                        e0.elapsed_time(e1) / 1e3, getattr(plan, "setup_s", None))
    if log is not None:
        log.write(rec)
    return x, infos, hists, rc, rec


def percentile(values, q: float) -> float | None:
    """The q-th percentile (0..100) by linear interpolation between order
    statistics; None for no values."""
    v = sorted(values)
    if not v:
        return None
    pos = (len(v) - 1) * q / 100.0
    lo = int(pos)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (pos - lo)


def serving_metrics(counters: dict, latencies_ms, wall_s: float) -> dict:
    """The record of a serving window: the server's counters (Server.stats),
    the latencies (ms, submit to completion) of the requests completed in
    the window and its wall time."""
    lat = list(latencies_ms)
    return {
        "event": "serve", "completed": len(lat), "queue_depth": counters.get("queued"),
        "running": counters.get("running"), "p50_ms": percentile(lat, 50), "p99_ms": percentile(lat, 99),
        "recon_per_s": len(lat) / wall_s if wall_s > 0 else None, "wall_s": wall_s, "counters": dict(counters),
    }


__all__ = ["JsonlLog", "solve_metrics", "profiled_solve", "percentile", "serving_metrics", "SOLVER_NAMES"]
