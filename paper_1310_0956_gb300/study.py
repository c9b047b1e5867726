"""Semi-convergence of the iterative solvers on noisy data (Section 4.2):
the error of the k-th iterate against the exact object, e_k = x_k - x_ex,
with x_0 = 0 so that ||e_0|| = ||x_ex||. Every iterate is that of a solve of
exactly k iterations (rtol 0) through the library's own solvers: the run is
continued from one k to the next (wmg_solve_resume), which gives bitwise the
iterate of a fresh k-iteration solve, so the whole curve costs one run to
the largest k."""
from __future__ import annotations

from . import SOLVER_GMRES, Plan


def error_curve(plan: Plan, b, x_true, solver: int, preconditioned: bool, ks, restart: int = 20):
    """For each k in ks: (k, iterations done, ||e_k||_2 / ||e_0||_2,
    ||e_k||_inf / ||e_0||_inf) for one problem of `plan` (b and x_true CUDA
    tensors of sizes M and N). A solve that ends early (breakdown) reports
    the iterations it did. GMRES continues a run only from a k that is a
    multiple of the restart length (a restart of the fresh solve) and solves
    afresh otherwise."""
    xt = x_true.double()
    n2, ninf = float(xt.norm()), float(xt.abs().max())
    out = []
    prev = None
    for k in (int(k) for k in ks):
        resumable = prev is not None and prev <= k and (solver != SOLVER_GMRES or prev % restart == 0)
        if resumable:
            x, info, _, _ = plan.resume(b, k, 0.0, problem_errors=False)
        else:
            x, info, _, _ = plan.solve(b, solver, preconditioned, k, 0.0, restart, problem_errors=False)
        prev = k
        e = x.double() - xt
        out.append((k, int(info[0][0]), float(e.norm()) / n2, float(e.abs().max()) / ninf))
    return out


def k_opt(curve):
    """The iterate count with the smallest L2 error, and that row of the
    curve (Section 4.2: k_opt = argmin_k ||e_k||)."""
    best = min(curve, key=lambda r: r[2])
    return best[0], best


def log_ks(kmax: int, per_decade: int = 8):
    """Iterate counts 1 .. kmax spread evenly on a log scale (the paper plots
    these curves against log k)."""
    import math
    ks, k = [], 1
    while k <= kmax:
        ks.append(k)
        k = max(k + 1, int(round(10 ** (math.log10(k) + 1.0 / per_decade))))
    if ks[-1] != kmax:
        ks.append(kmax)
    return ks


__all__ = ["error_curve", "k_opt", "log_ks"]
