"""Oracle runs that GPU parity tests hand to a spawned process pool: plain
functions of picklable arguments, importing only the oracle, the input
generator and numpy (no torch, no library), so a worker starts quickly and
never touches the GPU."""
import numpy as np

import oracle
import synthetic as S


def noisy_sinogram(p, op):
    """b = W x_phantom + sigma N(0,1), sigma = noise * max|W x| (the input
    recipe), with the oracle's projector."""
    b0 = op.project(p.image())
    return b0 + p.noise * np.abs(b0).max() * p.noise_unit()


def mid_gmres(i, count, b, iters, levels=5, hybrid_depth=1):
    """WMG-GMRES(20) of problem i of the 256^2 workload with the paper's
    cycle (no smoothing, hybrid update to `hybrid_depth`)."""
    P = S.workload_mid(count).problems[i]
    op = oracle.Op(P.n, P.m, P.D)
    M = oracle.Wmg(op, levels, 0, 0, 1.0, 0.0, oracle.CYCLE_HYBRID, hybrid_depth)
    return oracle.gmres(op, b, iters, 20, 0.0, 0.0, M)[0]


def batched_cgls(i, count, b, iters):
    """Additive WMG-CGLS (no smoothing) of problem i of the uneven batch,
    lambda = 1e-3 m / n."""
    p = S.workload_batched(count).problems[i]
    op = oracle.Op(p.n, p.m, p.D)
    lam = 1e-3 * p.m / p.n
    M = oracle.Wmg(op, p.levels, 0, 0, 1.0, lam, oracle.CYCLE_ADDITIVE, 0)
    return oracle.cgls(op, b, iters, 0.0, lam, M)[0]
