"""The 1024 x 1024, 1024-angle, 1449-bin workload at full size: sampled rows
of the FP32 and FP64 projectors against the oracle's single-row builder,
adjointness of the full operator pair, and the mixed-precision (FP32
operator) WMG-CGLS against the FP64 GPU path after the same iteration count
(relative image difference below 1e-4)."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

P = S.workload_large().problems[0]


def phantom_tensor(dtype):
    return torch.tensor(P.image().reshape(-1), dtype=dtype, device="cuda")


@pytest.mark.parametrize("prec,tol", [(wmg.PREC_F64, 1e-12), (wmg.PREC_F32, 2e-6)])
def test_sampled_rows_match_oracle(prec, tol):
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    plan = wmg.Plan(P.n, P.m, P.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=prec)
    x = phantom_tensor(dt)
    b = plan.project(x).double().cpu().numpy()
    xh = x.double().cpu().numpy()
    rng = np.random.default_rng(11)
    rows = rng.choice(P.m * P.D, 96, replace=False)
    for r in rows:
        col, val = oracle.ray_row(P.n, P.m, P.D, int(r // P.D), int(r % P.D))
        ref = float(np.dot(val, xh[col]))
        scale = float(np.dot(val, np.abs(xh[col]))) + 1e-300
        assert abs(b[r] - ref) <= tol * scale, (int(r), b[r], ref)
    plan.close()


def test_adjoint_full_size():
    plan = wmg.Plan(P.n, P.m, P.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.rand(P.N, dtype=torch.float64, device="cuda", generator=g)
    y = torch.rand(P.M, dtype=torch.float64, device="cuda", generator=g)
    lhs = torch.dot(plan.project(x), y).item()
    rhs = torch.dot(x, plan.backproject(y)).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    plan.close()


def test_mixed_precision_matches_fp64_path():
    lam = 1e-3 * P.m / P.n
    plan64 = wmg.Plan(P.n, P.m, P.D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    x_true = phantom_tensor(torch.float64)
    b = plan64.project(x_true)
    b = b + P.noise * b.abs().max() * torch.tensor(P.noise_unit(), dtype=torch.float64, device="cuda")
    plan64.close()
    xs = {}
    for prec in (wmg.PREC_F32, wmg.PREC_F64):
        pl = wmg.Plan(P.n, P.m, P.D, levels=P.levels, nu1=1, nu2=1, lam=lam, hybrid_depth=0,
                      cycle=wmg.CYCLE_ADDITIVE, precision=prec)
        bb = b.float().contiguous() if prec == wmg.PREC_F32 else b
        x, info, _, _ = pl.solve(bb, wmg.SOLVER_CGLS, True, 10, 0.0, 20)
        torch.cuda.synchronize()
        assert info[0][0] == 10
        xs[prec] = x.double()
        pl.close()
    diff = (torch.norm(xs[wmg.PREC_F32] - xs[wmg.PREC_F64]) / torch.norm(xs[wmg.PREC_F64])).item()
    assert diff < 1e-4, diff
