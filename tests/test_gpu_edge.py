"""Edge cases: an all-zero sinogram (the solution is 0: every solver stops at
once with WMG_OK), a non-finite sinogram (WMG_ERR_NAN, no fault), a batch
where some problems are empty and others are not (the others unaffected),
degenerate geometries (one angle, one bin, rays that miss the image, a 2x2
image) against the oracle, and the largest image side (2048, 720 angles) on
sampled rows."""
import math

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

SOLVERS = [wmg.SOLVER_CGLS, wmg.SOLVER_GMRES, wmg.SOLVER_BICGSTAB, wmg.SOLVER_SIRT]


def plan(prec, n=32, m=24, D=46, cycle=wmg.CYCLE_ADDITIVE, hd=0, levels=3):
    return wmg.Plan(n, m, D, levels=levels, nu1=1, nu2=1, hybrid_depth=hd, cycle=cycle, precision=prec)


@pytest.mark.parametrize("prec", [wmg.PREC_F64, wmg.PREC_F32])
@pytest.mark.parametrize("solver", SOLVERS)
def test_zero_sinogram(prec, solver):
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    p = plan(prec)
    b = torch.zeros(p.M, dtype=dt, device="cuda")
    x, info, _, rc = p.solve(b, solver, solver != wmg.SOLVER_SIRT, 20, 1e-6)
    assert rc == wmg.WMG_OK and info[0][1] == wmg.WMG_OK and info[0][2] == 0.0
    # SIRT runs its fixed iteration count (eq. sirt_it); the Krylov solvers stop at once
    assert info[0][0] == (20 if solver == wmg.SOLVER_SIRT else 0)
    assert torch.count_nonzero(x).item() == 0


@pytest.mark.parametrize("solver", [wmg.SOLVER_CGLS, wmg.SOLVER_GMRES, wmg.SOLVER_BICGSTAB])
def test_non_finite_sinogram(solver):
    p = plan(wmg.PREC_F64)
    b = torch.ones(p.M, dtype=torch.float64, device="cuda")
    b[17] = float("nan")
    with pytest.raises(wmg.WmgError) as e:
        p.solve(b, solver, True, 20, 1e-6)
    assert e.value.code == -7                       # WMG_ERR_NAN
    # the plan (and the GPU context) stays usable
    x, info, _, rc = p.solve(torch.zeros(p.M, dtype=torch.float64, device="cuda"), solver, True, 20, 1e-6)
    assert rc == wmg.WMG_OK


@pytest.mark.parametrize("solver", [wmg.SOLVER_CGLS, wmg.SOLVER_GMRES, wmg.SOLVER_BICGSTAB])
def test_empty_problems_in_a_batch(solver):
    n, m, D = 32, 24, 46
    p = plan(wmg.PREC_F32)
    op = oracle.Op(n, m, D)
    imgs = [S.phantom(n, 5, S.seed_for(9, i)) if i % 2 else np.zeros(n * n) for i in range(6)]
    bs = np.stack([op.project(x) for x in imgs])
    b = torch.tensor(bs.reshape(-1), dtype=torch.float32, device="cuda")
    x_all, info_all, _, _ = p.solve(b, solver, True, 40, 1e-6)
    single = plan(wmg.PREC_F32)
    for i in range(6):
        x1, info1, _, _ = single.solve(b[i * p.M:(i + 1) * p.M].contiguous(), solver, True, 40, 1e-6)
        torch.cuda.synchronize()
        assert info1[0][:2] == info_all[i][:2]
        assert torch.equal(x1, x_all[i * p.N:(i + 1) * p.N])
        if i % 2 == 0:
            assert info_all[i][0] == 0 and torch.count_nonzero(x1).item() == 0


@pytest.mark.parametrize("geom", [(16, 1, 23, 1.0, 0.0), (16, 12, 1, 1.0, 0.0), (16, 7, 9, 1.0, 40.0),
                                  (2, 5, 3, 1.0, 0.0), (9, 8, 13, 0.7, 0.3)])
@pytest.mark.parametrize("prec,tol", [(wmg.PREC_F64, 1e-13), (wmg.PREC_F32, 3e-6)])
def test_degenerate_geometries(geom, prec, tol):
    n, m, D, dt_, t0 = geom
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    op = oracle.Op(n, m, D, dt_, t0)
    p = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=prec,
                 det_spacing=dt_, det_offset=t0)
    rng = np.random.default_rng(3)
    x = rng.random(n * n)
    y = rng.random(m * D)
    b = p.project(torch.tensor(x, dtype=dt, device="cuda")).double().cpu().numpy()
    z = p.backproject(torch.tensor(y, dtype=dt, device="cuda")).double().cpu().numpy()
    bref, zref = op.project(x), op.backproject(y)
    sb = max(np.abs(bref).max(), 1e-300)
    sz = max(np.abs(zref).max(), 1e-300)
    assert np.abs(b - bref).max() <= tol * sb
    assert np.abs(z - zref).max() <= tol * sz
    if t0 == 40.0:                                  # every ray misses the image
        assert not bref.any() and not b.any() and not z.any()


@pytest.mark.slow
def test_largest_image_sampled_rows():
    n, m = 2048, 720
    D = S.detectors_for(n)
    p = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)
    x = torch.tensor(S.phantom(n, 40, S.seed_for(4, 7)).reshape(-1), dtype=torch.float32, device="cuda")
    b = p.project(x).double().cpu().numpy()
    xh = x.double().cpu().numpy()
    rng = np.random.default_rng(21)
    for r in rng.choice(m * D, 48, replace=False):
        col, val = oracle.ray_row(n, m, D, int(r // D), int(r % D))
        ref = float(np.dot(val, xh[col]))
        scale = float(np.dot(val, np.abs(xh[col]))) + 1e-300
        assert abs(b[r] - ref) <= 3e-6 * scale, (int(r), b[r], ref)
