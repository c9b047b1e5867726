"""Batches of problems with different geometries (image side, angle count,
bins, WMG levels) solved together, one launch per operator application: each
problem must give bitwise the same reconstruction as when solved alone with
its own plan, and the same as the FP64 oracle within the solver tolerances."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

PROBLEMS = [  # n, m, D, levels
    dict(n=32, m=24, D=46, levels=3), dict(n=48, m=30, D=68, levels=3), dict(n=32, m=24, D=46, levels=3),
    dict(n=64, m=36, D=91, levels=3), dict(n=24, m=20, D=34, levels=2),
]


def sinograms(problems):
    out = []
    for i, p in enumerate(problems):
        op = oracle.Op(p["n"], p["m"], p["D"])
        x = S.phantom(p["n"], 5, S.seed_for(3, 100 + i))
        b = op.project(x)
        b = b + 0.01 * np.abs(b).max() * S.noise_draws(op.M, S.seed_for(3, 100 + i))
        out.append((op, b))
    return out


@pytest.mark.parametrize("prec,cycle,hd,solver", [
    (wmg.PREC_F64, wmg.CYCLE_HYBRID, 1, wmg.SOLVER_GMRES),
    (wmg.PREC_F32, wmg.CYCLE_HYBRID, 2, wmg.SOLVER_GMRES),
    (wmg.PREC_F64, wmg.CYCLE_ADDITIVE, 0, wmg.SOLVER_CGLS),
    (wmg.PREC_F32, wmg.CYCLE_SYMMETRIC, 1, wmg.SOLVER_CGLS),
])
def test_batch_equals_alone(prec, cycle, hd, solver):
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    data = sinograms(PROBLEMS)
    batch = wmg.Batch(PROBLEMS, nu1=1, nu2=1, hybrid_depth=hd, cycle=cycle, precision=prec)
    bs = [torch.tensor(b, dtype=dt, device="cuda") for _, b in data]
    xs, infos, rc = batch.solve(bs, solver, True, max_iter=40, rtol=1e-6)
    torch.cuda.synchronize()
    for i, p in enumerate(PROBLEMS):
        plan = wmg.Plan(p["n"], p["m"], p["D"], levels=p["levels"], nu1=1, nu2=1, hybrid_depth=hd,
                        cycle=cycle, precision=prec)
        x1, info1, _, _ = plan.solve(bs[i], solver, True, max_iter=40, rtol=1e-6)
        torch.cuda.synchronize()
        assert info1[0][0] == infos[i][0]
        assert torch.equal(x1, xs[i]), i
        plan.close()


def test_batch_matches_oracle_f64():
    data = sinograms(PROBLEMS[:2])
    batch = wmg.Batch(PROBLEMS[:2], nu1=1, nu2=1, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F64)
    xs, infos, _ = batch.solve([torch.tensor(b, dtype=torch.float64, device="cuda") for _, b in data],
                               wmg.SOLVER_GMRES, True, max_iter=12, rtol=0.0)
    for i, p in enumerate(PROBLEMS[:2]):
        op, b = data[i]
        M = oracle.Wmg(op, p["levels"], 1, 1, 1.0, 0.0, oracle.CYCLE_HYBRID, 1)
        x_ref, k, _ = oracle.gmres(op, b, 12, 20, 0.0, 0.0, M)
        x = xs[i].cpu().numpy()
        assert infos[i][0] == k == 12
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10


def test_batch_mixed_bin_spacing_equals_alone():
    # a geometry with wider, offset bins in the batch must not change how the
    # unit-bin problems are computed (the FP32 backprojector picks its path
    # per geometry), and vice versa
    probs = [dict(n=32, m=24, D=46, levels=3), dict(n=32, m=24, D=40, levels=3, det_spacing=1.25, det_offset=0.5),
             dict(n=24, m=20, D=34, levels=2)]
    bs = []
    for i, p in enumerate(probs):
        op = oracle.Op(p["n"], p["m"], p["D"], p.get("det_spacing", 1.0), p.get("det_offset", 0.0))
        b = op.project(S.phantom(p["n"], 5, S.seed_for(3, 300 + i)))
        bs.append(torch.tensor(b, dtype=torch.float32, device="cuda"))
    batch = wmg.Batch(probs, nu1=1, nu2=1, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32)
    xs, infos, _ = batch.solve(bs, wmg.SOLVER_GMRES, True, max_iter=30, rtol=1e-6)
    torch.cuda.synchronize()
    for i, p in enumerate(probs):
        plan = wmg.Plan(p["n"], p["m"], p["D"], levels=p["levels"], nu1=1, nu2=1, hybrid_depth=1,
                        cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F32, det_spacing=p.get("det_spacing", 1.0),
                        det_offset=p.get("det_offset", 0.0))
        x1, info1, _, _ = plan.solve(bs[i], wmg.SOLVER_GMRES, True, max_iter=30, rtol=1e-6)
        torch.cuda.synchronize()
        plan.close()
        assert info1[0][0] == infos[i][0]
        assert torch.equal(x1, xs[i]), i


@pytest.mark.parametrize("solver,cycle", [(wmg.SOLVER_GMRES, wmg.CYCLE_HYBRID), (wmg.SOLVER_CGLS, wmg.CYCLE_ADDITIVE)])
def test_grouped_projector_tiles_equal_single(solver, cycle):
    # 11 problems of one geometry: the FP32 projector runs the first 8 as one
    # group tile (weights shared) and the other 3 one image per tile; every
    # problem must give the same bits as when solved alone
    n, m, D = 48, 30, 68
    plan = wmg.Plan(n, m, D, levels=3, nu1=1, nu2=1, hybrid_depth=1, cycle=cycle, precision=wmg.PREC_F32)
    op = oracle.Op(n, m, D)
    bs = np.stack([op.project(S.phantom(n, 5, S.seed_for(3, 400 + i))) for i in range(11)])
    b = torch.tensor(bs.reshape(-1), dtype=torch.float32, device="cuda")
    q_all = plan.project(torch.tensor(np.stack([S.phantom(n, 5, S.seed_for(3, 500 + i)).reshape(-1)
                                                for i in range(11)]).reshape(-1), dtype=torch.float32,
                                      device="cuda"))
    x_all, info_all, _, _ = plan.solve(b, solver, True, 25, 1e-6, 20)
    torch.cuda.synchronize()
    single = wmg.Plan(n, m, D, levels=3, nu1=1, nu2=1, hybrid_depth=1, cycle=cycle, precision=wmg.PREC_F32)
    for i in range(11):
        xi = torch.tensor(S.phantom(n, 5, S.seed_for(3, 500 + i)).reshape(-1), dtype=torch.float32, device="cuda")
        assert torch.equal(single.project(xi), q_all[i * m * D:(i + 1) * m * D]), i
        x1, info1, _, _ = single.solve(b[i * m * D:(i + 1) * m * D].contiguous(), solver, True, 25, 1e-6, 20)
        torch.cuda.synchronize()
        assert info1[0][0] == info_all[i][0]
        assert torch.equal(x1, x_all[i * n * n:(i + 1) * n * n]), i
    plan.close()
    single.close()


@pytest.mark.parametrize("geom", [(256, 36, 363, 1.0, 0.0), (64, 40, 140, 0.7, 0.3), (52, 17, 60, 1.0, -2.5),
                                  (36, 12, 200, 0.5, 0.0), (30, 20, 45, 1.0, 0.0)])
def test_grouped_projection_equals_single(geom):
    # group tiles (8 images sharing the weights; their pixels staged in
    # shared memory where the image side is a multiple of 4) against one
    # image per tile: bitwise equal, and within the FP32 bound of the oracle.
    # Geometries: the workload's, finer offset bins, a detector wider than
    # the image (rays that miss it), and a side that is not a multiple of 4.
    n, m, D, dt, t0 = geom
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32,
                    det_spacing=dt, det_offset=t0)
    single = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32,
                      det_spacing=dt, det_offset=t0)
    imgs = np.stack([S.phantom(n, 6, S.seed_for(8, 40 + i)).reshape(-1) for i in range(9)])
    x = torch.tensor(imgs.reshape(-1), dtype=torch.float32, device="cuda")
    q = plan.project(x)
    torch.cuda.synchronize()
    op = oracle.Op(n, m, D, dt, t0)
    for i in range(9):
        qi = single.project(x[i * n * n:(i + 1) * n * n].contiguous())
        assert torch.equal(qi, q[i * m * D:(i + 1) * m * D]), i
    ref = op.project(imgs[3])
    got = q[3 * m * D:4 * m * D].double().cpu().numpy()
    assert np.abs(got - ref).max() <= 3e-6 * max(np.abs(ref).max(), 1e-300)
    plan.close()
    single.close()


@pytest.mark.parametrize("prec,solver,cycle", [
    (wmg.PREC_F64, wmg.SOLVER_GMRES, wmg.CYCLE_HYBRID),
    (wmg.PREC_F32, wmg.SOLVER_GMRES, wmg.CYCLE_HYBRID),
    (wmg.PREC_F32, wmg.SOLVER_CGLS, wmg.CYCLE_ADDITIVE),
    (wmg.PREC_F64, wmg.SOLVER_BICGSTAB, wmg.CYCLE_HYBRID),
])
def test_solvers_on_the_problems_left_equal_alone(prec, solver, cycle):
    """Batched solves whose problems stop at different iterations: once few
    are left, the solver runs the remaining problems' work lists only (the
    stopped slots get no tiles, the WMG cycle walks the remaining slots; for
    GMRES also without the problems whose cycle has ended, until the cycle
    end). Every problem keeps the bits it gets alone: iterate, iteration
    count, status and residual. Four zero sinograms stop before the first
    iteration; noiseless and noisy phantoms, at 1e-4 (GMRES restarted every 5
    iterations), stop at different iterations (GMRES: 14 .. 23 in the
    oracle)."""
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    n, m, D = 64, 90, 91
    op = oracle.Op(n, m, D)
    bs = []
    for i in range(12):
        if i % 3 == 1:
            bs.append(np.zeros(op.M))
            continue
        b = op.project(S.phantom(n, 3 + i, S.seed_for(8, i)))
        noise = 0.0 if i % 3 == 0 else 0.002 * i
        bs.append(b + noise * np.abs(b).max() * S.noise_draws(op.M, S.seed_for(8, i)))
    hd = 0 if cycle == wmg.CYCLE_ADDITIVE else 1
    plan = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, hybrid_depth=hd, cycle=cycle, precision=prec)
    bt = torch.tensor(np.concatenate(bs), dtype=dt, device="cuda")
    x, info, _, _ = plan.solve(bt, solver, True, max_iter=80, rtol=1e-4, restart=5)
    torch.cuda.synchronize()
    iters = [i[0] for i in info]
    assert all(i[1] == 0 for i in info), info
    if solver == wmg.SOLVER_GMRES:
        assert len({(k - 1) // 5 for k in iters if k > 0}) >= 2, iters   # stopped in different cycles
    else:
        assert len({k for k in iters if k > 0}) >= 3, iters
    for i in range(12):
        xa, ia, _, _ = plan.solve(torch.tensor(bs[i], dtype=dt, device="cuda"), solver, True,
                                  max_iter=80, rtol=1e-4, restart=5)
        torch.cuda.synchronize()
        assert ia[0] == info[i], i
        assert torch.equal(xa, x[i * n * n:(i + 1) * n * n]), i
    # and the batch again (the plan's own work lists were restored)
    x2, info2, _, _ = plan.solve(bt, solver, True, max_iter=80, rtol=1e-4, restart=5)
    torch.cuda.synchronize()
    assert info2 == info and torch.equal(x2, x)
    plan.close()


@pytest.mark.parametrize("n,m,D,levels", [(32, 24, 48, 2), (64, 36, 92, 3)])
def test_backprojection_group_tiles_equal_one_image_tiles(n, m, D, levels):
    """FP32 backprojection of 11 problems of one geometry whose bins cover
    every pixel tile and whose angles come in quarter-turn pairs: the first 8
    run the group tiles (shared bins and weights, staged sinogram windows),
    the other 3 one-image tiles. Every problem equals its backprojection
    alone bit for bit, and the FP64 oracle's W^T to FP32 rounding; the same
    for the fused epilogue of a CGLS solve."""
    op = oracle.Op(n, m, D)
    plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)
    rng = np.random.default_rng(n + m)
    ys = rng.random((11, op.M))
    yt = torch.tensor(ys.reshape(-1), dtype=torch.float32, device="cuda")
    batch = plan.backproject(yt)
    torch.cuda.synchronize()
    batch_h = batch.double().cpu().numpy().reshape(11, -1)
    for i in range(11):
        alone = plan.backproject(yt[i * op.M:(i + 1) * op.M].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(alone, batch[i * op.N:(i + 1) * op.N]), i
        ref = op.backproject(ys[i].astype(np.float32).astype(np.float64))
        assert np.abs(batch_h[i] - ref).max() <= 2e-6 * np.abs(ref).max(), i
    bs = [op.project(S.phantom(n, 4, S.seed_for(9, i))) for i in range(11)]
    bt = torch.tensor(np.concatenate(bs), dtype=torch.float32, device="cuda")
    x, info, _, _ = plan.solve(bt, wmg.SOLVER_CGLS, True, max_iter=6, rtol=0.0)
    torch.cuda.synchronize()
    for i in (0, 7, 10):
        xa, ia, _, _ = plan.solve(bt[i * op.M:(i + 1) * op.M].contiguous(), wmg.SOLVER_CGLS, True, max_iter=6,
                                  rtol=0.0)
        torch.cuda.synchronize()
        assert ia[0] == info[i] and torch.equal(xa, x[i * op.N:(i + 1) * op.N]), i
    plan.close()
