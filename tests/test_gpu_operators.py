"""GPU parity of the operators against the FP64 oracle, element by element:
forward projection W, backprojection W^T (Section 2.1), the Haar packet
transforms (Section 3.1), the leaf inverses and one WMG cycle."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

GEOMS = [  # n, m, D, dt, t0 -- tiny, odd/even D, axis angles, non-unit spacing, ragged tiles
    (4, 8, 7, 1.0, 0.0), (5, 7, 8, 1.0, 0.0), (8, 24, 12, 1.0, 0.0), (6, 10, 11, 0.75, 0.3),
    (16, 1, 23, 1.0, 0.0), (16, 40, 33, 1.0, 0.5), (32, 36, 46, 1.0, 0.0), (33, 20, 48, 1.0, 0.0),
    (40, 13, 57, 1.3, -0.7), (64, 90, 91, 1.0, 0.0),
]


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("n,m,D,dt,t0", GEOMS)
def test_project_backproject_f64(n, m, D, dt, t0):
    op = oracle.Op(n, m, D, dt, t0)
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64,
                    det_spacing=dt, det_offset=t0)
    rng = np.random.default_rng(n * 1000 + m)
    x, y = rng.standard_normal(op.N), rng.standard_normal(op.M)
    assert relmax(host(plan.project(dev(x))), op.project(x)) < 1e-13
    assert relmax(host(plan.backproject(dev(y))), op.backproject(y)) < 1e-13


@pytest.mark.parametrize("n,m,D", [(64, 90, 91), (32, 36, 46), (256, 180, 363)])
def test_project_backproject_f32(n, m, D):
    op = oracle.Op(n, m, D)
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F32)
    rng = np.random.default_rng(3)
    x, y = rng.random(op.N), rng.random(op.M)
    assert relmax(host(plan.project(dev(x, torch.float32))), op.project(x)) < 2e-6
    assert relmax(host(plan.backproject(dev(y, torch.float32))), op.backproject(y)) < 2e-6


def test_batched_projection_equals_single():
    n, m, D = 64, 90, 91
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    rng = np.random.default_rng(4)
    xs = rng.standard_normal((3, n * n))
    batched = host(plan.project(dev(xs.reshape(-1)))).reshape(3, -1)
    for i in range(3):
        single = host(plan.project(dev(xs[i])))
        assert np.array_equal(single, batched[i])


def test_adjointness_gpu():
    n, m, D = 64, 90, 91
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=wmg.PREC_F64)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal(n * n), rng.standard_normal(m * D)
    lhs = host(plan.project(dev(x))) @ y
    rhs = x @ host(plan.backproject(dev(y)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("n,levels", [(16, 3), (64, 3), (32, 4), (48, 4), (256, 5)])
def test_haar_packets(n, levels):
    L = levels - 1
    plan = wmg.Plan(n, 4, 2 * n, levels=levels, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE,
                    precision=wmg.PREC_F64, lam=1.0)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(n * n)
    c = host(plan.haar_analysis(dev(x)))
    assert relmax(c, oracle.packet_analysis(x, n, L)) < 1e-14
    xr = host(plan.haar_synthesis(dev(c)))
    assert relmax(xr, oracle.packet_synthesis(c, n, L)) < 1e-14


@pytest.mark.parametrize("n,m,D,levels,lam", [(16, 24, 23, 3, 0.0), (32, 36, 46, 3, 0.1), (64, 90, 91, 3, 0.0)])
def test_leaf_inverses(n, m, D, levels, lam):
    op = oracle.Op(n, m, D)
    ref = oracle.Wmg(op, levels, lam=lam, factor=False)
    plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, lam=lam, cycle=wmg.CYCLE_ADDITIVE,
                    precision=wmg.PREC_F64)
    for k in range(ref.K):
        Dk = ref.leaf(k)
        inv = host(plan.leaf_inverse(k))
        assert np.abs(inv @ Dk - np.eye(Dk.shape[0])).max() < 1e-9
        assert np.abs(inv - inv.T).max() < 1e-12 * np.abs(inv).max()


CYCLES = [  # levels, nu1, nu2, cycle, hybrid depth, lambda
    (3, 0, 0, wmg.CYCLE_ADDITIVE, 0, 0.0),
    (3, 1, 1, wmg.CYCLE_ADDITIVE, 0, 0.0),
    (3, 0, 0, wmg.CYCLE_HYBRID, 2, 0.0),
    (3, 1, 1, wmg.CYCLE_HYBRID, 2, 0.3),
    (4, 0, 0, wmg.CYCLE_HYBRID, 1, 0.0),
    (4, 1, 1, wmg.CYCLE_HYBRID, 3, 0.0),
    (3, 1, 1, wmg.CYCLE_SYMMETRIC, 2, 0.0),
    (4, 2, 1, wmg.CYCLE_SYMMETRIC, 2, 0.1),
    (3, 0, 0, wmg.CYCLE_MULTIPLICATIVE, 2, 0.0),
    (4, 0, 0, wmg.CYCLE_MULTIPLICATIVE, 1, 0.0),
    (4, 1, 1, wmg.CYCLE_MULTIPLICATIVE, 3, 0.2),
]


@pytest.mark.parametrize("levels,nu1,nu2,cycle,hd,lam", CYCLES)
def test_wmg_cycle(levels, nu1, nu2, cycle, hd, lam):
    n, m, D = 32, 36, 46
    op = oracle.Op(n, m, D)
    ref = oracle.Wmg(op, levels, nu1, nu2, 1.0, lam, cycle, hd)
    plan = wmg.Plan(n, m, D, levels=levels, nu1=nu1, nu2=nu2, lam=lam, hybrid_depth=hd, cycle=cycle,
                    precision=wmg.PREC_F64)
    rng = np.random.default_rng(7)
    s = rng.standard_normal((2, op.N))
    z = host(plan.precond(dev(s.reshape(-1)))).reshape(2, -1)
    for i in range(2):
        assert relmax(z[i], ref.apply(s[i])) < 1e-10


@pytest.mark.parametrize("prec", [wmg.PREC_F64, wmg.PREC_F32])
def test_launch_shapes_do_not_change_results(prec):
    """The autotuned grid shapes (CTAs per SM) give bitwise equal operators
    and solves."""
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    n, m, D = 64, 36, 91
    plan = wmg.Plan(n, m, D, levels=3, nu1=1, nu2=1, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID, precision=prec)
    x = torch.tensor(np.stack([S.phantom(n, 6, S.seed_for(7, i)).reshape(-1) for i in range(8)]).reshape(-1),
                     dtype=dt, device="cuda")
    plan.project(x)                      # fixes the problem count (the autotune runs here)
    outs = []
    for shape in ((1, 1), (16, 16), (3, 5)):
        plan.tuning(*shape)
        b = plan.project(x)
        assert plan.tuning() == shape
        y = plan.backproject(b)
        xs, _, _, _ = plan.solve(b, wmg.SOLVER_GMRES, True, 8, 0.0, 20)
        torch.cuda.synchronize()
        outs.append((b.clone(), y.clone(), xs.clone()))
    for o in outs[1:]:
        for a_, b_ in zip(outs[0], o):
            assert torch.equal(a_, b_)


TWO_H = [  # n, m, D, dt, t0, levels, cycle, hybrid depth, kernel, band updates on the 2h grid
    (64, 36, 91, 1.0, 0.0, 4, wmg.CYCLE_HYBRID, 1, wmg.KERNEL_STRIP, True),
    (64, 30, 110, 0.8, 0.3, 4, wmg.CYCLE_HYBRID, 1, wmg.KERNEL_STRIP, True),
    (64, 36, 91, 1.0, 0.0, 3, wmg.CYCLE_MULTIPLICATIVE, 2, wmg.KERNEL_STRIP, True),
    (32, 36, 46, 1.0, 0.0, 2, wmg.CYCLE_HYBRID, 1, wmg.KERNEL_STRIP, False),    # L = 1: no 2h grid
    (64, 36, 91, 1.0, 0.0, 4, wmg.CYCLE_HYBRID, 1, wmg.KERNEL_JOSEPH, False),   # weights do not add over blocks
]


@pytest.mark.parametrize("n,m,D,dt,t0,levels,cycle,hd,kernel,on2h", TWO_H)
def test_band_updates_on_the_2h_grid(n, m, D, dt, t0, levels, cycle, hd, kernel, on2h):
    """Band updates whose input lies in the first split's LL band project an
    n/2 x n/2 image on the 2h grid (Section 2.3; W I_{2h}^h c = W^{2h} c / 2
    for exact intersection lengths, L >= 2), the others on W's grid. The
    cycle matches the oracle's (FP64 plan at 1e-10, FP32 plan at 1e-4 on 11
    problems: groups of 8 staged by TMA and one-image tiles on the 2h grid),
    and a problem alone gets the bits it gets in the batch."""
    okernel = oracle.KERNEL_JOSEPH if kernel == wmg.KERNEL_JOSEPH else oracle.KERNEL_STRIP
    op = oracle.Op(n, m, D, dt=dt, t0=t0, kernel=okernel)
    ref = oracle.Wmg(op, levels, 0, 0, 1.0, 0.0, cycle, hd)
    rng = np.random.default_rng(n + m + levels)
    s = rng.standard_normal((11, op.N))
    for prec, tol in ((wmg.PREC_F64, 1e-10), (wmg.PREC_F32, 1e-4)):
        dtype = torch.float64 if prec == wmg.PREC_F64 else torch.float32
        plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, hybrid_depth=hd, cycle=cycle, precision=prec,
                        det_spacing=dt, det_offset=t0, kernel=kernel)
        z = host(plan.precond(dev(s.reshape(-1), dtype))).reshape(11, -1)
        for i in (0, 5, 10):
            assert relmax(z[i], ref.apply(s[i])) < tol, (prec, i)
        for i in (0, 10):
            alone = host(plan.precond(dev(s[i], dtype)))
            assert np.array_equal(alone, z[i]), (prec, i)
        b = plan.project(dev(s.reshape(-1), dtype))
        x = torch.empty_like(dev(s.reshape(-1), dtype))
        prof = plan.profile_step(b, x, 3, 0.0, 20)
        assert (prof["project_2h"]["launches"] > 0) == on2h, prof
        assert prof["project"]["launches"] > 0
        plan.close()
