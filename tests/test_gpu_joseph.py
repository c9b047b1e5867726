"""Joseph's kernel on the GPU (the paper's W, Section 2.1) against the FP64
oracle's Joseph operator: W and W^T element by element in FP64 and FP32
(unit and non-unit bins, offsets, odd and even angle and bin counts, a
detector narrower than the image, the 8-image group tiles), adjointness,
the nonzero count, the leaf Galerkin inverses, one WMG cycle, a WMG-GMRES
solve, the stored-matrix comparator, and the request server (a Joseph and a
strip request of the same sizes are different geometries)."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

J = wmg.KERNEL_JOSEPH
OJ = oracle.KERNEL_JOSEPH

GEOMS = [  # n, m, D, dt, t0
    (4, 8, 7, 1.0, 0.0), (5, 7, 8, 1.0, 0.0), (8, 24, 12, 1.0, 0.0), (6, 10, 11, 0.75, 0.3),
    (16, 40, 33, 1.0, 0.5), (32, 36, 46, 1.0, 0.0), (33, 20, 48, 1.0, 0.0), (40, 13, 57, 1.3, -0.7),
    (64, 90, 91, 1.0, 0.0), (40, 16, 40, 1.0, 0.0),
]


def dev(a, dtype=torch.float64):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def plan(n, m, D, dt=1.0, t0=0.0, prec=wmg.PREC_F64, levels=0, **kw):
    kw.setdefault("cycle", wmg.CYCLE_ADDITIVE)
    return wmg.Plan(n, m, D, levels=levels, nu1=kw.pop("nu1", 0), nu2=kw.pop("nu2", 0), precision=prec,
                    det_spacing=dt, det_offset=t0, kernel=J, **kw)


@pytest.mark.parametrize("n,m,D,dt,t0", GEOMS)
def test_project_backproject_f64(n, m, D, dt, t0):
    op = oracle.Op(n, m, D, dt, t0, kernel=OJ)
    p = plan(n, m, D, dt, t0)
    rng = np.random.default_rng(n * 1000 + m)
    x, y = rng.standard_normal(op.N), rng.standard_normal(op.M)
    assert relmax(host(p.project(dev(x))), op.project(x)) < 1e-13
    assert relmax(host(p.backproject(dev(y))), op.backproject(y)) < 1e-13


@pytest.mark.parametrize("n,m,D,dt,t0", [(64, 90, 91, 1.0, 0.0), (32, 36, 46, 1.0, 0.0), (256, 180, 363, 1.0, 0.0),
                                         (40, 13, 57, 1.3, -0.7), (40, 16, 40, 1.0, 0.0), (48, 31, 68, 1.0, 0.0)])
def test_project_backproject_f32(n, m, D, dt, t0):
    op = oracle.Op(n, m, D, dt, t0, kernel=OJ)
    p = plan(n, m, D, dt, t0, prec=wmg.PREC_F32)
    rng = np.random.default_rng(3)
    x, y = rng.random(op.N), rng.random(op.M)
    assert relmax(host(p.project(dev(x, torch.float32))), op.project(x)) < 3e-6
    assert relmax(host(p.backproject(dev(y, torch.float32))), op.backproject(y)) < 3e-6


def test_group_tiles_equal_single():
    # 9 images: one 8-image group tile (TMA-staged pixels) and one single tile
    n, m, D = 64, 30, 91
    grp, one = plan(n, m, D, prec=wmg.PREC_F32), plan(n, m, D, prec=wmg.PREC_F32)
    x = dev(np.random.default_rng(9).random(9 * n * n), torch.float32)
    q = grp.project(x)
    for i in range(9):
        assert torch.equal(one.project(x[i * n * n:(i + 1) * n * n].contiguous()), q[i * m * D:(i + 1) * m * D])


def test_adjointness_and_nnz():
    n, m, D = 64, 90, 91
    p = plan(n, m, D)
    rng = np.random.default_rng(5)
    x, y = rng.standard_normal(n * n), rng.standard_normal(m * D)
    lhs = host(p.project(dev(x))) @ y
    rhs = x @ host(p.backproject(dev(y)))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    _, _, val = oracle.Op(n, m, D, kernel=OJ).csr()
    assert p.nnz() == int(np.count_nonzero(val * n > 1e-12))


@pytest.mark.parametrize("n,m,D,levels,lam", [(16, 24, 23, 3, 0.0), (32, 36, 46, 3, 0.1)])
def test_leaf_inverses(n, m, D, levels, lam):
    op = oracle.Op(n, m, D, kernel=OJ)
    ref = oracle.Wmg(op, levels, lam=lam, factor=False)
    p = plan(n, m, D, levels=levels, lam=lam)
    for k in range(ref.K):
        Dk = ref.leaf(k)
        inv = host(p.leaf_inverse(k))
        assert np.abs(inv @ Dk - np.eye(Dk.shape[0])).max() < 1e-9


@pytest.mark.parametrize("cycle,hd,nu", [(wmg.CYCLE_ADDITIVE, 0, 1), (wmg.CYCLE_HYBRID, 2, 0)])
def test_wmg_cycle(cycle, hd, nu):
    n, m, D = 32, 36, 46
    op = oracle.Op(n, m, D, kernel=OJ)
    ref = oracle.Wmg(op, 3, nu, nu, 1.0, 0.0, cycle, hd)
    p = plan(n, m, D, levels=3, nu1=nu, nu2=nu, hybrid_depth=hd, cycle=cycle)
    s = np.random.default_rng(7).standard_normal(op.N)
    assert relmax(host(p.precond(dev(s))), ref.apply(s)) < 1e-10


def test_wmg_gmres_matches_oracle():
    n, m, D = 64, 60, 91
    op = oracle.Op(n, m, D, kernel=OJ)
    b = op.project(S.phantom(n, 6, S.seed_for(11, 1)))
    ref = oracle.Wmg(op, 3, 0, 0, 1.0, 0.0, oracle.CYCLE_HYBRID, 1)
    x_ref, k, _ = oracle.gmres(op, b, 12, 20, 0.0, 0.0, ref)
    p = plan(n, m, D, levels=3, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID)
    x, info, _, _ = p.solve(dev(b), wmg.SOLVER_GMRES, True, 12, 0.0, 20)
    assert info[0][0] == k == 12
    assert np.linalg.norm(host(x) - x_ref) / np.linalg.norm(x_ref) < 1e-10


def test_stored_matrix_comparator():
    n, m, D = 48, 40, 68
    p = plan(n, m, D, prec=wmg.PREC_F32)
    W, WT = p.csr(), p.csr(transposed=True)
    x = dev(np.random.default_rng(2).random(n * n), torch.float32)
    y = dev(np.random.default_rng(3).random(m * D), torch.float32)
    assert relmax(host(W.apply(x)), host(p.project(x))) < 3e-6
    assert relmax(host(WT.apply(y)), host(p.backproject(y))) < 3e-6
    assert W.nnz == p.nnz()


def test_server_keeps_kernels_apart():
    n, m, D = 32, 24, 46
    reqs = [dict(n=n, m=m, D=D, levels=3, kernel=J), dict(n=n, m=m, D=D, levels=3)]
    srv = wmg.Server(1 << 30, max_slots=4, preconditioned=True, max_iter=30, rtol=1e-6, restart=10, levels=3,
                     nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID, precision=wmg.PREC_F64)
    xs = []
    tickets = []
    for i, r in enumerate(reqs):
        op = oracle.Op(n, m, D, kernel=OJ if r.get("kernel") == J else oracle.KERNEL_STRIP)
        b = dev(op.project(S.phantom(n, 5, S.seed_for(12, i))))
        tickets.append((srv.submit(r, b), r, b))
    done = {}
    for _ in range(10000):
        pending = srv.step()
        for t, _, _ in tickets:
            got = srv.poll(t) if t not in done else None
            if got is not None:
                done[t] = got
        if pending == 0 and len(done) == len(tickets):
            break
    st = srv.stats()
    srv.close()
    assert st["geometry_setups"] == 2
    for t, r, b in tickets:
        pl = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                      precision=wmg.PREC_F64, kernel=r.get("kernel", wmg.KERNEL_STRIP))
        x, info, _, _ = pl.solve(b, wmg.SOLVER_GMRES, True, 30, 1e-6, 10)
        torch.cuda.synchronize()
        assert info[0][0] == done[t][1][0]
        assert torch.equal(x, done[t][0])
        pl.close()
