"""The FP32 leaf solves on the tensor cores (Section 3.1.2: exact solves of
the coarsest-level subproblems, many right-hand sides at once) against the
FP64 oracle.

The additive cycle without smoothing sweeps is z = Q blockdiag(D_k^-1) Q^T s
(the leaf solves between two orthogonal packet transforms), so its error is
that of the leaf solves. The F32 plan stores D_k^-1 rounded to FP32 and forms
the products from TF32 splits of both operands (about 2^-21 relative per
product, 256-term sums): measured 5e-7 .. 1.4e-6 of max|z| against the FP64
oracle, held here below 1e-5. Leaf sizes 16^2, 12^2 and 13^2 (an odd P, so
the K chunks and row blocks have ragged tails) and runs of 1, 70 and 300
problems (more than the four groups of 64 a tile's work items cover at
once). A problem computes the same bits alone and in the batch, call after
call."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [  # n, m, D, levels (leaf side n / 2^(levels-1)), problems
    (64, 90, 91, 3, 1),
    (64, 90, 91, 3, 70),
    (96, 60, 136, 4, 5),
    (104, 40, 148, 4, 3),
    (32, 30, 46, 2, 300),
]


@pytest.mark.parametrize("n,m,D,levels,count", CASES)
def test_leaf_solves_f32_match_oracle(n, m, D, levels, count):
    plan = wmg.Plan(n, m, D, levels=levels, nu1=0, nu2=0, hybrid_depth=0, cycle=wmg.CYCLE_ADDITIVE,
                    precision=wmg.PREC_F32)
    rng = np.random.default_rng(n + count)
    s = torch.tensor(rng.standard_normal(count * n * n), dtype=torch.float32, device="cuda")
    z = plan.precond(s)
    z2 = plan.precond(s)
    torch.cuda.synchronize()
    assert torch.equal(z, z2)
    zh = z.double().cpu().numpy()
    pre = oracle.Wmg(oracle.Op(n, m, D), levels, 0, 0, 1.0, 0.0, oracle.CYCLE_ADDITIVE, 0)
    for i in sorted({0, count // 2, count - 1}):
        sl = slice(i * n * n, (i + 1) * n * n)
        ref = pre.apply(s[sl].double().cpu().numpy())
        err = np.abs(zh[sl] - ref).max() / np.abs(ref).max()
        assert err < 1e-5, (i, err)
    last = slice((count - 1) * n * n, count * n * n)
    alone = plan.precond(s[last].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(alone, z[last])
    plan.close()


def test_leaf_solves_skip_inactive_problems_in_a_solve():
    """In a batched solve the problems that converged stop being solved for;
    the others' leaf solves, and so their iterates, do not change: a batch
    mixing a zero sinogram (converged at once) with real ones gives each real
    problem its bits alone."""
    n, m, D = 64, 90, 91
    op = oracle.Op(n, m, D)
    rng = np.random.default_rng(11)
    bs = [op.project(rng.random(n * n)) for _ in range(2)]
    batch = np.concatenate([bs[0], np.zeros(m * D), bs[1]])
    plan = wmg.Plan(n, m, D, levels=3, nu1=0, nu2=0, hybrid_depth=1, cycle=wmg.CYCLE_HYBRID,
                    precision=wmg.PREC_F32)
    bt = torch.tensor(batch, dtype=torch.float32, device="cuda")
    x, info, _, _ = plan.solve(bt, wmg.SOLVER_GMRES, True, max_iter=12, rtol=0.0)
    assert info[1][0] == 0
    for j, i in ((0, 0), (1, 2)):
        xa, _, _, _ = plan.solve(torch.tensor(bs[j], dtype=torch.float32, device="cuda"), wmg.SOLVER_GMRES, True,
                                 max_iter=12, rtol=0.0)
        torch.cuda.synchronize()
        assert torch.equal(xa, x[i * n * n:(i + 1) * n * n])
    plan.close()
