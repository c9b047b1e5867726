"""Stored-matrix comparator: W and W^T assembled as CSR on the device must
have exactly the oracle's nonzero count (entries above 1e-12 pixel widths)
and the matrix-free kernels' count, and
their products must equal the matrix-free projector / backprojector up to
summation order (FP64) or FP32 rounding (F32)."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

GEOMS = [(32, 24, 46, 1.0, 0.0), (48, 30, 68, 1.0, 0.0), (40, 17, 57, 1.0, 0.0), (32, 20, 40, 1.25, 0.5),
         (64, 90, 91, 1.0, 0.0)]


@pytest.mark.parametrize("n,m,D,dt,t0", GEOMS)
def test_nnz_matches_oracle(n, m, D, dt, t0):
    op = oracle.Op(n, m, D, dt, t0)
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, det_spacing=dt, det_offset=t0)
    Wc, WTc = plan.csr(False), plan.csr(True)
    # nonzeros = chords above 1e-12 pixel widths (lines through a pixel corner
    # leave rounding-size chords on either side)
    nnz_ref = int((op.csr()[2] > 1e-12 / n).sum())
    assert plan.nnz() == nnz_ref == Wc.nnz == WTc.nnz
    assert (Wc.rows, Wc.cols, WTc.rows, WTc.cols) == (op.M, op.N, op.N, op.M)


@pytest.mark.parametrize("prec,tol", [(wmg.PREC_F64, 1e-13), (wmg.PREC_F32, 2e-6)])
@pytest.mark.parametrize("n,m,D,dt,t0", GEOMS)
def test_stored_equals_matrix_free(n, m, D, dt, t0, prec, tol):
    dtp = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    plan = wmg.Plan(n, m, D, levels=0, nu1=0, nu2=0, cycle=wmg.CYCLE_ADDITIVE, precision=prec,
                    det_spacing=dt, det_offset=t0)
    x = torch.tensor(np.stack([S.phantom(n, 5, S.seed_for(6, i)).reshape(-1) for i in range(3)]).reshape(-1),
                     dtype=dtp, device="cuda")
    b = plan.project(x)
    b_csr = plan.csr(False).apply(x)
    y = torch.rand(3 * m * D, dtype=dtp, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    z = plan.backproject(y)
    z_csr = plan.csr(True).apply(y)
    torch.cuda.synchronize()
    assert (torch.norm(b - b_csr) / torch.norm(b)).item() < tol
    assert (torch.norm(z - z_csr) / torch.norm(z)).item() < tol
