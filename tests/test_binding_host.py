"""Host logic of the Python binding (argument marshalling only): problem
counts derived from the tensors, outputs of the wrong size refused before
any library call (a short output would be written past its end on the
device), and the count passed to the library's resume call. The library
calls are replaced by recorders and the tensors are CPU tensors."""
import pytest

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402


def _arg_cpu(self, t, size):
    if t.dtype != self.dtype or not t.is_contiguous():
        raise TypeError("dtype")
    if t.numel() % size:
        raise ValueError("size")
    return t.data_ptr(), t.numel() // size


@pytest.fixture
def plan(monkeypatch):
    monkeypatch.setattr(wmg.Plan, "_arg", _arg_cpu)
    p = object.__new__(wmg.Plan)
    p._torch, p.dtype, p.N, p.M, p.handle = torch, torch.float64, 4, 6, None
    p._stream = lambda: None
    return p


def test_resume_passes_the_problem_count(plan, monkeypatch):
    calls = []

    def rec(handle, count, b, x, max_iter, rtol, info, hist, stream, allow=()):
        calls.append((count, b, x, max_iter, rtol))
        for i in range(count):
            info[i].iters, info[i].status = max_iter, 1
        return 1
    monkeypatch.setattr(wmg, "wmg_solve_resume", rec)
    b = torch.zeros(2 * 6, dtype=torch.float64)
    x, infos, hists, rc = plan.resume(b, 9, 0.0)
    assert calls == [(2, b.data_ptr(), x.data_ptr(), 9, 0.0)]
    assert x.numel() == 2 * 4 and infos == [(9, 1, 0.0), (9, 1, 0.0)] and rc == 1
    with pytest.raises(ValueError):
        plan.resume(b, 9, 0.0, out=torch.zeros(4, dtype=torch.float64))
    assert len(calls) == 1


def test_outputs_of_the_wrong_size_are_refused(plan, monkeypatch):
    def never(*a, **kw):
        raise AssertionError("the library was called")
    for name in ("wmg_solve", "wmg_solve_x0", "wmg_project", "wmg_backproject", "wmg_precond_apply",
                 "wmg_haar_analysis", "wmg_haar_synthesis"):
        monkeypatch.setattr(wmg, name, never)
    x2 = torch.zeros(2 * 4, dtype=torch.float64)
    b2 = torch.zeros(2 * 6, dtype=torch.float64)
    one_img = torch.zeros(4, dtype=torch.float64)
    with pytest.raises(ValueError):
        plan.solve(b2, wmg.SOLVER_GMRES, True, 5, 0.0, out=one_img)
    with pytest.raises(ValueError):
        plan.solve(b2, wmg.SOLVER_GMRES, True, 5, 0.0, x0=one_img)
    with pytest.raises(ValueError):
        plan.project(x2, out=torch.zeros(6, dtype=torch.float64))
    with pytest.raises(ValueError):
        plan.backproject(b2, out=one_img)
    for f in (plan.precond, plan.haar_analysis, plan.haar_synthesis):
        with pytest.raises(ValueError):
            f(x2, out=one_img)


def test_solve_from_x0_marshals_both_buffers(plan, monkeypatch):
    calls = []

    def rec(handle, solver, pre, count, b, x0, x, max_iter, rtol, restart, info, hist, stream, allow=()):
        calls.append((solver, pre, count, b, x0, x, max_iter, restart))
        return 0
    monkeypatch.setattr(wmg, "wmg_solve_x0", rec)
    b2 = torch.zeros(2 * 6, dtype=torch.float64)
    x0 = torch.ones(2 * 4, dtype=torch.float64)
    x, _, _, _ = plan.solve(b2, wmg.SOLVER_BICGSTAB, False, 7, 0.0, 20, x0=x0)
    assert calls == [(wmg.SOLVER_BICGSTAB, 0, 2, b2.data_ptr(), x0.data_ptr(), x.data_ptr(), 7, 20)]


def test_batch_needs_every_problem():
    bt = object.__new__(wmg.Batch)
    bt._torch, bt.dtype, bt.count, bt.handle = torch, torch.float64, 2, None
    bt.sizes = [(4, 6), (9, 12)]
    b0 = torch.zeros(6, dtype=torch.float64)
    outs = [torch.zeros(4, dtype=torch.float64), torch.zeros(9, dtype=torch.float64)]
    # checked before any tensor: a short list would leave the library reading
    # pointers past the end of the array it is given
    with pytest.raises(ValueError):
        bt.solve([b0], outs=outs)
    with pytest.raises(ValueError):
        bt.solve([b0, torch.zeros(12, dtype=torch.float64)], outs=outs[:1])


def test_noalloc_projection_checks_its_buffers(monkeypatch):
    # a short b would be written past its end on the device: every size,
    # dtype and device is checked before the library is reached
    def never():
        raise AssertionError("the library was called")
    monkeypatch.setattr(wmg, "lib", never)
    n, m, D = 8, 5, 13
    x = torch.zeros(n * n, dtype=torch.float32)
    b = torch.zeros(m * D, dtype=torch.float32)
    with pytest.raises(ValueError):
        wmg.wmg_project_noalloc(n, m, D, x, torch.zeros(m * D - 1, dtype=torch.float32))
    with pytest.raises(ValueError):
        wmg.wmg_project_noalloc(n, m, D, torch.zeros(n * n + 1, dtype=torch.float32), b)
    with pytest.raises(TypeError):
        wmg.wmg_project_noalloc(n, m, D, x, b)                  # host tensors
    with pytest.raises(TypeError):
        wmg.wmg_project_noalloc(n, m, D, x.data_ptr(), b)       # a raw pointer


def test_problem_statuses_are_returned_only_when_asked(plan, monkeypatch):
    # a breakdown ends its problem with the last iterate in x: solve raises
    # by default, and returns the status (with x and info) when asked
    def rec(handle, solver, pre, count, b, x, max_iter, rtol, restart, info, hist, stream, allow=()):
        info[0].iters, info[0].status = 3, wmg.WMG_ERR_BREAKDOWN
        return wmg._check(wmg.WMG_ERR_BREAKDOWN, True, allow)
    monkeypatch.setattr(wmg, "wmg_solve", rec)
    b = torch.zeros(6, dtype=torch.float64)
    with pytest.raises(wmg.WmgError):
        plan.solve(b, wmg.SOLVER_BICGSTAB, False, 9, 0.0)
    x, infos, _, rc = plan.solve(b, wmg.SOLVER_BICGSTAB, False, 9, 0.0, problem_errors=False)
    assert rc == wmg.WMG_ERR_BREAKDOWN and infos[0][:2] == (3, wmg.WMG_ERR_BREAKDOWN) and x.numel() == 4
    with pytest.raises(wmg.WmgError):                  # errors of the call itself still raise
        wmg._check(wmg.WMG_ERR_INVALID_ARG, True, wmg.PROBLEM_STATUSES)
