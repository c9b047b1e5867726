"""Continuous-batching server: requests of different geometries arrive while
others run, are admitted as slots and memory free up, share every operator
launch, and retire when converged. Each request must give bitwise the same
reconstruction alone, in the mix, and through wmg_solve on its own plan, and
the FP64 oracle's GMRES result within 1e-10 after the same iteration count."""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
import paper_1310_0956_gb300 as wmg  # noqa: E402

pytestmark = pytest.mark.gpu

ANGLES_IRREGULAR = list(np.sort(np.random.default_rng(7).uniform(0.0, np.pi, 22)))
REQUESTS = [  # n, m, D, levels (one with an explicit, irregular angle set)
    dict(n=32, m=24, D=46, levels=3), dict(n=48, m=30, D=68, levels=3), dict(n=32, m=24, D=46, levels=3),
    dict(n=24, m=20, D=34, levels=2), dict(n=32, m=22, D=46, levels=3, angles=ANGLES_IRREGULAR),
    dict(n=64, m=36, D=91, levels=3),
]
RESTART, MAX_ITER, RTOL = 5, 40, 1e-6


def sinograms(reqs, dtype):
    out = []
    for i, p in enumerate(reqs):
        op = oracle.Op(p["n"], p["m"], p["D"], angles=p.get("angles"))
        x = S.phantom(p["n"], 5, S.seed_for(5, 200 + i))
        b = op.project(x)
        b = b + 0.01 * np.abs(b).max() * S.noise_draws(op.M, S.seed_for(5, 200 + i))
        out.append((op, torch.tensor(b, dtype=dtype, device="cuda")))
    return out


def run_to_end(srv, tickets, max_ticks=10000):
    done = {}
    for _ in range(max_ticks):
        pending = srv.step()
        for t in list(tickets):
            r = srv.poll(t)
            if r is not None:
                done[t] = r
                tickets.remove(t)
        if pending == 0 and not tickets:
            return done
    raise AssertionError("server did not drain")


def make_server(prec, pre=True, budget=1 << 30, state=0, slots=3, max_iter=MAX_ITER, rtol=RTOL):
    return wmg.Server(budget, max_slots=slots, state_bytes=state, preconditioned=pre, max_iter=max_iter,
                      rtol=rtol, restart=RESTART, levels=3, nu1=1, nu2=1, hybrid_depth=1,
                      cycle=wmg.CYCLE_HYBRID, precision=prec)


@pytest.mark.parametrize("prec,pre", [(wmg.PREC_F64, True), (wmg.PREC_F32, True), (wmg.PREC_F32, False)])
def test_mix_equals_alone_and_plan(prec, pre):
    dt = torch.float64 if prec == wmg.PREC_F64 else torch.float32
    data = sinograms(REQUESTS, dt)
    srv = make_server(prec, pre)
    # staggered arrivals: two, then two more after two ticks, then the rest
    tickets, order = [], []
    for i in (0, 1):
        tickets.append(srv.submit(REQUESTS[i], data[i][1])); order.append(i)
    srv.step(); srv.step()
    for i in (2, 3):
        tickets.append(srv.submit(REQUESTS[i], data[i][1])); order.append(i)
    srv.step()
    for i in (4, 5):
        tickets.append(srv.submit(REQUESTS[i], data[i][1])); order.append(i)
    by_ticket = dict(zip(tickets, order))
    done = run_to_end(srv, list(tickets))
    st = srv.stats()
    assert st["completed"] == len(REQUESTS) and st["running"] == 0 and st["queued"] == 0
    assert st["geometry_setups"] == 5                     # requests 0 and 2 share a geometry
    srv.close()
    mixed = {by_ticket[t]: r for t, r in done.items()}
    for i, p in enumerate(REQUESTS):
        x_mix, info_mix, _ = mixed[i]
        assert info_mix[1] in (wmg.WMG_OK, wmg.WMG_NOT_CONVERGED), (i, info_mix)
        alone = make_server(prec, pre)
        t = alone.submit(p, data[i][1])
        x_alone, info_alone, _ = run_to_end(alone, [t])[t]
        alone.close()
        assert info_alone == info_mix
        assert torch.equal(x_alone, x_mix), i
        plan = wmg.Plan(p["n"], p["m"], p["D"], levels=p["levels"], nu1=1, nu2=1, hybrid_depth=1,
                        cycle=wmg.CYCLE_HYBRID, precision=prec, angles=p.get("angles"))
        x_plan, info_plan, _, _ = plan.solve(data[i][1], wmg.SOLVER_GMRES, pre, MAX_ITER, RTOL, RESTART)
        torch.cuda.synchronize()
        plan.close()
        assert info_plan[0][0] == info_mix[0]
        assert torch.equal(x_plan, x_mix), i


def test_f64_matches_oracle():
    reqs = REQUESTS[:2] + REQUESTS[4:5]
    data = sinograms(reqs, torch.float64)
    srv = make_server(wmg.PREC_F64, rtol=0.0, max_iter=12)
    tickets = [srv.submit(p, b) for p, (_, b) in zip(reqs, data)]
    done = run_to_end(srv, list(tickets))
    srv.close()
    for t, p, (op, _) in zip(tickets, reqs, data):
        x, info, _ = done[t]
        b = data[reqs.index(p)][1].cpu().numpy()
        M = oracle.Wmg(op, p["levels"], 1, 1, 1.0, 0.0, oracle.CYCLE_HYBRID, 1)
        x_ref, k, _ = oracle.gmres(op, b, 12, RESTART, 0.0, 0.0, M)
        assert info[0] == k == 12
        x = x.cpu().numpy()
        assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) < 1e-10


def test_admission_by_footprint_and_rejection():
    # state pools for exactly two 32 x 32 requests (152 bytes per pixel and
    # 24 per ray for F64, restart 5, hybrid depth 1; 4 rays per pixel)
    state = 2048 * (152 + 4 * 24)
    reqs = [REQUESTS[0], REQUESTS[2], REQUESTS[0], REQUESTS[4]]
    data = sinograms(reqs, torch.float64)
    srv = make_server(wmg.PREC_F64, budget=state + (8 << 20), state=state, slots=8)
    st = srv.stats()
    assert st["state_bytes_capacity"] <= state
    tickets = [srv.submit(p, b) for p, (_, b) in zip(reqs, data)]
    big = sinograms([REQUESTS[5]], torch.float64)[0][1]
    with pytest.raises(wmg.WmgError) as e:
        srv.submit(REQUESTS[5], big)                   # 64 x 64 can never fit
    assert e.value.code == -8
    peak = 0
    left = list(tickets)
    results = {}
    for _ in range(1000):
        pending = srv.step()
        st = srv.stats()
        peak = max(peak, st["running"])
        assert st["state_bytes_used"] <= st["state_bytes_capacity"]
        for t in list(left):
            r = srv.poll(t)
            if r is not None:
                results[t] = r
                left.remove(t)
        if pending == 0:
            break
    assert not left and peak == 2
    st = srv.stats()
    assert st["rejected"] == 1 and st["completed"] == 4
    srv.close()
    # the same answers as without memory pressure
    ref = make_server(wmg.PREC_F64)
    rt = [ref.submit(p, b) for p, (_, b) in zip(reqs, data)]
    rres = run_to_end(ref, list(rt))
    ref.close()
    for t, u in zip(tickets, rt):
        assert torch.equal(results[t][0], rres[u][0])


def test_geometry_eviction():
    # a geometry budget that fits any one geometry's setup but not the three
    # geometries of the stream cached together with a setup: a setup has to
    # evict an unused cached geometry; results must not change
    reqs = [REQUESTS[0], REQUESTS[3], REQUESTS[4], REQUESTS[0], REQUESTS[3]]
    data = sinograms(reqs, torch.float64)
    probe = make_server(wmg.PREC_F64)
    fps = [probe.footprint(p)[1:] for p in (REQUESTS[0], REQUESTS[3], REQUESTS[4])]
    probe.close()
    gbud = max(g + t for g, t in fps) + 4096
    assert gbud < sum(g for g, _ in fps) + min(t for _, t in fps)
    state = 64 << 20
    srv = make_server(wmg.PREC_F64, budget=state + gbud, state=state, slots=4)
    tickets = [srv.submit(p, b) for p, (_, b) in zip(reqs, data)]
    done = {}
    left = list(tickets)
    for _ in range(100000):
        pending = srv.step()
        st = srv.stats()
        assert st["geometry_bytes_used"] <= gbud
        for t in list(left):
            r = srv.poll(t)
            if r is not None:
                done[t] = r
                left.remove(t)
        if pending == 0 and not left:
            break
    st = srv.stats()
    srv.close()
    assert not left
    assert st["geometries_evicted"] >= 1 and st["geometry_setups"] >= 3
    ref = make_server(wmg.PREC_F64)
    for t, p, (_, b) in zip(tickets, reqs, data):
        u = ref.submit(p, b)
        assert torch.equal(run_to_end(ref, [u])[u][0], done[t][0])
    ref.close()
