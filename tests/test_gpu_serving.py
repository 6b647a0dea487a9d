"""Continuous-batching server: requests of different sizes admitted as slots and HBM budget
free up, overlapping on the device; every result equals the same system solved alone (within
the path's tolerance) and the oracle's."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _mix():
    ps = [W.two_level(w, N=20) for w in (0.4, 1.1, 1.7)]
    ps += [W.spin1_bichromatic(0.3, 0.2, N1=5, N2=4), W.random_small(12, D=7, Ns=[3, 2], nharm=[1, 2])]
    ps += [q for q in W.uneven_batch(count=30, seed=0) if q.n <= 600][:5]
    return ps


def _alone(ctx, p, precision, nt):
    b = M.Batch(ctx, [M.System(ctx, p)], precision, nt)
    b.set_times(0.0, W.time_grid(p, nt)[None, :])
    b.run()
    b.sync()
    return b.get(0)


@pytest.mark.parametrize("precision", [M.MMF_MIXED, M.MMF_FP64])
def test_served_results_equal_alone(precision):
    ctx = M.Context(0)
    nt = 16
    ps = _mix()
    srv = M.Server(ctx, slots=3, max_batch=3, precision=precision)
    systems = [M.System(ctx, p) for p in ps]
    tickets = [srv.submit(s, W.time_grid(p, nt)) for s, p in zip(systems, ps)]
    results = [srv.wait(t, timeout_ms=120000) for t in tickets]
    e_rel, up = (1e-9, 1e-8) if precision == M.MMF_MIXED else (1e-12, 1e-10)
    for p, (E, U, P, st) in zip(ps, results):
        assert st == 0
        E1, U1, P1 = _alone(ctx, p, precision, nt)
        nrm = np.abs(E1).max()
        assert np.abs(E - E1).max() <= e_rel * nrm
        assert np.abs(U - U1).max() <= up and np.abs(P - P1).max() <= up
    # two of them against the oracle as well
    for i in (0, 3):
        ref = O.solve(ps[i], t=W.time_grid(ps[i], nt), t0=0.0)
        E, U, P, _ = results[i]
        assert np.abs(E - ref["E"]).max() <= e_rel * np.abs(ref["E"]).max()
        assert np.abs(U - ref["U"]).max() <= up and np.abs(P - ref["P"]).max() <= up
    st = srv.stats()
    assert st["completed"] == len(ps) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    assert ctx.bytes_in_use() == 0


def test_admission_waits_for_budget():
    """A budget that holds one plan at a time: requests queue and are admitted as memory frees."""
    p = W.spin1_bichromatic(0.3, 0.2, N1=5, N2=4)
    probe = M.Context(0)
    one = M.Batch(probe, [M.System(probe, p)], M.MMF_MIXED, 8).bytes()
    ctx = M.Context(0, budget=int(one * 1.5))
    srv = M.Server(ctx, slots=4, max_batch=4, precision=M.MMF_MIXED)
    s = M.System(ctx, p)
    tickets = [srv.submit(s, W.time_grid(p, 8)) for _ in range(6)]
    outs = [srv.wait(t, timeout_ms=120000) for t in tickets]
    for E, U, P, st in outs[1:]:
        assert st == 0
        assert np.abs(E - outs[0][0]).max() <= 1e-9 * np.abs(E).max()
    srv.close()
    assert ctx.bytes_in_use() == 0


@pytest.mark.parametrize("precision", [M.MMF_MIXED, M.MMF_FP64])
def test_resident_plan_reused_with_new_values(precision):
    """Requests of one structure but different frequencies and couplings, one after another: the
    second and third reuse the first plan (new coefficients and frequencies uploaded into it), and
    each result equals the same system solved alone."""
    ctx = M.Context(0)
    srv = M.Server(ctx, slots=1, max_batch=1, precision=precision)
    nt = 8
    ps = [W.spin1_bichromatic(a, b, N1=5, N2=4) for a, b in ((0.3, 0.2), (0.1, 0.45))]
    ps[1].omegas = [1.07, 0.55]
    ps.append(W.two_level(0.9, N=20))
    ps.append(W.two_level(1.3, N=20))
    e_rel, up = (1e-9, 1e-8) if precision == M.MMF_MIXED else (1e-12, 1e-10)
    for p in ps:
        E, U, P, st = srv.wait(srv.submit(M.System(ctx, p), W.time_grid(p, nt)), timeout_ms=120000)
        assert st == 0
        E1, U1, P1 = _alone(ctx, p, precision, nt)
        assert np.abs(E - E1).max() <= e_rel * np.abs(E1).max()
        assert np.abs(U - U1).max() <= up and np.abs(P - P1).max() <= up
    ps_ = srv.plan_stats()
    assert ps_["created"] == 2 and ps_["reused"] == 2, ps_
    srv.close()
    assert ctx.bytes_in_use() == 0


def test_unknown_ticket():
    ctx = M.Context(0)
    srv = M.Server(ctx, slots=1, max_batch=1, precision=M.MMF_FP64)
    with pytest.raises(M.MmfError) as ei:
        srv.poll(12345)
    assert ei.value.code == M.MMF_ERR_ARG
    srv.close()
