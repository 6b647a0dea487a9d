"""Failure paths provoked on the host or by parameters (no device fault): an iteration cap that
the Jacobi kernel reaches returns MMF_ST_NOCONV through mmf_batch_sync and mmf_diagonalise, and
a serving wait that runs out of time returns MMF_ERR_STATE while the request stays valid."""

import numpy as np
import pytest

from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_jacobi_sweep_cap_reports_noconv(precision):
    ctx = M.Context(0)
    ctx.set_option(M.MMF_OPT_JACOBI_SWEEPS, 1)
    # a Jacobi-size system (n = 82) that needs several sweeps, and a Householder-size one
    ps = [W.two_level(1.1, N=20), W.spin1_bichromatic(0.3, 0.2, N1=6, N2=5)]
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, 4)
    b.set_times(0.0, np.stack([W.time_grid(p, 4) for p in ps]))
    b.run()
    st = b.sync()
    assert st[0] == M.MMF_ST_NOCONV and st[1] == M.MMF_OK
    rc = M.lib().mmf_batch_sync(b.h, None)
    assert rc == M.MMF_ST_NOCONV and b"system 0" in M.lib().mmf_last_error()
    s = M.System(ctx, ps[0])
    s.build(precision)
    assert s.diagonalise() == M.MMF_ST_NOCONV
    # the default cap converges
    ctx.set_option(M.MMF_OPT_JACOBI_SWEEPS, -1)
    b2 = M.Batch(ctx, [M.System(ctx, ps[0])], precision, 4)
    b2.set_times(0.0, W.time_grid(ps[0], 4)[None, :])
    b2.run()
    assert (b2.sync() == 0).all()


def test_serving_wait_times_out_then_completes():
    ctx = M.Context(0)
    srv = M.Server(ctx, slots=1, max_batch=4, precision=M.MMF_MIXED)
    ps = W.spin1_amplitude_set(4, seed=1)  # n = 1323: far more than 1 ms of work
    systems = [M.System(ctx, p) for p in ps]
    tickets = [srv.submit(s, W.time_grid(p, 16)) for s, p in zip(systems, ps)]
    with pytest.raises(M.MmfError) as ei:
        srv.wait(tickets[-1], timeout_ms=1)
    assert ei.value.code == M.MMF_ERR_STATE
    srv.poll(tickets[-1])  # still known to the server after the time-out (no error)
    outs = [srv.wait(t, timeout_ms=-1) for t in tickets]
    assert all(o[3] == 0 for o in outs)
    with pytest.raises(M.MmfError):
        srv.poll(tickets[0])  # released by its wait
    srv.close()


def test_refinement_reports_a_cluster_too_large_to_separate():
    """Two modes of the same frequency and no coupling: H_F is diagonal with E - (n1 + n2) w, so
    the value E appears 2N + 1 = 41 times, a cluster beyond the refinement's 32-vector
    separation.  The mixed path says so with MMF_ST_CLUSTER (its quasienergies stay exact); the
    FP64 path, which has no refinement, reports nothing."""
    D, N, w = 1, 20, 0.7
    p = W.Problem(D=D, H0=np.array([[0.25]], dtype=complex), omegas=[w, w], Ns=[N, N],
                  couplings=[[np.zeros((1, 1), dtype=complex)], [np.zeros((1, 1), dtype=complex)]])
    ctx = M.Context(0)
    expect = np.sort(np.array([0.25 - (a + c) * w for a in range(-N, N + 1) for c in range(-N, N + 1)]))
    for precision, status in ((M.MMF_MIXED, M.MMF_ST_CLUSTER), (M.MMF_FP64, M.MMF_OK)):
        b = M.Batch(ctx, [M.System(ctx, p)], precision, 2)
        b.set_times(0.0, W.time_grid(p, 2)[None, :])
        b.run()
        st = b.sync()
        assert st[0] == status, (precision, st)
        E, _, P = b.get(0)
        assert np.abs(E - expect).max() <= 1e-9 * np.abs(expect).max()
        np.testing.assert_allclose(P, [[1.0]], atol=1e-8)  # one level: Pbar = 1
