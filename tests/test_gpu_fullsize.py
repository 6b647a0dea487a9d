"""Full-size parity at the benchmark's workload and launch configuration: 64 spin-1 two-mode
systems with n = 1323 solved in one batch.  System 0 is compared element by element with the
stored oracle result (tests/golden/spin1_c1_sys0.npz, written by tests/golden/gen_golden.py);
every system is checked against invariants that hold at any size."""

import os

import numpy as np
import pytest

from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "spin1_c1_sys0.npz")
TOL = {M.MMF_FP64: (1e-12, 1e-10), M.MMF_MIXED: (1e-9, 1e-8)}


@pytest.fixture(scope="module")
def ctx():
    return M.Context(0)


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_spin1_batch_full_size(ctx, precision):
    ps = W.spin1_amplitude_set(64, seed=1)
    nt = 64
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
    b.set_times(0.0, ts)
    b.run()
    st = b.sync()
    assert (st == 0).all()
    E, U, P = b.results()
    g = np.load(GOLD)
    e, u, pp = b.unpack(E, U, P, 0)
    e_rel, up_abs = TOL[precision]
    nrm = np.abs(g["E"]).max()
    assert np.abs(e - g["E"]).max() <= e_rel * nrm
    assert np.abs(u - g["U"]).max() <= up_abs
    assert np.abs(pp - g["P"]).max() <= up_abs
    for i in range(len(ps)):
        e, u, pp = b.unpack(E, U, P, i)
        assert np.all(np.diff(e) >= 0)
        np.testing.assert_allclose(u[0], np.eye(3), atol=up_abs)          # U(t0, t0) = I
        np.testing.assert_allclose(pp.sum(axis=1), 1.0, atol=up_abs)      # sum_j Pbar = 1
        # Floquet copies: the central eigenvalue recurs shifted by omega_1
        mid = e[np.argmin(np.abs(e))]
        assert np.min(np.abs(e - (mid + 1.0))) <= 1e-6
