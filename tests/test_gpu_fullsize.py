"""Full-size parity at the benchmark's workloads and launch configurations, against stored oracle
results written by tests/golden/gen_golden.py (which calls only the oracle):
- 64 spin-1 two-mode systems with n = 1323 in one batch: systems 0..6 element by element
  (spin1_c1_sys0.npz, spin1_c1_sys1_6.npz); every system against invariants that hold at any size;
- the 4096-system uneven batch (n = 18 ... 1998) in one mixed-precision launch: 20 systems spread
  over the range of n element by element (uneven_c2_sample.npz), every system against the
  invariants; the same 20 systems on the FP64 path."""

import os

import numpy as np
import pytest

from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(__file__), "golden")
TOL = {M.MMF_FP64: (1e-12, 1e-10), M.MMF_MIXED: (1e-9, 1e-8)}


def _c1_gold():
    g = {}
    z = np.load(os.path.join(HERE, "spin1_c1_sys0.npz"))
    g[0] = (z["E"], z["U"], z["P"])
    z = np.load(os.path.join(HERE, "spin1_c1_sys1_6.npz"))
    for i in z["indices"]:
        g[int(i)] = (z[f"E_{i}"], z[f"U_{i}"], z[f"P_{i}"])
    return g


def _c2_gold():
    z = np.load(os.path.join(HERE, "uneven_c2_sample.npz"))
    return {int(i): (z[f"E_{i}"], z[f"U_{i}"], z[f"P_{i}"]) for i in z["indices"]}


def _compare(e, u, pp, gold, precision, what):
    ge, gu, gp = gold
    e_rel, up_abs = TOL[precision]
    nrm = np.abs(ge).max()
    assert np.abs(e - ge).max() <= e_rel * nrm, what
    assert np.abs(u - gu).max() <= up_abs, what
    assert np.abs(pp - gp).max() <= up_abs, what


def _invariants(e, u, pp, D, tol):
    assert np.all(np.diff(e) >= 0)
    np.testing.assert_allclose(u[0], np.eye(D), atol=tol)          # U(t0, t0) = I
    np.testing.assert_allclose(pp.sum(axis=1), 1.0, atol=tol)      # sum_j Pbar = 1
    assert np.all(pp >= -tol)


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
    gold = _c1_gold()
    assert sorted(gold) == list(range(7))
    for i, g in gold.items():
        _compare(*b.unpack(E, U, P, i), g, precision, f"system {i}")
    for i in range(len(ps)):
        e, u, pp = b.unpack(E, U, P, i)
        _invariants(e, u, pp, 3, TOL[precision][1])
        # Floquet copies: the central eigenvalue recurs shifted by omega_1
        mid = e[np.argmin(np.abs(e))]
        assert np.min(np.abs(e - (mid + 1.0))) <= 1e-6


def test_uneven_batch_full_size_mixed(ctx):
    """The 4096-system uneven batch in one mixed-precision launch (the timed configuration)."""
    ps = W.uneven_batch(4096, seed=0)
    nt = 64
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, ts)
    b.run()
    st = b.sync()
    assert (st == 0).all(), np.unique(st, return_counts=True)
    E, U, P = b.results()
    gold = _c2_gold()
    assert len(gold) == 20
    for i, g in gold.items():
        _compare(*b.unpack(E, U, P, i), g, M.MMF_MIXED, f"system {i} (n = {ps[i].n})")
    for i, p in enumerate(ps):
        e, u, pp = b.unpack(E, U, P, i)
        _invariants(e, u, pp, p.D, 1e-8)
    b.close()


def test_uneven_sample_fp64(ctx):
    """The same 20 sampled systems on the FP64 path, in one batch."""
    allp = W.uneven_batch(4096, seed=0)
    gold = _c2_gold()
    idx = sorted(gold)
    ps = [allp[i] for i in idx]
    nt = 64
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_FP64, nt)
    b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in ps]))
    b.run()
    assert (b.sync() == 0).all()
    E, U, P = b.results()
    for k, i in enumerate(idx):
        _compare(*b.unpack(E, U, P, k), gold[i], M.MMF_FP64, f"system {i} (n = {allp[i].n})")
