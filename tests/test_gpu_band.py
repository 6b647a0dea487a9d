"""The band path (f3): H_F reduced from its band to real tridiagonal form by Householder bulge
chasing (O(n^2 b) instead of the dense reduction's O(n^3)), then Z = Q Y from the chase's
reflectors.  Every window class (band widths up to 8, 16, 32, 64) in both precisions, compared
element by element with the oracle, with the dense path of the same systems, and in one mixed
batch with each system alone."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MMF_FP64: (1e-12, 1e-10), M.MMF_MIXED: (1e-9, 1e-8)}


def _chain(N=100, h0=0.37, v=0.21, omega=0.93):
    return W.Problem(D=1, H0=np.array([[h0]], dtype=complex), omegas=[omega], Ns=[N],
                     couplings=[[np.array([[v]], dtype=complex)]])


# (problem, expected half-bandwidth)
CASES = {
    "chain_b1": (lambda: _chain(), 1),
    "random_D4_b7": (lambda: W.random_small(5, D=4, Ns=[20], nharm=[1]), 7),
    "random_D5_h2_b14": (lambda: W.random_small(9, D=5, Ns=[30], nharm=[2]), 14),
    "random_D2_two_mode_b19": (lambda: W.random_small(7, D=2, Ns=[4, 8], nharm=[1, 1]), 19),
    "spin1_b33": (lambda: W.spin1_bichromatic(0.2, 0.4, N1=5, N2=6), 33),
    "spin1_b63": (lambda: W.spin1_bichromatic(0.3, 0.2, N1=10, N2=4), 63),
}

_ORACLE = {}


def _oracle(name, p, t):
    if name not in _ORACLE:
        _ORACLE[name] = O.solve(p, t=t, t0=0.0)
    return _ORACLE[name]


def _band_ctx():
    ctx = M.Context(0)
    ctx.set_option(M.MMF_OPT_BAND_MAX, 64)  # the band path in both precisions
    return ctx


def _solve(ctx, ps, precision, nt):
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
    b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in ps]))
    b.run()
    st = b.sync()
    E, U, P = b.results()
    return b, st, [b.unpack(E, U, P, i) for i in range(len(ps))]


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
@pytest.mark.parametrize("name", sorted(CASES))
def test_band_path_matches_oracle_and_dense_path(name, precision):
    p, band = CASES[name][0](), CASES[name][1]
    nt = 8
    t = W.time_grid(p, nt)
    ref = _oracle(name, p, t)
    e_rel, up = TOL[precision]
    ctx = _band_ctx()
    b, st, res = _solve(ctx, [p], precision, nt)
    assert b.path(0) == (M.MMF_PATH_BAND, band)
    assert st[0] == 0
    e, u, pp = res[0]
    nrm = np.abs(ref["E"]).max()
    assert np.abs(e - ref["E"]).max() <= e_rel * nrm
    assert np.abs(u - ref["U"]).max() <= up
    assert np.abs(pp - ref["P"]).max() <= up
    # the dense path of the same system
    ctx.set_option(M.MMF_OPT_BAND_MAX, 0)
    b2, st2, res2 = _solve(ctx, [p], precision, nt)
    assert b2.path(0)[0] in (M.MMF_PATH_DENSE, M.MMF_PATH_WHOLE_GPU) and st2[0] == 0
    e2, u2, p2 = res2[0]
    assert np.abs(e - e2).max() <= 2 * e_rel * nrm
    assert np.abs(u - u2).max() <= 2 * up and np.abs(pp - p2).max() <= 2 * up


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_band_classes_in_one_batch_equal_alone(precision):
    names = sorted(CASES)
    ps = [CASES[k][0]() for k in names]
    nt = 8
    ctx = _band_ctx()
    b, st, res = _solve(ctx, ps, precision, nt)
    assert (st == 0).all()
    e_rel, up = TOL[precision]
    for i, (k, p) in enumerate(zip(names, ps)):
        assert b.path(i) == (M.MMF_PATH_BAND, CASES[k][1])
        _, _, (one,) = _solve(ctx, [p], precision, nt)
        e, u, pp = res[i]
        assert np.abs(e - one[0]).max() <= e_rel * np.abs(one[0]).max()
        assert np.abs(u - one[1]).max() <= up and np.abs(pp - one[2]).max() <= up


def test_band_limit_option():
    p = W.spin1_bichromatic(0.2, 0.4, N1=5, N2=6)  # b = 33
    ctx = M.Context(0)
    # defaults: band path on the FP64 path, dense reduction on the mixed path
    assert M.Batch(ctx, [M.System(ctx, p)], M.MMF_FP64, 2).path(0) == (M.MMF_PATH_BAND, 33)
    assert M.Batch(ctx, [M.System(ctx, p)], M.MMF_MIXED, 2).path(0) == (M.MMF_PATH_DENSE, 0)
    ctx.set_option(M.MMF_OPT_BAND_MAX, 32)
    assert M.Batch(ctx, [M.System(ctx, p)], M.MMF_FP64, 2).path(0) == (M.MMF_PATH_DENSE, 0)
    ctx.set_option(M.MMF_OPT_BAND_MAX, 64)
    assert M.Batch(ctx, [M.System(ctx, p)], M.MMF_MIXED, 2).path(0) == (M.MMF_PATH_BAND, 33)


# the mixed band path's back-transform for half-bandwidths 33..64: on the tensor cores (blocks of
# 64 sweeps in compact WY form, split-TF32 products) from n = MMF_OPT_BT_TC_N on, FP32 units below
SIMT_ONLY = 1 << 40
TC_CASES = {
    "random_D4_h9_b39_n100": (lambda: W.random_small(5, D=4, Ns=[12], nharm=[9]), 39),
    "random_D3_h12_b38_n183": (lambda: W.random_small(11, D=3, Ns=[30], nharm=[12]), 38),
    "spin1_b33": CASES["spin1_b33"],
    "spin1_b63": CASES["spin1_b63"],
}


@pytest.mark.parametrize("bt_tc_n", [0, SIMT_ONLY])
@pytest.mark.parametrize("name", sorted(TC_CASES))
def test_band_backtransform_units_match_oracle(name, bt_tc_n):
    """Both units forced: one 128-column slab with partial blocks (n = 100), a ragged second slab
    (n = 183), several slabs and up to 13 passes (n = 429, 567); against the oracle."""
    p, band = TC_CASES[name][0](), TC_CASES[name][1]
    nt = 8
    t = W.time_grid(p, nt)
    ref = _oracle(name, p, t)
    ctx = _band_ctx()
    ctx.set_option(M.MMF_OPT_BT_TC_N, bt_tc_n)
    ctx.set_option(M.MMF_OPT_JACOBI_N_MIXED, 4)  # n = 100 would take the shared-memory Jacobi kernel
    b, st, res = _solve(ctx, [p], M.MMF_MIXED, nt)
    assert b.path(0) == (M.MMF_PATH_BAND, band)
    assert st[0] == 0
    e, u, pp = res[0]
    e_rel, up = TOL[M.MMF_MIXED]
    assert np.abs(e - ref["E"]).max() <= e_rel * np.abs(ref["E"]).max()
    assert np.abs(u - ref["U"]).max() <= up
    assert np.abs(pp - ref["P"]).max() <= up
    Z = b.eigenvectors(0)
    HF = O.build_hf(p)
    assert np.abs(HF @ Z - Z * e[None, :]).max() <= e_rel * np.abs(e).max()
