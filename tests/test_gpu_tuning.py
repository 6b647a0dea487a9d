"""Tuning rules (mmf_ctx_add_rule / mmf_ctx_load_tuning): per-system solver choices by n and
half-bandwidth take effect, leave results within the path's tolerance of the oracle, and do not
depend on the rest of the batch."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MMF_FP64: (1e-12, 1e-10), M.MMF_MIXED: (1e-9, 1e-8)}


def _run(ctx, ps, precision, nt=8):
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
    b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in ps]))
    b.run()
    st = b.sync()
    E, U, P = b.results()
    return b, st, [b.unpack(E, U, P, i) for i in range(len(ps))]


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_rules_choose_paths_and_keep_results(precision):
    qubit = W.two_level(1.3, N=20)                      # n = 82: Jacobi by default
    spin = W.spin1_bichromatic(0.3, 0.2, N1=6, N2=5)    # n = 429, b = 3 x 13 = 39
    ctx = M.Context(0)
    bw = M.System(ctx, spin).bandwidth()
    assert bw == 39
    ctx.add_rule(precision, 1, 100, 0, 100, jacobi=0)
    ctx.add_rule(precision, 400, 500, bw, bw, band=1 if precision == M.MMF_MIXED else 0, bt_tc=0)
    b, st, res = _run(ctx, [qubit, spin], precision)
    assert (st == 0).all()
    assert b.path(0)[0] in (M.MMF_PATH_DENSE, M.MMF_PATH_BAND)
    assert b.path(1) == ((M.MMF_PATH_BAND, bw) if precision == M.MMF_MIXED else (M.MMF_PATH_DENSE, 0))
    e_rel, up = TOL[precision]
    for p, (e, u, pp) in zip([qubit, spin], res):
        ref = O.solve(p, t=W.time_grid(p, 8), t0=0.0)
        assert np.abs(e - ref["E"]).max() <= e_rel * np.abs(ref["E"]).max()
        assert np.abs(u - ref["U"]).max() <= up and np.abs(pp - ref["P"]).max() <= up
    # the same system alone takes the same path (rules see only n and the band)
    b1, _, _ = _run(ctx, [spin], precision)
    assert b1.path(0) == b.path(1)
    ctx.clear_rules()
    b2, _, _ = _run(ctx, [qubit], precision)
    assert b2.path(0)[0] == M.MMF_PATH_JACOBI


def test_mixed_back_transform_choice():
    p = W.spin1_bichromatic(0.2, 0.3, N1=8, N2=5)  # n = 561, dense reduction on the mixed path
    outs = []
    for tc in (0, 1):
        ctx = M.Context(0)
        ctx.add_rule(M.MMF_MIXED, 1, 10 ** 6, 0, 10 ** 6, jacobi=0, band=0, bt_tc=tc)
        b, st, res = _run(ctx, [p], M.MMF_MIXED)
        assert st[0] == 0 and b.path(0) == (M.MMF_PATH_DENSE, 0)
        outs.append(res[0])
    assert np.abs(outs[0][0] - outs[1][0]).max() <= 2e-9 * np.abs(outs[0][0]).max()
    assert np.abs(outs[0][1] - outs[1][1]).max() <= 2e-8


def test_load_tuning_file(tmp_path):
    f = tmp_path / "t.txt"
    f.write_text("# a table\nmixed 1 100 0 100 0 -1 -1   # comment\n\nfp64 200 300 0 64 -1 1 -1\n")
    ctx = M.Context(0)
    assert ctx.load_tuning(str(f)) == 2
    b, st, _ = _run(ctx, [W.two_level(0.8, N=20)], M.MMF_MIXED)
    assert b.path(0)[0] != M.MMF_PATH_JACOBI and st[0] == 0
    bad = tmp_path / "bad.txt"
    bad.write_text("mixed 1 100 0 100 0 -1\n")
    with pytest.raises(M.MmfError) as ei:
        ctx.load_tuning(str(bad))
    assert ":1:" in str(ei.value)
