"""GPU path vs the FP64 CPU oracle, element by element, on seeded inputs (C ABI via ctypes).

Tolerances (FP64 path): assembly bit-exact; quasienergies within 1e-12 ||H_F||_2; U and Pbar
within 1e-10 absolute (eigenvector error of a backward-stable FP64 solver is ~eps ||H|| / gap;
U and Pbar are insensitive to rotations inside near-degenerate pairs).
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

E_REL = 1e-12
UP_ABS = 1e-10


@pytest.fixture(scope="module")
def ctx():
    return M.Context(0)


def _appendix_a_problem():
    rng = W.SplitMix64(77)
    D = 2

    def g():
        return np.array([[rng.complex_gaussian(0.4) for _ in range(D)] for _ in range(D)])

    H0 = W.hermitian_gaussian(rng, D, 1.0)
    return W.Problem(D=D, H0=H0, omegas=[0.731, 1.187], Ns=[3, 3], couplings=[[g(), g()], [g()]])


ASSEMBLY_CASES = {
    "appendixA": _appendix_a_problem,
    "qubit_c0": lambda: W.two_level(0.83, N=20),
    "spin1_small": lambda: W.spin1_bichromatic(0.3, 0.2, N1=3, N2=2),
    "random_3mode": lambda: W.random_small(5, D=3, Ns=[2, 1, 2], nharm=[2, 1, 3]),
    "uneven_c2_like": lambda: W.uneven_batch(count=3, seed=0)[2],
    "single_level": lambda: W.Problem(D=1, H0=np.array([[0.7]], dtype=complex), omegas=[1.3],
                                      Ns=[0], couplings=[[np.array([[0.2 + 0.1j]])]]),
}


@pytest.mark.parametrize("case", sorted(ASSEMBLY_CASES))
def test_assembly_bit_exact_fp64(ctx, case):
    p = ASSEMBLY_CASES[case]()
    s = M.System(ctx, p)
    assert s.build(M.MMF_FP64) == p.n
    HF = s.hamiltonian()
    ref = O.build_hf(p)
    assert np.array_equal(HF.real, ref.real) and np.array_equal(HF.imag, ref.imag)


@pytest.mark.parametrize("case", ["appendixA", "random_3mode", "spin1_small"])
def test_assembly_fp32_is_round_to_nearest(ctx, case):
    p = ASSEMBLY_CASES[case]()
    s = M.System(ctx, p)
    s.build(M.MMF_MIXED)
    HF = s.hamiltonian()
    ref = O.build_hf(p)
    assert np.array_equal(HF.real, ref.real.astype(np.float32).astype(np.float64))
    assert np.array_equal(HF.imag, ref.imag.astype(np.float32).astype(np.float64))


def _compare(p, E, U, P, t, t0, ref=None, e_rel=E_REL, up_abs=UP_ABS):
    if ref is None:
        ref = O.solve(p, t=t, t0=t0)
    nrm = max(abs(ref["E"][0]), abs(ref["E"][-1]))
    dE = np.abs(E - ref["E"]).max()
    assert dE <= e_rel * nrm, f"quasienergies off by {dE:.3e} (|H|={nrm:.3g})"
    if U is not None:
        dU = np.abs(U - ref["U"]).max()
        assert dU <= up_abs, f"U off by {dU:.3e}"
    dP = np.abs(P - ref["P"]).max()
    assert dP <= up_abs, f"Pbar off by {dP:.3e}"
    return ref


def _solve_gpu(ctx, p, t, t0, precision=M.MMF_FP64):
    s = M.System(ctx, p)
    s.build(precision)
    st = s.diagonalise()
    assert st == 0
    E = s.quasienergies()
    U = s.time_evolution(t, t0)
    P = s.transition_avg()
    return s, E, U, P


SOLVE_CASES = {
    # small n: shared-memory Jacobi
    "qubit_n82": lambda: W.two_level(1.37, N=20),
    "qubit_resonant_n82": lambda: W.two_level(1.0, N=20),
    "spin1_n27": lambda: W.spin1_bichromatic(0.4, 0.3, N1=1, N2=1),
    "random_n60": lambda: W.random_small(3, D=2, Ns=[7, 1], nharm=[2, 1]),
    # Householder path (several 32-column panels, ragged tails)
    "qubit_n242": lambda: W.two_level(0.61, N=60),
    "single_level_n101": lambda: W.Problem(D=1, H0=np.array([[0.3]], dtype=complex), omegas=[0.9],
                                           Ns=[50], couplings=[[np.array([[0.25 - 0.1j]])]]),
    "random_n125": lambda: W.random_small(8, D=5, Ns=[12], nharm=[2]),
    "random_n245": lambda: W.random_small(12, D=7, Ns=[3, 2], nharm=[1, 2]),
    "spin1_n297": lambda: W.spin1_bichromatic(0.35, 0.2, N1=5, N2=4),
    "c2_like_n": lambda: next(q for q in W.uneven_batch(count=40, seed=0) if 150 < q.n < 400),
}


@pytest.mark.parametrize("case", sorted(SOLVE_CASES))
def test_fp64_path_matches_oracle(ctx, case):
    p = SOLVE_CASES[case]()
    t = W.time_grid(p, 16)
    t0 = 0.3
    s, E, U, P = _solve_gpu(ctx, p, t, t0)
    _compare(p, E, U, P, t, t0)


@pytest.mark.parametrize("case", ["random_n125", "spin1_n297", "qubit_n82"])
def test_eigenpairs_residual_and_orthogonality(ctx, case):
    p = SOLVE_CASES[case]()
    s = M.System(ctx, p)
    s.build(M.MMF_FP64)
    assert s.diagonalise() == 0
    E, Z = s.quasienergies(), s.eigenvectors()
    HF = O.build_hf(p)
    nrm = np.abs(E).max()
    assert np.all(np.diff(E) >= 0)
    assert np.abs(HF @ Z - Z * E[None, :]).max() <= 1e-12 * nrm
    assert np.abs(Z.conj().T @ Z - np.eye(p.n)).max() <= 1e-12


def test_identity_at_t0_and_sum_rule_gpu(ctx):
    p = SOLVE_CASES["random_n245"]()
    t0 = 0.55
    s, E, U, P = _solve_gpu(ctx, p, np.array([t0, t0 + 1.0]), t0)
    np.testing.assert_allclose(U[0], np.eye(p.D), atol=1e-12)
    np.testing.assert_allclose(P.sum(axis=1), 1.0, atol=1e-12)


def test_zero_coupling_degenerate(ctx):
    """V = 0 with a degenerate H0: exact clusters in both the Jacobi and Householder paths."""
    for N in (5, 30):
        D = 2
        p = W.Problem(D=D, H0=np.diag([0.3, 0.3]).astype(complex), omegas=[1.1], Ns=[N],
                      couplings=[[np.zeros((D, D))]])
        t = np.array([0.0, 0.7, 2.0])
        s, E, U, P = _solve_gpu(ctx, p, t, 0.0)
        ev = np.sort([0.3 - k * 1.1 for k in range(-N, N + 1) for _ in range(D)])
        np.testing.assert_allclose(E, ev, atol=1e-13)
        for k, tk in enumerate(t):
            np.testing.assert_allclose(U[k], np.exp(-0.3j * tk) * np.eye(D), atol=1e-12)
        np.testing.assert_allclose(P, np.eye(D), atol=1e-12)


def test_single_state(ctx):
    """n = 1: H_F = H0 (one level, no Fourier copies)."""
    p = W.Problem(D=1, H0=np.array([[0.7]], dtype=complex), omegas=[1.0], Ns=[0],
                  couplings=[[np.array([[0.5]])]])
    s, E, U, P = _solve_gpu(ctx, p, np.array([0.0, 2.0]), 0.0)
    assert E.tolist() == [0.7]
    np.testing.assert_allclose(U[:, 0, 0], np.exp(-0.7j * np.array([0.0, 2.0])), atol=1e-15)
    assert P[0, 0] == pytest.approx(1.0, abs=1e-15)


def test_batch_alone_vs_mixed(ctx):
    """Uneven batch (Jacobi and Householder sizes together): every system's result in the mix
    equals its result alone and the oracle's."""
    ps = [SOLVE_CASES[k]() for k in ("qubit_n82", "random_n245", "spin1_n27", "qubit_n242",
                                     "random_n125", "random_n60")]
    nt = 8
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    systems = [M.System(ctx, p) for p in ps]
    b = M.Batch(ctx, systems, M.MMF_FP64, nt)
    b.set_times(0.0, ts)
    nk = b.run()
    assert nk >= 5
    st = b.sync()
    assert (st == 0).all()
    E, U, P = b.results()
    for i, p in enumerate(ps):
        e, u, pp = b.unpack(E, U, P, i)
        solo = M.Batch(ctx, [M.System(ctx, p)], M.MMF_FP64, nt)
        solo.set_times(0.0, ts[i:i + 1])
        solo.run()
        solo.sync()
        e1, u1, p1 = solo.get(0)
        nrm = np.abs(e1).max()
        assert np.abs(e - e1).max() <= 1e-13 * nrm
        assert np.abs(u - u1).max() <= 1e-12 and np.abs(pp - p1).max() <= 1e-12
        _compare(p, e, u, pp, ts[i], 0.0)


def test_rerun_is_reproducible(ctx):
    ps = [SOLVE_CASES["random_n125"](), SOLVE_CASES["qubit_n82"]()]
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_FP64, 4)
    b.set_times(0.0, np.stack([W.time_grid(p, 4) for p in ps]))
    b.run()
    b.sync()
    r1 = [x.copy() for x in b.results()]
    b.upload()
    b.run()
    b.sync()
    r2 = b.results()
    for a, c in zip(r1, r2):
        assert np.abs(a - c).max() <= 1e-13


def test_budget_admission(ctx):
    small = M.Context(0, budget=1 << 20)
    p = SOLVE_CASES["spin1_n297"]()
    with pytest.raises(M.MmfError) as ei:
        M.Batch(small, [M.System(small, p)], M.MMF_FP64, 4)
    assert ei.value.code == M.MMF_ERR_BUDGET
    assert small.bytes_in_use() == 0
    before = ctx.bytes_in_use()
    b = M.Batch(ctx, [M.System(ctx, p)], M.MMF_FP64, 4)
    bb = b.bytes()
    assert bb > 0 and ctx.bytes_in_use() == before + bb
    b.close()
    assert ctx.bytes_in_use() == before


def test_argument_and_state_errors(ctx):
    bad = np.array([[0, 1], [2, 0]], dtype=complex)  # not Hermitian
    with pytest.raises(M.MmfError) as ei:
        M.System(ctx, W.Problem(D=2, H0=bad, omegas=[1.0], Ns=[1], couplings=[[np.eye(2)]]))
    assert ei.value.code == M.MMF_ERR_ARG
    s = M.System(ctx, W.two_level(1.0, N=3))
    with pytest.raises(M.MmfError) as ei:
        s.quasienergies()
    assert ei.value.code == M.MMF_ERR_STATE
    huge = W.random_small(1, D=64, Ns=[30, 30, 30])  # n = 14.5 million: beyond any HBM budget
    with pytest.raises(M.MmfError) as ei:
        M.Batch(ctx, [M.System(ctx, huge)], M.MMF_FP64, 1)
    assert ei.value.code == M.MMF_ERR_BUDGET


def test_micromotion_matches_oracle(ctx):
    p = SOLVE_CASES["random_n125"]()
    s = M.System(ctx, p)
    s.build(M.MMF_FP64)
    s.diagonalise()
    t = np.array([0.0, 0.4, 1.9])
    UF, reps = s.micromotion(t)
    r = O.solve(p)
    reps_o = O.zone_representatives(p, r["E"], r["Z"])
    assert reps.tolist() == reps_o.tolist()
    UF_o = O.micromotion(p, r["Z"], reps_o, t)
    # eigenvector phases are arbitrary: align each column's phase on its largest entry
    for a in range(p.D):
        k, j = np.unravel_index(np.argmax(np.abs(UF_o[:, :, a])), UF_o[:, :, a].shape)
        ph = UF[k, j, a] / UF_o[k, j, a]
        assert abs(abs(ph) - 1.0) < 1e-10
        np.testing.assert_allclose(UF[:, :, a], ph * UF_o[:, :, a], atol=1e-10)


# ---------------------------------------------------------------------- mixed precision path
# FP32 reduction + FP64 tridiagonal solve + Ogita-Aishima refinement; bound: quasienergies within
# 1e-9 ||H_F||_2, U and Pbar within 1e-8 absolute of the FP64 oracle.
MIX_E_REL = 1e-9
MIX_UP_ABS = 1e-8


@pytest.mark.parametrize("case", sorted(SOLVE_CASES))
def test_mixed_path_matches_oracle(ctx, case):
    p = SOLVE_CASES[case]()
    t = W.time_grid(p, 16)
    t0 = 0.3
    s, E, U, P = _solve_gpu(ctx, p, t, t0, precision=M.MMF_MIXED)
    _compare(p, E, U, P, t, t0, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)


def test_mixed_zero_coupling_degenerate(ctx):
    for N in (5, 30):
        D = 2
        p = W.Problem(D=D, H0=np.diag([0.3, 0.3]).astype(complex), omegas=[1.1], Ns=[N],
                      couplings=[[np.zeros((D, D))]])
        t = np.array([0.0, 0.7, 2.0])
        s, E, U, P = _solve_gpu(ctx, p, t, 0.0, precision=M.MMF_MIXED)
        ev = np.sort([0.3 - k * 1.1 for k in range(-N, N + 1) for _ in range(D)])
        np.testing.assert_allclose(E, ev, atol=1e-9 * np.abs(ev).max())
        for k, tk in enumerate(t):
            np.testing.assert_allclose(U[k], np.exp(-0.3j * tk) * np.eye(D), atol=1e-8)
        np.testing.assert_allclose(P, np.eye(D), atol=1e-8)


def test_mixed_eigenpairs_residual(ctx):
    p = SOLVE_CASES["spin1_n297"]()
    s = M.System(ctx, p)
    s.build(M.MMF_MIXED)
    assert s.diagonalise() == 0
    E, Z = s.quasienergies(), s.eigenvectors()
    HF = O.build_hf(p)
    nrm = np.abs(E).max()
    assert np.all(np.diff(E) >= 0)
    assert np.abs(HF @ Z - Z * E[None, :]).max() <= 1e-10 * nrm
    assert np.abs(Z.conj().T @ Z - np.eye(p.n)).max() <= 1e-10


def test_mixed_batch_alone_vs_mixed(ctx):
    ps = [SOLVE_CASES[k]() for k in ("qubit_n82", "random_n245", "spin1_n27", "qubit_n242")]
    nt = 8
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, ts)
    b.run()
    assert (b.sync() == 0).all()
    E, U, P = b.results()
    for i, p in enumerate(ps):
        e, u, pp = b.unpack(E, U, P, i)
        solo = M.Batch(ctx, [M.System(ctx, p)], M.MMF_MIXED, nt)
        solo.set_times(0.0, ts[i:i + 1])
        solo.run()
        solo.sync()
        e1, u1, p1 = solo.get(0)
        nrm = np.abs(e1).max()
        assert np.abs(e - e1).max() <= 1e-9 * nrm
        assert np.abs(u - u1).max() <= 1e-8 and np.abs(pp - p1).max() <= 1e-8
        _compare(p, e, u, pp, ts[i], 0.0, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)


def test_graph_replay_matches_plain_launches(ctx):
    """The batch's launch sequence captured in a CUDA graph and replayed gives the plain run's
    results (two replays in a row, then after new inputs)."""
    ps = [SOLVE_CASES[k]() for k in ("qubit_n82", "random_n125", "spin1_n27")]
    nt = 8
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    for precision in (M.MMF_FP64, M.MMF_MIXED):
        plain = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
        plain.set_times(0.0, ts)
        plain.run()
        plain.sync()
        ref = [x.copy() for x in plain.results()]
        g = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
        g.set_times(0.0, ts)
        g.graph(True)
        # runs differ only in the order of floating-point atomics: compare at the path's tolerance
        tol = 1e-10 if precision == M.MMF_FP64 else 1e-8
        for _ in range(2):
            assert g.run() > 0
            assert (g.sync() == 0).all()
            out = g.results()
            for a, c in zip(ref, out):
                assert np.abs(a - c).max() <= tol * max(1.0, np.abs(a).max())
        g.set_times(0.4, ts)  # new t0: re-captured
        g.run()
        g.sync()
        plain.set_times(0.4, ts)
        plain.run()
        plain.sync()
        for a, c in zip(plain.results(), g.results()):
            assert np.abs(a - c).max() <= tol * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_many_systems_single_cta_reduction(ctx, precision):
    """More systems than fit two CTAs each on the GPU: the reduction runs one CTA per system.
    Every result must match the same system solved alone (two CTAs per system) and, for a sample,
    the oracle."""
    ps = [q for q in W.uneven_batch(count=400, seed=5) if 120 < q.n <= 260][:90]
    assert len(ps) == 90
    nt = 4
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], precision, nt)
    b.set_times(0.0, ts)
    b.run()
    assert (b.sync() == 0).all()
    E, U, P = b.results()
    e_rel, up = (1e-12, 1e-10) if precision == M.MMF_FP64 else (1e-9, 1e-8)
    for i in (0, 17, 45, 89):
        e, u, pp = b.unpack(E, U, P, i)
        E1, U1, P1 = M.Batch(ctx, [M.System(ctx, ps[i])], precision, nt), None, None
        E1.set_times(0.0, ts[i:i + 1])
        E1.run()
        E1.sync()
        e1, u1, p1 = E1.get(0)
        nrm = np.abs(e1).max()
        assert np.abs(e - e1).max() <= e_rel * nrm
        assert np.abs(u - u1).max() <= up and np.abs(pp - p1).max() <= up
        if i in (0, 45):
            _compare(ps[i], e, u, pp, ts[i], 0.0, e_rel=e_rel, up_abs=up)


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
@pytest.mark.parametrize("case", ["random_n245", "spin1_n297", "single_level_n101"])
def test_whole_gpu_reduction_path(case, precision):
    """The whole-GPU Householder reduction (used alone for systems too large for one CTA) forced
    on small systems, against the oracle."""
    c = M.Context(0)
    c.set_option(M.MMF_OPT_LARGE_N, 90)
    p = SOLVE_CASES[case]()
    t = W.time_grid(p, 8)
    s, E, U, P = _solve_gpu(c, p, t, 0.2, precision=precision)
    e_rel, up = (E_REL, UP_ABS) if precision == M.MMF_FP64 else (MIX_E_REL, MIX_UP_ABS)
    _compare(p, E, U, P, t, 0.2, e_rel=e_rel, up_abs=up)


@pytest.mark.parametrize("case", ["random_n60", "qubit_n242", "random_n245", "spin1_n297"])
def test_mixed_second_full_refinement_step(case):
    """The mixed path's second full refinement step (used alone for large n, where G of the FP64
    iterate is G(fl32 X) + C' + C'^H) forced on small systems, against the oracle; and a batch of
    both kinds of second step against each system solved alone."""
    c = M.Context(0)
    c.set_option(M.MMF_OPT_REFINE_FULL_N, 0)
    p = SOLVE_CASES[case]()
    t = W.time_grid(p, 8)
    s, E, U, P = _solve_gpu(c, p, t, 0.2, precision=M.MMF_MIXED)
    _compare(p, E, U, P, t, 0.2, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)


def test_mixed_batch_both_second_steps():
    c = M.Context(0)
    c.set_option(M.MMF_OPT_REFINE_FULL_N, 200)   # n >= 200: full second step, below: banded
    ps = [SOLVE_CASES[k]() for k in ("qubit_n82", "random_n245", "random_n125", "spin1_n297")]
    nt = 8
    b = M.Batch(c, [M.System(c, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in ps]))
    b.run()
    assert (b.sync() == 0).all()
    for i, p in enumerate(ps):
        E, U, P = b.get(i)
        ref = O.solve(p, t=W.time_grid(p, nt), t0=0.0)
        assert np.abs(E - ref["E"]).max() <= MIX_E_REL * np.abs(ref["E"]).max()
        assert np.abs(U - ref["U"]).max() <= MIX_UP_ABS
        assert np.abs(P - ref["P"]).max() <= MIX_UP_ABS


# ---------------------------------------------------------------------- back-transform paths
# The mixed path's back-transform (Z = Q Y) runs on the tensor cores (super-blocks of 128
# reflectors, split-TF32 products) from n = MMF_OPT_BT_TC_N on, on the FP32 SIMT kernel below.
SIMT_ONLY = 1 << 40


@pytest.mark.parametrize("case", ["random_n125", "qubit_n242", "random_n245", "spin1_n297", "c2_like_n"])
@pytest.mark.parametrize("bt_tc_n", [0, SIMT_ONLY])
def test_mixed_backtransform_paths_match_oracle(case, bt_tc_n):
    """Both back-transform paths forced on systems with one to three super-blocks (ragged last
    ones), against the oracle."""
    c = M.Context(0)
    c.set_option(M.MMF_OPT_BT_TC_N, bt_tc_n)
    p = SOLVE_CASES[case]()
    t = W.time_grid(p, 8)
    s, E, U, P = _solve_gpu(c, p, t, 0.2, precision=M.MMF_MIXED)
    _compare(p, E, U, P, t, 0.2, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)


def test_mixed_backtransform_many_super_blocks():
    """n = 693 (six super-blocks, the last one ragged) on the tensor-core path, against the
    oracle, with eigenpair residuals and orthonormality of all eigenvectors within the mixed
    path's bound (residual <= 1e-9 ||H_F||, the quasienergy tolerance)."""
    c = M.Context(0)
    p = W.spin1_bichromatic(0.35, 0.2, N1=10, N2=5)
    assert p.n == 693
    t = W.time_grid(p, 8)
    s, E, U, P = _solve_gpu(c, p, t, 0.1, precision=M.MMF_MIXED)
    _compare(p, E, U, P, t, 0.1, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)
    Z = s.eigenvectors()
    HF = O.build_hf(p)
    nrm = np.abs(E).max()
    res = np.abs(HF @ Z - Z * E[None, :]).max() / nrm
    orth = np.abs(Z.conj().T @ Z - np.eye(p.n)).max()
    print(f"n = 693: residual {res:.3e} |H_F|, orthogonality {orth:.3e}")
    assert res <= MIX_E_REL
    assert orth <= MIX_E_REL


def test_mixed_batch_both_backtransform_paths():
    """A batch whose systems take different back-transform paths (and different numbers of
    super-blocks) against each system solved alone on the other path."""
    c = M.Context(0)
    c.set_option(M.MMF_OPT_BT_TC_N, 240)   # n >= 240: tensor cores, below: SIMT
    ps = [SOLVE_CASES[k]() for k in ("qubit_n82", "random_n125", "spin1_n297", "qubit_n242", "random_n245")]
    nt = 8
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(c, [M.System(c, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, ts)
    b.run()
    assert (b.sync() == 0).all()
    c2 = M.Context(0)
    c2.set_option(M.MMF_OPT_BT_TC_N, 100)  # every Householder system on the tensor cores
    for i, p in enumerate(ps):
        e, u, pp = b.get(i)
        solo = M.Batch(c2, [M.System(c2, p)], M.MMF_MIXED, nt)
        solo.set_times(0.0, ts[i:i + 1])
        solo.run()
        assert solo.sync()[0] == 0
        e1, u1, p1 = solo.get(0)
        assert np.abs(e - e1).max() <= 1e-9 * np.abs(e1).max()
        assert np.abs(u - u1).max() <= 1e-8 and np.abs(pp - p1).max() <= 1e-8


def test_mixed_many_levels_time_evolution():
    """More than 16 levels: the mixed path's U falls back from the tensor-core contraction to the
    double-FP32 one; against the oracle, alone and in a batch with a tensor-core system."""
    c = M.Context(0)
    big = W.random_small(4, D=17, Ns=[2], nharm=[1])
    small = SOLVE_CASES["random_n125"]()
    t = W.time_grid(big, 8)
    s, E, U, P = _solve_gpu(c, big, t, 0.2, precision=M.MMF_MIXED)
    _compare(big, E, U, P, t, 0.2, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)
    nt = 8
    ps = [small, big]
    ts = np.stack([W.time_grid(p, nt) for p in ps])
    b = M.Batch(c, [M.System(c, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, ts)
    b.run()
    assert (b.sync() == 0).all()
    for i, p in enumerate(ps):
        e, u, pp = b.get(i)
        _compare(p, e, u, pp, ts[i], 0.0, e_rel=MIX_E_REL, up_abs=MIX_UP_ABS)
