"""Driven 1-D lattice (Sec. 4.2, Eq. 9) on the GPU.

D = 256 sites put Pbar on the many-level path: a D x n x D product plus per-cluster terms,
instead of one shared-memory table per system. They also put the eigensolver at
n = 256 (2N + 1).
- Small cases (D > 64, several panels, a ragged tail, exactly degenerate clusters) are compared
  element by element with the oracle.
- The full-size sweep (D = 256, N = 3, n = 1792, 64 frequencies in one batch, the launch
  configuration the benchmark times) is checked against LAPACK's eigenvalues of the oracle's
  H_F. Pbar and U are checked against the oracle evaluated on LAPACK's eigenpairs; both are
  invariant to the choice of eigenvectors inside a degenerate cluster. Residuals and
  orthogonality of the GPU's own eigenvectors are checked too.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MMF_FP64: (1e-12, 1e-10), M.MMF_MIXED: (1e-9, 1e-8)}


@pytest.fixture(scope="module")
def ctx():
    return M.Context(0)


def _twin_lattice(w=0.61):
    """Two identical, uncoupled 36-site lattices (D = 72): every quasienergy is exactly doubly
    degenerate, so Pbar needs its cluster terms."""
    q = W.driven_lattice(w, D=36, N=1, V=0.2)
    Z36 = np.zeros((36, 36), dtype=complex)
    H0 = np.block([[q.H0, Z36], [Z36, q.H0]])
    V = q.couplings[0][0]
    return W.Problem(D=72, H0=H0, omegas=[w], Ns=[1], couplings=[[np.block([[V, Z36], [Z36, V]])]])


SMALL = {
    "lattice_D96_N1_n288": lambda: W.driven_lattice(0.55, D=96, N=1, V=0.15),
    "lattice_D70_N0_n70": lambda: W.driven_lattice(0.8, D=70, N=0),
    "lattice_D66_N2_n330": lambda: W.driven_lattice(0.37, D=66, N=2, V=0.1, phi=0.7),
    "twin_lattice_D72_n216": _twin_lattice,
}


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
@pytest.mark.parametrize("case", sorted(SMALL))
def test_lattice_matches_oracle(ctx, case, precision):
    p = SMALL[case]()
    t, t0 = np.array([0.0, 1.7, 4.1]), 0.4
    ref = O.solve(p, t=t, t0=t0)
    s = M.System(ctx, p)
    s.build(precision)
    assert s.diagonalise() == 0
    E = s.quasienergies()
    U = s.time_evolution(t, t0)
    P = s.transition_avg()
    e_rel, up_abs = TOL[precision]
    nrm = max(abs(ref["E"][0]), abs(ref["E"][-1]))
    assert np.abs(E - ref["E"]).max() <= e_rel * nrm
    assert np.abs(U - ref["U"]).max() <= up_abs
    assert np.abs(P - ref["P"]).max() <= up_abs


def test_twin_lattice_has_degenerate_clusters():
    """The cluster case really exercises the cluster terms: consecutive quasienergies coincide
    to rounding (well inside the 1e-8 max|E| clustering threshold) in pairs."""
    E = O.solve(_twin_lattice())["E"]
    gaps = np.diff(E)
    assert (gaps[0::2] < 1e-12).all() and (gaps[1::2] > 1e-6).all()


def _lapack_check(p, E, Z, P, precision, U=None, t=None, t0=0.0):
    e_rel, up_abs = TOL[precision]
    HF = O.build_hf(p)
    El, Zl = np.linalg.eigh(HF)
    nrm = np.abs(El).max()
    assert np.abs(E - El).max() <= e_rel * nrm
    R = HF @ Z - Z * E[None, :]
    assert np.abs(R).max() <= e_rel * nrm
    G = Z.conj().T @ Z
    assert np.abs(G - np.eye(len(E))).max() <= up_abs
    Pref = O.transition_avg(p, El, Zl)
    assert np.abs(P - Pref).max() <= up_abs
    if U is not None:
        Uref = O.time_evolution(p, El, Zl, t, t0)
        assert np.abs(U - Uref).max() <= up_abs


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_lattice_full_size_single(ctx, precision):
    """One resonant sweep point at full size with U at two times (D = 256 U contraction)."""
    p = W.driven_lattice(0.6)
    assert p.n == 1792
    s = M.System(ctx, p)
    s.build(precision)
    assert s.diagonalise() == 0
    t, t0 = np.array([0.0, 2.3]), 0.0
    U = s.time_evolution(t, t0)
    E, Z = s.quasienergies(), s.eigenvectors()
    _lapack_check(p, E, Z, s.transition_avg(), precision, U, t, t0)
    np.testing.assert_allclose(U[0], np.eye(256), rtol=0, atol=TOL[precision][1])
    # near-degenerate pairs (tunnel splittings down to 1e-10) leave the mixed path's refinement as
    # clusters separated by Rayleigh-Ritz on their span: orthonormal to FP64 rounding among
    # themselves, so that their eigenvalues carry no |E| |Z_C^H Z_C - I| error
    close = np.nonzero(np.diff(E) < 1e-6)[0]
    assert close.size >= 8
    for k in close:
        G = Z[:, k:k + 2].conj().T @ Z[:, k:k + 2]
        assert np.abs(G - np.eye(2)).max() <= 1e-12, (k, np.abs(G - np.eye(2)).max())


def test_lattice_sweep_batch_full_size(ctx):
    """The benchmark's launch: 64 frequencies of the D = 256 lattice in one mixed batch."""
    ps = W.lattice_sweep()
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_MIXED, 0)
    b.set_times(0.0, np.zeros((len(ps), 0)))
    b.run()
    assert (b.sync() == 0).all()
    E, U, P = b.results()
    for i, p in enumerate(ps):
        e, _, pp = b.unpack(E, U, P, i)
        assert np.all(np.diff(e) >= 0)
        np.testing.assert_allclose(pp.sum(axis=1), 1.0, rtol=0, atol=1e-8)
        assert (pp >= -1e-12).all()
    for i in (0, 40):
        e, _, pp = b.unpack(E, U, P, i)
        _lapack_check(ps[i], e, b.eigenvectors(i), pp, M.MMF_MIXED)
