"""Dressed-basis evolution on the GPU (Sec. 3.3, Eq. 4): Ud = U_F(t2)^dagger U(t2, t1) U_F(t1)
with U_F the micromotion of the dressing modes alone, compared element by element with the
oracle's dressed_time_evolution, in both precisions, for one system and for a batch; plus the
two physical facts the oracle is pinned by (no probe: diagonal dressed evolution; Sec. 4.1's
probe resonance at the dressed splitting)."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {M.MMF_FP64: 1e-10, M.MMF_MIXED: 1e-8}


def _dressed_qubit(omega_p, amp_pz, N_d=6, N_p=5, amp_x=0.05):
    """Qubit of Eq. 8: w0 S_z, a resonant dressing drive amp_x cos(t) S_x (mode 1) and a probe
    amp_pz cos(omega_p t) S_z (mode 2)."""
    sx = 0.5 * np.array([[0, 1], [1, 0]], dtype=complex)
    sz = 0.5 * np.array([[1, 0], [0, -1]], dtype=complex)
    return W.Problem(D=2, H0=1.0 * sz, omegas=[1.0, omega_p], Ns=[N_d, N_p],
                     couplings=[[0.5 * amp_x * sx], [0.5 * amp_pz * sz]])


def _spin1_dressed(a1, a2):
    """Spin-1 (w0 = 1) with a detuned dressing drive along x at w1 = 1.37 (mode 1) and a weak
    second drive along z (mode 2).  Detuned, so that each Floquet state of the dressing drive has
    one dominant Fourier block and the zone representatives are unambiguous (under a resonant
    drive the central-block weights of a state and of its copies shifted by w1 tie)."""
    return W.spin1_bichromatic(a1, a2, N1=8, N2=4, omega1=1.37)


def _assert_same_up_to_basis_phases(Ug, Uo, tol):
    """Ug and Uo (nt x D x D) are the same dressed evolutions if Ug[k] = P^dagger Uo[k] P for one
    diagonal unitary P (the eigenvector phases of the zone representatives are arbitrary, Sec. 3.2
    leaves them open): the diagonals agree as they are; each off-diagonal entry (a, c) agrees after
    one phase e^{i theta_ac} common to all times, taken where |Uo[:, a, c]| is largest, and these
    phases compose as differences (theta_ac = phi_c - phi_a)."""
    nt, D, _ = Uo.shape
    theta = {}
    for a in range(D):
        assert np.abs(Ug[:, a, a] - Uo[:, a, a]).max() <= tol, ("diagonal", a)
        for c in range(D):
            if a == c:
                continue
            k = int(np.argmax(np.abs(Uo[:, a, c])))
            if abs(Uo[k, a, c]) < 1e-6:
                assert np.abs(Ug[:, a, c]).max() <= tol + 1e-6, ("small entry", a, c)
                continue
            r = Ug[k, a, c] / Uo[k, a, c]
            assert abs(abs(r) - 1.0) <= tol / abs(Uo[k, a, c]) + 1e-12, ("modulus", a, c)
            ph = r / abs(r)
            theta[(a, c)] = ph
            assert np.abs(Ug[:, a, c] - ph * Uo[:, a, c]).max() <= 2 * tol, ("entry", a, c)
    for (a, c), ph in theta.items():
        if (c, a) in theta:  # theta_ca = -theta_ac
            assert abs(ph * theta[(c, a)] - 1.0) <= 1e-6, ("inverse", a, c)
        for b in range(D):
            if (a, b) in theta and (b, c) in theta:  # theta_ac = theta_ab + theta_bc
                assert abs(theta[(a, b)] * theta[(b, c)] / ph - 1.0) <= 1e-6, ("compose", a, b, c)


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_single_system_matches_oracle(precision):
    ctx = M.Context(0)
    t1 = 1.5
    t2 = np.array([1.5, 7.0, 33.3, 60.0])
    for p in (_dressed_qubit(0.031, 0.004), _spin1_dressed(0.3, 0.05)):
        s = M.System(ctx, p)
        Ud, Eb = s.dressed_time_evolution([0], t1, t2, precision)
        refs = [O.dressed_time_evolution(p, [0], t1, float(t)) for t in t2]
        _assert_same_up_to_basis_phases(Ud, np.stack([r[0] for r in refs]), TOL[precision])
        np.testing.assert_allclose(Eb, refs[0][1], rtol=0, atol=1e-12 * max(1.0, np.abs(refs[0][1]).max()))
        np.testing.assert_allclose(Ud[0], np.eye(p.D), atol=TOL[precision])  # t2 = t1


def test_batch_matches_oracle():
    ctx = M.Context(0)
    ps = [_dressed_qubit(w, 0.004) for w in (0.02, 0.025, 0.031)] + [_spin1_dressed(0.2, 0.04)]
    systems = [M.System(ctx, p) for p in ps]
    nt = 5
    t1 = 0.7
    ts = np.stack([np.linspace(t1, t1 + 80.0, nt) for _ in ps])
    full = M.Batch(ctx, systems, M.MMF_MIXED, nt)
    full.set_times(t1, ts)
    full.run()
    assert (full.sync() == 0).all()
    dress = M.Batch(ctx, [s.restrict([0]) for s in systems], M.MMF_MIXED, 0)
    dress.run()
    assert (dress.sync() == 0).all()
    out = full.dressed(dress)
    for i, p in enumerate(ps):
        Ud, Eb = out[i]
        refs = [O.dressed_time_evolution(p, [0], t1, float(ts[i, k])) for k in range(nt)]
        _assert_same_up_to_basis_phases(Ud, np.stack([r[0] for r in refs]), 1e-8)
        np.testing.assert_allclose(Eb, refs[0][1], rtol=0, atol=1e-12)


def test_without_probe_the_dressed_evolution_is_diagonal():
    ctx = M.Context(0)
    p = _dressed_qubit(0.03, 0.0)
    t1, t2 = 3.0, np.array([41.0, 90.0])
    Ud, Eb = M.System(ctx, p).dressed_time_evolution([0], t1, t2, M.MMF_FP64)
    for k, t in enumerate(t2):
        np.testing.assert_allclose(Ud[k], np.diag(np.exp(-1j * Eb * (t - t1))), rtol=0, atol=1e-9)


def test_probe_resonance_on_the_gpu():
    """Sec. 4.1: the probe transfers population between the dressed states at their splitting."""
    ctx = M.Context(0)
    amp_pz = 0.005
    _, Eb = M.System(ctx, _dressed_qubit(0.03, 0.0)).dressed_time_evolution([0], 0.0, [1.0], M.MMF_MIXED)
    split = abs(Eb[1] - Eb[0]) % 1.0
    split = min(split, 1.0 - split)
    times = np.linspace(0.0, 2.5 * np.pi / (0.5 * amp_pz), 9)[1:]

    def transfer(wp):
        Ud, _ = M.System(ctx, _dressed_qubit(wp, amp_pz)).dressed_time_evolution([0], 0.0, times, M.MMF_MIXED)
        return float(np.max(np.abs(Ud[:, 1, 0]) ** 2))

    on, off = transfer(split), transfer(3.0 * split)
    assert on > 0.8 and off < 0.1, (on, off)


def test_restrict_checks_modes():
    ctx = M.Context(0)
    s = M.System(ctx, _dressed_qubit(0.03, 0.001))
    for bad in ([2], [0, 0], [-1]):
        with pytest.raises(M.MmfError):
            s.restrict(bad)
    r = s.restrict([1])
    assert r.n == 2 * 11
