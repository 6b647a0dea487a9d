"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the block layout
printed in Appendix A, closed-form solutions, LAPACK, scipy's expm and ODE
integrators, and invariants.  None needs a GPU.
"""

import math
import os

import numpy as np
import pytest
import scipy.linalg
from scipy.integrate import solve_ivp

from oracle import oracle as O
from paper_2005_03426_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_herm(rng, D, scale=1.0):
    G = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    return scale * 0.5 * (G + G.conj().T)


# --------------------------------------------------------------------- assembly
def _parse_blocks(tag):
    rows = []
    with open(os.path.join(GOLDEN, "appendix_a_blocks.txt")) as f:
        for line in f:
            if line.startswith(tag + " "):
                rows.append(line.split()[1:])
    return rows


def test_appendix_a_layout():
    """Appendix A: H0 driven at w1 (harmonics 1, 2) and w2 (harmonic 1), N_F = 3.
    The expected matrix is assembled block by block from the printed pattern."""
    rng = np.random.default_rng(11)
    D = 2
    H0 = _rand_herm(rng, D)
    V11 = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    V12 = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    V21 = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    w1, w2 = 0.731, 1.187
    p = W.Problem(D=D, H0=H0, omegas=[w1, w2], Ns=[3, 3], couplings=[[V11, V12], [V21]])

    tok1 = {"V11": V11, "V12": V12, "V11*": V11.conj().T, "V12*": V12.conj().T,
            "0": np.zeros((D, D))}
    H1 = np.zeros((7 * D, 7 * D), dtype=complex)
    for r, row in enumerate(_parse_blocks("H1")):
        for c, t in enumerate(row):
            blk = H0 + int(t[1:]) * w1 * np.eye(D) if t.startswith("D") else tok1[t]
            H1[r * D:(r + 1) * D, c * D:(c + 1) * D] = blk
    Wb = np.kron(np.eye(7), V21)
    tok2 = {"W": Wb, "W*": Wb.conj().T, "0": np.zeros((7 * D, 7 * D))}
    m = 7 * D
    H = np.zeros((7 * m, 7 * m), dtype=complex)
    for r, row in enumerate(_parse_blocks("H2")):
        for c, t in enumerate(row):
            blk = H1 + int(t[1:]) * w2 * np.eye(m) if t.startswith("E") else tok2[t]
            H[r * m:(r + 1) * m, c * m:(c + 1) * m] = blk

    HF = O.build_hf(p)
    assert HF.shape == (98, 98)
    np.testing.assert_allclose(HF, H, rtol=0, atol=1e-14)


def test_hf_hermitian_bitwise_and_diagonal_rounding():
    p = W.random_small(5, D=3, Ns=[2, 3], nharm=[2, 1])
    HF = O.build_hf(p)
    assert np.array_equal(HF, HF.conj().T)
    # diagonal = E_ii - sum_k n_k w_k, accumulated k ascending, no fused multiply-add
    D = p.D
    for b in range(p.M):
        n1 = b % 5 - 2
        n2 = b // 5 - 3
        s = 0.0
        s = s + float(n1) * p.omegas[0]
        s = s + float(n2) * p.omegas[1]
        for i in range(D):
            assert HF[b * D + i, b * D + i].real == p.H0[i, i].real - s
            assert HF[b * D + i, b * D + i].imag == 0.0


def test_dimension_rule():
    p = W.random_small(1, D=4, Ns=[1, 2, 3])
    assert O.dim(p) == 4 * 3 * 5 * 7


# --------------------------------------------------------------------- eigensolver
@pytest.mark.parametrize("n", [1, 2, 17, 64])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    A = _rand_herm(rng, n, 3.0)
    w, Z, st, _ = O.eigh(A)
    assert st == 0
    nrm = np.linalg.norm(A, 2)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-13 * nrm)
    assert np.abs(A @ Z - Z * w[None, :]).max() <= 1e-13 * nrm
    assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= 1e-13


def test_jacobi_degenerate_and_diagonal():
    A = np.diag([3.0, -1.0, 3.0, 0.5]).astype(complex)
    w, Z, st, sweeps = O.eigh(A)
    assert st == 0 and sweeps == 0
    assert list(w) == [-1.0, 0.5, 3.0, 3.0]
    # ties keep the original column order
    assert np.argmax(np.abs(Z[:, 2])) == 0 and np.argmax(np.abs(Z[:, 3])) == 2


def test_jacobi_sweep_cap_reports_status():
    rng = np.random.default_rng(3)
    A = _rand_herm(rng, 30)
    _, _, st, sweeps = O.eigh(A, max_sweeps=1)
    assert st == 1 and sweeps == 1


# --------------------------------------------------------------------- closed forms
def _circular_tls(omega0, omega, Omega, N):
    H0 = np.diag([0.5 * omega0, -0.5 * omega0]).astype(complex)
    V = np.zeros((2, 2), dtype=complex)
    V[1, 0] = 0.5 * Omega
    return W.Problem(D=2, H0=H0, omegas=[omega], Ns=[N], couplings=[[V]])


@pytest.mark.parametrize("N", [1, 3, 8])
def test_circular_rabi_closed_form(N):
    """H = (w0/2) sz + (Omega/2)(|1><0| e^{iwt} + h.c.): H_F splits into 2 x 2 blocks with
    eigenvalues -(k + 1/2) w +- sqrt(Delta^2 + Omega^2)/2 (k = -N..N-1) plus the edge
    singletons +-(w0/2 + N w), and Pbar_{0->1} = Omega^2 / (2 (Delta^2 + Omega^2))."""
    w0, w, Om = 1.0, 0.7, 0.3
    p = _circular_tls(w0, w, Om, N)
    r = O.solve(p)
    delta = w0 - w
    R = 0.5 * math.sqrt(delta ** 2 + Om ** 2)
    ev = [-(k + 0.5) * w + s * R for k in range(-N, N) for s in (-1, 1)]
    ev += [0.5 * w0 + N * w, -(0.5 * w0 + N * w)]
    np.testing.assert_allclose(r["E"], np.sort(ev), rtol=0, atol=1e-13)
    pb = Om ** 2 / (2 * (delta ** 2 + Om ** 2))
    np.testing.assert_allclose(r["P"], [[1 - pb, pb], [pb, 1 - pb]], rtol=0, atol=1e-13)


def test_commuting_drive_closed_form():
    """H = (w0/2) sz + A cos(wt) sz: U = exp(-i sz [w0 (t-t0)/2 + (A/w)(sin wt - sin wt0)]),
    Pbar = I."""
    w0, A, w = 1.0, 0.8, 0.9
    sz = np.diag([1.0, -1.0]).astype(complex)
    p = W.Problem(D=2, H0=0.5 * w0 * sz, omegas=[w], Ns=[25], couplings=[[0.5 * A * sz]])
    t = np.array([0.0, 0.37, 2.9, 6.5])
    t0 = 0.41
    r = O.solve(p, t=t, t0=t0)
    for k, tk in enumerate(t):
        phi = w0 * (tk - t0) / 2 + (A / w) * (math.sin(w * tk) - math.sin(w * t0))
        exact = np.diag([np.exp(-1j * phi), np.exp(1j * phi)])
        np.testing.assert_allclose(r["U"][k], exact, rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["P"], np.eye(2), rtol=0, atol=1e-13)


def test_spin1_is_su2_representation():
    """H linear in (Fx, Fz): the spin-1 evolution is the symmetric square of the spin-1/2
    evolution with the same coefficients (|1,1>, |1,0>, |1,-1> = |uu>, (|ud>+|du>)/sqrt2, |dd>)."""
    a1, a2 = 0.2, 0.15
    Ns = [6, 5]
    p1 = W.spin1_bichromatic(a1, a2, N1=Ns[0], N2=Ns[1])
    Fx, _, Fz = W.spin_matrices(1)
    w1, w2 = p1.omegas
    ph = W.Problem(D=2, H0=1.0 * Fz, omegas=[w1, w2], Ns=Ns,
                   couplings=[[0.5 * a1 * Fx], [0.5 * a2 * Fz]])
    t = np.array([0.4, 1.2])  # truncation error grows with t; converged here to ~1e-10
    U1 = O.solve(p1, t=t)["U"]
    Uh = O.solve(ph, t=t)["U"]
    P = np.zeros((4, 3))
    P[0, 0] = 1.0
    P[1, 1] = P[2, 1] = 1 / math.sqrt(2)
    P[3, 2] = 1.0
    for k in range(t.size):
        rep = P.T @ np.kron(Uh[k], Uh[k]) @ P
        np.testing.assert_allclose(U1[k], rep, rtol=0, atol=1e-9)


# --------------------------------------------------------------------- invariants
def test_zero_coupling():
    """V = 0: E = sorted{E_i - n.w}, U = diag(e^{-i E_i (t - t0)}), Pbar = I."""
    D = 3
    Ei = np.array([0.13, 0.71, -0.44])
    p = W.Problem(D=D, H0=np.diag(Ei).astype(complex), omegas=[1.0, math.sqrt(2)], Ns=[2, 1],
                  couplings=[[np.zeros((D, D))], [np.zeros((D, D))]])
    t, t0 = np.array([0.0, 1.3, 4.4]), 0.5
    r = O.solve(p, t=t, t0=t0)
    ev = sorted(e - (n1 * 1.0 + n2 * math.sqrt(2)) for e in Ei for n1 in range(-2, 3)
                for n2 in range(-1, 2))
    np.testing.assert_allclose(r["E"], ev, rtol=0, atol=1e-14)
    for k, tk in enumerate(t):
        np.testing.assert_allclose(r["U"][k], np.diag(np.exp(-1j * Ei * (tk - t0))), atol=1e-14)
    np.testing.assert_allclose(r["P"], np.eye(D), atol=1e-14)


def test_static_lattice_closed_form():
    """Undriven lattice of Eq. 9 (V = 0): the staggered offsets anticommute with the
    nearest-neighbour hopping, so H0^2 = V0^2 + T^2, and T (an open chain with |t| on every
    bond; the bond phases gauge away) has eigenvalues 2 t cos(pi j/(D+1)).  Hence the static
    levels are +-sqrt(V0^2 + 4 t^2 cos^2(pi j/(D+1))), j = 1..D/2, and the quasienergies are
    those levels shifted by k w, k = -N..N.  With no drive, Pbar is the static time average
    sum_a |<j|a>|^2 |<a|i>|^2 over the eigenvectors of H0 (LAPACK's, levels nondegenerate)."""
    D, N, w, V0, tt = 12, 2, 0.53, 0.25, 0.125
    p = W.driven_lattice(w, D=D, N=N, V0=V0, t=tt, V=0.0)
    lev = [s * math.sqrt(V0 ** 2 + 4 * tt ** 2 * math.cos(math.pi * j / (D + 1)) ** 2)
           for j in range(1, D // 2 + 1) for s in (1.0, -1.0)]
    ev = sorted(e + k * w for e in lev for k in range(-N, N + 1))
    r = O.solve(p)
    np.testing.assert_allclose(r["E"], ev, rtol=0, atol=1e-14)
    _, Q = np.linalg.eigh(p.H0)
    w2 = np.abs(Q) ** 2
    np.testing.assert_allclose(r["P"], w2 @ w2.T, rtol=0, atol=1e-13)


def test_driven_lattice_matches_time_domain_integration():
    """Driven lattice of Eq. 9 with a nonzero drive phase: the Floquet U(t, t0) at a converged
    truncation equals DOP853 integration of Eq. 1 with H(t) written out from Eq. 9."""
    D, w, V0, tt, V, phi = 6, 0.7, 0.25, 0.125, 0.3, 0.9

    def ham(time):
        H = np.zeros((D, D), dtype=complex)
        for m in range(1, D + 1):
            H[m - 1, m - 1] = (-1) ** m * V0
        for m in range(1, D):
            hop = tt * np.exp(1j * math.cos(2 * math.pi * m / D)) + V * math.cos(w * time + phi)
            H[m - 1, m] = hop
            H[m, m - 1] = np.conj(hop)
        return H

    t0, t1 = 0.2, 3.1
    sol = solve_ivp(lambda s, y: (-1j * ham(s) @ y.reshape(D, D)).reshape(-1), (t0, t1),
                    np.eye(D, dtype=complex).reshape(-1), method="DOP853", rtol=1e-12, atol=1e-13)
    p = W.driven_lattice(w, D=D, N=14, V0=V0, t=tt, V=V, phi=phi)
    U_f = O.solve(p, t=np.array([t1]), t0=t0)["U"][0]
    np.testing.assert_allclose(U_f, sol.y[:, -1].reshape(D, D), rtol=0, atol=1e-9)


def test_identity_at_t0_and_sum_rule():
    p = W.random_small(7, D=3, Ns=[2, 2], nharm=[2, 1])
    t0 = 0.77
    r = O.solve(p, t=np.array([t0]), t0=t0)
    np.testing.assert_allclose(r["U"][0], np.eye(3), rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["P"].sum(axis=1), np.ones(3), rtol=0, atol=1e-13)
    assert (r["P"] >= -1e-15).all()


def test_expm_identity():
    """U(t, t0)_{ji} = sum_n e^{-i n.w t} [expm(-i H_F (t - t0))]_{(j,n),(i,0)} exactly at
    any truncation (scipy's expm as the independent reference)."""
    p = W.random_small(9, D=2, Ns=[3, 2], nharm=[1, 2])
    t, t0 = np.array([0.3, 2.2, 5.0]), 0.6
    r = O.solve(p, t=t, t0=t0)
    D, M = p.D, p.M
    b0 = 3 + 7 * 2
    nw = np.array([(b % 7 - 3) * p.omegas[0] + (b // 7 - 2) * p.omegas[1] for b in range(M)])
    for k, tk in enumerate(t):
        G = scipy.linalg.expm(-1j * r["HF"] * (tk - t0))
        U = np.zeros((D, D), dtype=complex)
        for b in range(M):
            U += np.exp(-1j * nw[b] * tk) * G[b * D:(b + 1) * D, b0 * D:(b0 + 1) * D]
        np.testing.assert_allclose(r["U"][k], U, rtol=0, atol=1e-11)


def _ham(p, t):
    H = p.H0.astype(complex).copy()
    for l, cl in enumerate(p.couplings):
        for h, V in enumerate(cl, start=1):
            e = np.exp(1j * h * p.omegas[l] * t)
            H += V * e + V.conj().T * np.conj(e)
    return H


def _ivp(p, t0, t1):
    D = p.D

    def f(t, y):
        U = y.reshape(D, D)
        return (-1j * _ham(p, t) @ U).reshape(-1)

    sol = solve_ivp(f, (t0, t1), np.eye(D, dtype=complex).reshape(-1), method="DOP853",
                    rtol=1e-12, atol=1e-13)
    return sol.y[:, -1].reshape(D, D)


def test_rk4_matches_scipy_integrator():
    p = W.random_small(4, D=3, Ns=[1, 1], nharm=[2, 1], sigma=0.2)
    U_rk = O.rk4(p, 0.3, 2.5, 4000)
    np.testing.assert_allclose(U_rk, _ivp(p, 0.3, 2.5), rtol=0, atol=1e-10)


def test_floquet_matches_time_domain_integration():
    """Brute force: the Floquet U(t, t0) of a converged truncation equals direct RK4
    integration of i dpsi/dt = H(t) psi (Eq. 1), with t0 != 0: a D = 3 system with two
    harmonics of one drive, and the two-mode spin-1 system."""
    p = W.random_small(21, D=3, Ns=[16], nharm=[2], sigma=0.15, full_h0=True)
    t0, t1 = 0.45, 2.0
    U_f = O.solve(p, t=np.array([t1]), t0=t0)["U"][0]
    np.testing.assert_allclose(U_f, O.rk4(p, t0, t1, 6000), rtol=0, atol=1e-10)
    p = W.spin1_bichromatic(0.2, 0.15, 6, 5)
    U_f = O.solve(p, t=np.array([1.1]), t0=0.3)["U"][0]
    np.testing.assert_allclose(U_f, O.rk4(p, 0.3, 1.1, 4000), rtol=0, atol=1e-9)


def test_convergence_in_truncation():
    errs = []
    t = np.array([1.7])
    ref = O.solve(W.two_level(0.9, N=24), t=t)["U"][0]
    for N in (2, 4, 6, 8):
        U = O.solve(W.two_level(0.9, N=N), t=t)["U"][0]
        errs.append(np.abs(U - ref).max())
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-6
    p2 = W.spin1_bichromatic(0.2, 0.15, 2, 2)
    p4 = W.spin1_bichromatic(0.2, 0.15, 4, 4)
    e2 = np.abs(O.solve(p2, t=t)["U"][0] - O.rk4(p2, 0.0, 1.7, 3000)).max()
    e4 = np.abs(O.solve(p4, t=t)["U"][0] - O.rk4(p4, 0.0, 1.7, 3000)).max()
    assert e4 < 0.1 * e2


def test_quasienergy_periodicity():
    """Interior eigenvalues recur shifted by w (Floquet-copy structure of Eq. 6)."""
    p = W.two_level(1.1, N=20)
    E = O.solve(p)["E"]
    inner = E[np.abs(E) < 5 * 1.1]
    for e in inner:
        assert np.min(np.abs(E - (e + 1.1))) < 1e-12


def test_pbar_invariant_inside_degenerate_cluster():
    """Exact degeneracy: rotating eigenvectors inside a degenerate cluster leaves Pbar
    unchanged, and a time average of |U|^2 reproduces it."""
    D = 2
    H0 = np.diag([0.3, 0.3]).astype(complex)
    V = np.array([[0.0, 0.2], [0.2, 0.0]], dtype=complex)
    p = W.Problem(D=D, H0=H0, omegas=[1.3], Ns=[6], couplings=[[V]])
    r = O.solve(p)
    E, Z = r["E"], r["Z"].copy()
    rng = np.random.default_rng(0)
    c0 = 0
    while c0 < E.size:
        c1 = c0 + 1
        while c1 < E.size and E[c1] - E[c1 - 1] < 1e-8 * np.abs(E).max():
            c1 += 1
        if c1 - c0 > 1:
            G = rng.standard_normal((c1 - c0,) * 2) + 1j * rng.standard_normal((c1 - c0,) * 2)
            Qr, _ = np.linalg.qr(G)
            Z[:, c0:c1] = Z[:, c0:c1] @ Qr
        c0 = c1
    np.testing.assert_allclose(O.transition_avg(p, E, Z), r["P"], atol=1e-13)


def test_pbar_equals_brute_force_time_average():
    """Pbar against an explicit average of |U(t0 + tau, t0)|^2 over t0 in one period and a long
    tau window, with U from an expm of H_F (LAPACK's eigh, independent of the oracle's Jacobi).
    The tau average is Hann-weighted over [0, L]: an oscillating term e^{i Delta tau} then
    averages to O((Delta L)^-3) instead of O((Delta L)^-1) (1.4e-4 with a flat window at
    L = 3000, 3e-10 with the Hann window at L = 6000).  The 32 points of t0 average every
    harmonic difference |n - n'| <= 12 of the truncation exactly."""
    p = W.two_level(1.37, N=6)
    HF = O.build_hf(p)
    D, M = 2, p.M
    b0 = 6
    nw = np.array([(b - 6) * p.omegas[0] for b in range(M)])
    # U(t0 + tau, t0) = sum_n e^{-i n w (t0 + tau)} [expm(-i HF tau)]_{(j,n),(i,0)}
    evals, evecs = np.linalg.eigh(HF)  # LAPACK, only to evaluate expm cheaply on a grid
    T = 2 * math.pi / p.omegas[0]
    L = 6000.0
    taus = np.linspace(0.0, L, 24001)
    wts = np.sin(np.pi * taus / L) ** 2
    Zb = evecs[b0 * D:(b0 + 1) * D, :].conj().T
    G = np.einsum("ak,tk,ki->tai", evecs, np.exp(-1j * np.outer(taus, evals)), Zb).reshape(taus.size, M, D, D)
    acc = np.zeros((D, D))
    t0s = np.linspace(0, T, 32, endpoint=False)
    for t0 in t0s:
        U = np.einsum("tb,tbji->tji", np.exp(-1j * np.outer(t0 + taus, nw)), G)
        acc += np.einsum("t,tji->ji", wts, np.abs(U) ** 2)
    acc /= wts.sum() * t0s.size
    P = O.solve(p)["P"]
    # acc[j, i] = avg |U_ji|^2 = Pbar_{i->j}
    np.testing.assert_allclose(acc.T, P, atol=2e-9)


# ------------------------------------------------------------ dressed basis (Sec. 3.3)
def _dressed_qubit(omega_p, amp_pz, N_d=6, N_p=5, amp_x=0.05):
    """Qubit of Eq. 8: w0 S_z, a resonant dressing drive amp_x cos(t) S_x (mode 1) and a probe
    amp_pz cos(omega_p t) S_z (mode 2)."""
    sx = 0.5 * np.array([[0, 1], [1, 0]], dtype=complex)
    sz = 0.5 * np.array([[1, 0], [0, -1]], dtype=complex)
    return W.Problem(D=2, H0=1.0 * sz, omegas=[1.0, omega_p], Ns=[N_d, N_p],
                     couplings=[[0.5 * amp_x * sx], [0.5 * amp_pz * sz]])


def test_dressed_frame_without_probe_is_diagonal():
    """Eq. 4 with only the dressing modes driving: U(t2, t1) = U_F(t2) e^{-i Ebar (t2 - t1)}
    U_F(t1)^dagger, so the dressed-frame evolution is diag(e^{-i Ebar_a (t2 - t1)}), whereas
    the bare-frame evolution mixes the levels (Rabi oscillation of the dressing drive)."""
    p = _dressed_qubit(0.03, 0.0)
    t1, t2 = 3.0, 41.0
    Ud, Eb = O.dressed_time_evolution(p, [0], t1, t2)
    np.testing.assert_allclose(Ud, np.diag(np.exp(-1j * Eb * (t2 - t1))), rtol=0, atol=1e-9)
    U = O.solve(p, t=np.array([t2]), t0=t1)["U"][0]
    assert abs(U[1, 0]) > 0.3


def test_dressed_frame_probe_resonance():
    """Sec. 4.1: a weak probe along z drives transitions between the two dressed states when
    its frequency matches their splitting (about amp_x / 2), and hardly at all when detuned by
    much more than its own Rabi frequency."""
    amp_pz = 0.005
    Eb = O.dressed_time_evolution(_dressed_qubit(0.03, 0.0), [0], 0.0, 1.0)[1]
    split = abs(Eb[1] - Eb[0]) % 1.0
    split = min(split, 1.0 - split)
    assert abs(split - 0.025) < 2e-3
    times = np.linspace(0.0, 2.5 * np.pi / (0.5 * amp_pz), 9)[1:]

    def transfer(wp):
        p = _dressed_qubit(wp, amp_pz)
        return max(abs(O.dressed_time_evolution(p, [0], 0.0, t)[0][1, 0]) ** 2 for t in times)

    on, off = transfer(split), transfer(3.0 * split)
    assert on > 0.8 and off < 0.1, (on, off)


def test_dressed_frame_is_unitary():
    Ud, _ = O.dressed_time_evolution(_dressed_qubit(0.031, 0.004), [0], 1.5, 60.0)
    np.testing.assert_allclose(Ud.conj().T @ Ud, np.eye(2), rtol=0, atol=1e-8)
