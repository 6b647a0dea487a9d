"""Spin couplings from field amplitudes and phases (Sec. 3.4, Eq. 7).

The oracle's angular-momentum matrices are pinned by the algebra, and its drive convention by
Eq. 8 in the time domain. The library's host-side builder (mmf_spin_components, no GPU) then
matches the oracle element by element.
"""

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import build as B
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W


@pytest.mark.parametrize("S2", [1, 2, 3, 4, 7])
def test_spin_operators_obey_the_algebra(S2):
    Sx, Sy, Sz = O.spin_operators(S2)
    S = S2 / 2.0
    np.testing.assert_allclose(Sx @ Sy - Sy @ Sx, 1j * Sz, atol=1e-13)
    np.testing.assert_allclose(Sy @ Sz - Sz @ Sy, 1j * Sx, atol=1e-13)
    np.testing.assert_allclose(Sz @ Sx - Sx @ Sz, 1j * Sy, atol=1e-13)
    np.testing.assert_allclose(Sx @ Sx + Sy @ Sy + Sz @ Sz, S * (S + 1) * np.eye(S2 + 1), atol=1e-13)
    np.testing.assert_allclose(np.linalg.eigvalsh(Sx), np.sort([S - k for k in range(S2 + 1)]), atol=1e-13)


def test_spin_half_is_pauli_over_two():
    Sx, Sy, Sz = O.spin_operators(1)
    np.testing.assert_array_equal(Sx, 0.5 * np.array([[0, 1], [1, 0]]))
    np.testing.assert_array_equal(Sy, 0.5 * np.array([[0, -1j], [1j, 0]]))
    np.testing.assert_array_equal(Sz, 0.5 * np.array([[1, 0], [0, -1]]))


def test_drive_convention_matches_eq8_in_time_domain():
    """H(t) = H0 + V e^{iwt} + V^dagger e^{-iwt} from the builder equals Eq. 8's
    w0 S_z + sum_i A_i cos(w t + phi_i) S_i written out, for a spin-1 with all three components."""
    S2, w0, w = 2, 1.0, 0.73
    A, phi = (0.4, 0.25, 0.3), (0.2, -1.1, 2.0)
    Sx, Sy, Sz = O.spin_operators(S2)
    H0 = O.spin_components(S2, (0.0, 0.0, w0), static=True)
    V = O.spin_components(S2, A, phi)
    for t in (0.0, 0.9, 3.7):
        H = H0 + V * np.exp(1j * w * t) + V.conj().T * np.exp(-1j * w * t)
        ref = w0 * Sz + sum(A[k] * math.cos(w * t + phi[k]) * op for k, op in enumerate((Sx, Sy, Sz)))
        np.testing.assert_allclose(H, ref, atol=1e-15)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


@pytest.mark.parametrize("S2", [1, 2, 3, 6, 9])
@pytest.mark.parametrize("static", [False, True])
def test_library_builder_matches_oracle(lib, S2, static):
    rng = np.random.default_rng(S2 + 10 * static)
    A = rng.uniform(-1, 1, 3)
    phi = rng.uniform(-math.pi, math.pi, 3)
    V = M.spin_components(S2, A, phi, static=static)
    np.testing.assert_allclose(V, O.spin_components(S2, A, phi, static=static), rtol=0, atol=1e-15)


def test_library_builder_reproduces_the_spin1_workload(lib):
    p = W.spin1_bichromatic(0.37, 0.21)
    assert np.allclose(M.spin_components(2, (0.0, 0.0, 1.0), static=True), p.H0, rtol=0, atol=1e-15)
    assert np.allclose(M.spin_components(2, (0.37, 0.0, 0.0)), p.couplings[0][0], rtol=0, atol=1e-15)
    assert np.allclose(M.spin_components(2, (0.0, 0.0, 0.21)), p.couplings[1][0], rtol=0, atol=1e-15)


def test_library_builder_rejects_bad_arguments(lib):
    with pytest.raises(M.MmfError):
        M.spin_components(0, (1.0, 0.0, 0.0))
