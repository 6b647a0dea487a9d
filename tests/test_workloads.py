"""Shapes of the seeded synthetic workloads (no method arithmetic involved)."""

import math

import numpy as np

from paper_2005_03426_gb300 import workloads as W


def test_splitmix64_reference_values():
    # SplitMix64 with seed 0: first outputs of the published generator
    r = W.SplitMix64(0)
    assert r.next_u64() == 0xE220A8397B1DCDAF
    assert r.next_u64() == 0x6E789E6AA1B965F4
    assert r.next_u64() == 0x06C45D188009454F


def test_qubit_sweep_shape():
    ps = W.qubit_sweep()
    assert len(ps) == 200 and all(p.n == 82 for p in ps)
    assert ps[0].omegas[0] == 0.2 and ps[-1].omegas[0] == 2.0
    np.testing.assert_array_equal(ps[0].couplings[0][0], [[0, 0.25], [0.25, 0]])


def test_spin1_set_shape():
    ps = W.spin1_amplitude_set()
    assert len(ps) == 64 and all(p.n == 1323 for p in ps)
    for p in ps:
        a1 = 2 * p.couplings[0][0][0, 1].real * math.sqrt(2)
        assert 0.05 <= a1 <= 0.5
    assert abs(ps[0].omegas[1] - 0.6180339887498949) < 1e-15


def test_uneven_batch_shape():
    ps = W.uneven_batch(count=300)
    ns = [p.n for p in ps]
    assert min(ns) >= 18 and max(ns) <= 2000
    for p in ps:
        assert 2 <= p.D <= 8 and p.K in (1, 2)
        for V in (c[0] for c in p.couplings):
            assert np.array_equal(V, V.conj().T)


def test_large_instance_shape():
    p = W.large_instance()
    assert p.n == 17576 and p.D == 8
    ev = np.linalg.eigvalsh(p.H0)
    assert ev.min() >= 0.0 and ev.max() <= 2.0
    assert np.allclose(p.H0, p.H0.conj().T)


def test_driven_lattice_matches_eq9_in_time_domain():
    """H(t) = H0 + V e^{iwt} + V^dagger e^{-iwt} from the generator equals Eq. 9 evaluated
    directly at several times (offsets (-1)^m V0, hopping t e^{i cos(2 pi m/D)}, and the bond
    modulation V cos(w t + phi)), for a nonzero phase."""
    D, w, V0, tt, V, phi = 10, 0.55, 0.25, 0.125, 0.0625, 0.4
    p = W.driven_lattice(w, D=D, N=2, V0=V0, t=tt, V=V, phi=phi)
    assert p.n == D * 5 and p.K == 1 and p.Ns == [2]
    for time in (0.0, 0.37, 2.9):
        H = p.H0 + p.couplings[0][0] * np.exp(1j * w * time) + \
            p.couplings[0][0].conj().T * np.exp(-1j * w * time)
        ref = np.zeros((D, D), dtype=complex)
        for m in range(1, D + 1):
            ref[m - 1, m - 1] = (-1) ** m * V0
        for m in range(1, D):
            hop = tt * np.exp(1j * math.cos(2 * math.pi * m / D)) + V * math.cos(w * time + phi)
            ref[m - 1, m] += hop
            ref[m, m - 1] += np.conj(hop)
        np.testing.assert_allclose(H, ref, rtol=0, atol=1e-15)


def test_lattice_sweep_shape():
    ps = W.lattice_sweep()
    assert len(ps) == 64 and all(p.n == 1792 and p.D == 256 for p in ps)
    assert ps[0].omegas[0] == 0.2 and ps[-1].omegas[0] == 1.0


def test_driven_lattice_has_exactly_degenerate_mirror_pairs():
    """The driven lattice's Floquet spectrum contains exactly degenerate pairs: mirror-image
    states localised near sites D/4 and 3D/4.  The undriven chain has none.  These pairs are
    why the mixed path's refinement clusters pairs by absolute gap.  LAPACK on the FP64 H_F;
    N = 1 keeps it small."""
    from oracle import oracle as O

    p = W.driven_lattice(0.6, D=256, N=1)
    E, Z = np.linalg.eigh(O.build_hf(p))
    gaps = np.diff(E)
    pairs = np.nonzero(gaps < 1e-12 * np.abs(E).max())[0]
    assert len(pairs) >= 4
    D = p.D
    for k in pairs[:2]:
        centres = []
        for col in (k, k + 1):
            w = np.bincount(np.arange(Z.shape[0]) % D, weights=np.abs(Z[:, col]) ** 2, minlength=D)
            centres.append((w * np.arange(D)).sum())
        lo, hi = sorted(c / D for c in centres)
        assert abs(lo - 0.25) < 0.05 and abs(hi - 0.75) < 0.05, (lo, hi)
    E0 = np.linalg.eigvalsh(W.driven_lattice(0.6, D=256, N=0).H0)
    assert (np.diff(E0) > 1e-9).all()
