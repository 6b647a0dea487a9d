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
