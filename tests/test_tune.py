"""The autotuner's bucketing and candidate lists (host logic, no GPU)."""

from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import tune as T


def test_buckets_cover_every_size_and_band():
    seen = set()
    for n in list(range(1, 3000, 7)) + [2 ** 20]:
        for band in (1, 8, 9, 16, 17, 32, 33, 48, 49, 64, 65, 4000):
            nb, bc = T.bucket_of(n, band)
            assert nb[0] <= n <= nb[1] and bc[0] <= band <= bc[1]
            seen.add((nb, bc))
    assert len(seen) == (len(T.N_EDGES) - 1) * len(T.BAND_CLASSES)


def test_candidates():
    # small: Jacobi or Householder; mixed Householder below 128 has no tensor-core choice
    assert T.candidates(M.MMF_MIXED, (65, 84), (0, 8), True) == [(1, -1, -1), (0, 0, -1), (0, 1, -1)]
    # beyond the Jacobi kernel's size, mixed: band, or dense with either back-transform
    assert T.candidates(M.MMF_MIXED, (1024, 1399), (49, 64), True) == [(0, 0, 1), (0, 0, 0), (0, 1, -1)]
    assert T.candidates(M.MMF_FP64, (1024, 1399), (49, 64), True) == [(0, 0, -1), (0, 1, -1)]
    # a band too wide for the chase: only the dense reduction (nothing to tune on FP64)
    assert T.candidates(M.MMF_FP64, (1400, 2047), (65, 2 ** 31 - 1), False) == [(0, 0, -1)]


def test_sample_spreads_over_the_bucket():
    """A bucket's sample takes systems spread over its whole list (every source workload that
    falls in it), not the first ones."""
    items = list(range(200))
    got = T.spread(items, 64)
    assert len(got) == 64 and got[0] == 0 and got[-1] >= 190 and len(set(got)) == 64
    assert T.spread(items[:10], 64) == items[:10]
