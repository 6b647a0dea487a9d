"""The allocation-free tridiagonal eigensolver (mmf_tridiag_eig_noalloc).

It exists for callers that cannot allocate device memory (their HBM belongs to another
allocator, or cudaMalloc's implicit synchronisation is not acceptable to them).  A one-level
system driven at one frequency with a real coupling has a Floquet matrix that is already real
symmetric tridiagonal: d_b = h0 - (b - N) w, e_b = v.  The allocation-free call on (d, e) must give
the same eigenpairs as the library's regular entry points (mmf_build + mmf_diagonalise) on that
system, on two calls in a row that share the fixed scratch array.  Its results are also compared
with the FP64 oracle's Jacobi solve of the same tridiagonal matrix, at n = 1, in the middle of
the range and at the largest n the scratch array holds, and its status output is checked.

This file is collected last so that a run stopping at its first failure has run every other test.
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _chain(omega, N, h0=0.37, v=0.21):
    return W.Problem(D=1, H0=np.array([[h0]], dtype=complex), omegas=[omega], Ns=[N],
                     couplings=[[np.array([[v]], dtype=complex)]])


def _chain_tridiag(p):
    N, n, w = p.Ns[0], p.n, p.omegas[0]
    d = np.array([p.H0[0, 0].real - float(b - N) * w for b in range(n)])
    e = np.full(n - 1, p.couplings[0][0][0, 0].real)
    return d, e


def _random_tridiag(n, seed):
    rng = W.SplitMix64(seed)
    d = np.array([rng.uniform_in(-1.0, 1.0) for _ in range(n)])
    e = np.array([rng.uniform_in(-0.5, 0.5) for _ in range(n - 1)])
    return d, e


def _noalloc(d, e, with_status=True):
    import torch

    n = d.size
    dev = torch.device("cuda", 0)
    td = torch.tensor(d, device=dev)
    te = torch.tensor(e, device=dev) if n > 1 else None
    tE = torch.empty(n, dtype=torch.float64, device=dev)
    tY = torch.empty(n * n, dtype=torch.float64, device=dev)
    tS = torch.full((1,), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rc = M.lib().mmf_tridiag_eig_noalloc(td.data_ptr(), te.data_ptr() if te is not None else None, n,
                                         tE.data_ptr(), tY.data_ptr(),
                                         tS.data_ptr() if with_status else None, stream)
    assert rc == 0, M.lib().mmf_last_error()
    torch.cuda.synchronize()
    st = int(tS.cpu().item()) if with_status else 0
    return tE.cpu().numpy(), tY.cpu().numpy().reshape(n, n), st


def _regular(ctx, p):
    s = M.System(ctx, p)
    s.build(M.MMF_FP64)
    assert s.diagonalise() == 0
    return s.quasienergies(), s.eigenvectors()


def _oracle(d, e):
    n = d.size
    T = np.diag(d).astype(np.complex128)
    if n > 1:
        T += np.diag(e, 1) + np.diag(e, -1)
    w, Z, st, _ = O.eigh(T)
    assert st == 0
    return w, Z.real


def _same_vectors(Y, Z, atol):
    # distinct eigenvalues: eigenvectors agree up to a sign per column
    sgn = np.sign(np.sum(Y * Z, axis=0))
    sgn[sgn == 0] = 1.0
    return np.abs(Y * sgn[None, :] - Z).max() <= atol


def test_noalloc_matches_regular_entry_points_twice():
    ctx = M.Context(0)
    for omega in (0.93, 1.41):  # two calls in a row on the shared scratch
        p = _chain(omega, N=100)
        d, e = _chain_tridiag(p)
        E1, Y1, st = _noalloc(d, e)
        assert st == M.MMF_OK
        E0, Z0 = _regular(ctx, p)
        nrm = np.abs(E0).max()
        assert np.abs(E1 - E0).max() <= 1e-12 * nrm
        assert _same_vectors(Y1, Z0.real, 1e-10)
        assert np.abs(Z0.imag).max() <= 1e-10
        assert np.abs(Y1.T @ Y1 - np.eye(p.n)).max() <= 1e-12


@pytest.mark.parametrize("n", [1, 2, 137, 256])
def test_noalloc_matches_the_oracle(n):
    for seed in (11, 12):  # two calls in a row
        d, e = _random_tridiag(n, seed + n)
        E1, Y1, st = _noalloc(d, e, with_status=(seed == 11))
        assert st == M.MMF_OK
        w, Z = _oracle(d, e)
        nrm = np.abs(w).max()
        assert np.abs(E1 - w).max() <= 1e-12 * nrm
        gaps = np.diff(w).min() if n > 1 else 1.0
        assert gaps > 1e-6  # distinct eigenvalues: vectors are unique up to sign
        assert _same_vectors(Y1, Z, 1e-10)
        assert np.abs(Y1.T @ Y1 - np.eye(n)).max() <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = 257
    rc = M.lib().mmf_tridiag_eig_noalloc(None, None, n, None, None, None, None)
    assert rc == M.MMF_ERR_UNSUPPORTED
    assert b"256" in M.lib().mmf_last_error()
