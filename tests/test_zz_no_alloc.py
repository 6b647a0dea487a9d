"""The allocation-free tridiagonal eigensolver (mmf_tridiag_eig_noalloc).

It exists for callers that cannot allocate device memory (their HBM belongs to another
allocator, or cudaMalloc's implicit synchronisation is not acceptable to them).  A one-level
system driven at one frequency with a real coupling has a Floquet matrix that is already real
symmetric tridiagonal: d_b = h0 - (b - N) w, e_b = v.  The allocation-free call on (d, e) must give
the same eigenpairs as the library's regular entry points (mmf_build + mmf_diagonalise) on that
system, on two calls in a row that share the fixed scratch array.
"""

import numpy as np
import pytest

from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _chain(omega, N, h0=0.37, v=0.21):
    return W.Problem(D=1, H0=np.array([[h0]], dtype=complex), omegas=[omega], Ns=[N],
                     couplings=[[np.array([[v]], dtype=complex)]])


def _noalloc(p):
    import torch

    N, n, w = p.Ns[0], p.n, p.omegas[0]
    d = np.array([p.H0[0, 0].real - float(b - N) * w for b in range(n)])
    e = np.full(n - 1, p.couplings[0][0][0, 0].real)
    dev = torch.device("cuda", 0)
    td = torch.tensor(d, device=dev)
    te = torch.tensor(e, device=dev)
    tE = torch.empty(n, dtype=torch.float64, device=dev)
    tY = torch.empty(n * n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    rc = M.lib().mmf_tridiag_eig_noalloc(td.data_ptr(), te.data_ptr(), n, tE.data_ptr(),
                                         tY.data_ptr(), stream)
    assert rc == 0, M.lib().mmf_last_error()
    torch.cuda.synchronize()
    return tE.cpu().numpy(), tY.cpu().numpy().reshape(n, n)


def _regular(ctx, p):
    s = M.System(ctx, p)
    s.build(M.MMF_FP64)
    assert s.diagonalise() == 0
    return s.quasienergies(), s.eigenvectors()


def test_noalloc_matches_regular_entry_points_twice():
    ctx = M.Context(0)
    for omega in (0.93, 1.41):  # two calls in a row on the shared scratch
        p = _chain(omega, N=100)
        E1, Y1 = _noalloc(p)
        E0, Z0 = _regular(ctx, p)
        nrm = np.abs(E0).max()
        assert np.abs(E1 - E0).max() <= 1e-12 * nrm
        # distinct eigenvalues: eigenvectors agree up to a sign per column
        sgn = np.sign(np.sum(Y1 * Z0.real, axis=0))
        assert np.abs(Y1 * sgn[None, :] - Z0.real).max() <= 1e-10
        assert np.abs(Z0.imag).max() <= 1e-10
        assert np.abs(Y1.T @ Y1 - np.eye(p.n)).max() <= 1e-12


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = 257
    rc = M.lib().mmf_tridiag_eig_noalloc(None, None, n, None, None, None)
    assert rc == M.MMF_ERR_UNSUPPORTED
    assert b"256" in M.lib().mmf_last_error()
