"""Device-pointer variants of the result calls (mmf_*_dev, mmf_batch_results_dev): the results
written into torch-owned device tensors on a torch stream equal the host-array results of the
same calls, element by element, and the oracle's within the path's tolerance."""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2005_03426_gb300 import mmf as M
from paper_2005_03426_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [M.MMF_FP64, M.MMF_MIXED])
def test_single_system_dev_results(precision):
    import torch

    dev = torch.device("cuda", 0)
    p = W.spin1_bichromatic(0.3, 0.2, N1=6, N2=5)  # n = 429: Householder path in both precisions
    ctx = M.Context(0)
    s = M.System(ctx, p)
    s.build(precision)
    assert s.diagonalise() == 0
    nt = 12
    t = W.time_grid(p, nt)
    # plan the outputs for nt times first (a change of nt re-solves the system, and the reduction's
    # floating-point atomics make a re-solve differ in the last bits)
    U_host = s.time_evolution(t)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        tt = torch.tensor(t, device=dev)  # produced on the caller's stream
        E = torch.full((p.n,), float("nan"), dtype=torch.float64, device=dev)
        Z = torch.full((p.n, p.n), float("nan"), dtype=torch.complex128, device=dev)
        U = torch.full((nt, p.D, p.D), float("nan"), dtype=torch.complex128, device=dev)
        P = torch.full((p.D, p.D), float("nan"), dtype=torch.float64, device=dev)
        h = st.cuda_stream
        s.quasienergies_dev(E.data_ptr(), h)
        s.eigenvectors_dev(Z.data_ptr(), h)
        s.time_evolution_dev(0.0, nt, tt.data_ptr(), U.data_ptr(), h)
        s.transition_avg_dev(P.data_ptr(), h)
    st.synchronize()
    E, Z, U, P = E.cpu().numpy(), Z.cpu().numpy().T, U.cpu().numpy(), P.cpu().numpy()  # Z: column-major
    # E and Z: copies of the same device state as the host getters read; U and Pbar are
    # recomputed by each call (their sums use atomics, so the last bits may differ)
    np.testing.assert_array_equal(E, s.quasienergies())
    np.testing.assert_array_equal(Z, s.eigenvectors())
    np.testing.assert_allclose(U, U_host, rtol=0, atol=1e-13)
    np.testing.assert_allclose(P, s.transition_avg(), rtol=0, atol=1e-13)
    ref = O.solve(p, t=t, t0=0.0)
    e_rel, up = (1e-12, 1e-10) if precision == M.MMF_FP64 else (1e-9, 1e-8)
    assert np.abs(E - ref["E"]).max() <= e_rel * np.abs(ref["E"]).max()
    assert np.abs(U - ref["U"]).max() <= up and np.abs(P - ref["P"]).max() <= up


def test_batch_results_dev_equal_host_results():
    import torch

    dev = torch.device("cuda", 0)
    ps = [W.two_level(0.7, N=20), W.random_small(5, D=4, Ns=[6, 3], nharm=[1, 1]),
          W.spin1_bichromatic(0.2, 0.4, N1=8, N2=4)]
    nt = 8
    ctx = M.Context(0)
    b = M.Batch(ctx, [M.System(ctx, p) for p in ps], M.MMF_MIXED, nt)
    b.set_times(0.0, np.stack([W.time_grid(p, nt) for p in ps]))
    b.run()
    assert (b.sync() == 0).all()
    Eh, Uh, Ph = b.results()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        E = torch.empty(b.nE, dtype=torch.float64, device=dev)
        U = torch.empty(b.nU, dtype=torch.complex128, device=dev)
        P = torch.empty(b.nP, dtype=torch.float64, device=dev)
        b.results_dev(E.data_ptr(), U.data_ptr(), P.data_ptr(), st.cuda_stream)
        # a later run of the batch on the library's stream must not overwrite what is being read
        b.run()
    st.synchronize()
    np.testing.assert_array_equal(E.cpu().numpy(), Eh)
    np.testing.assert_array_equal(U.cpu().numpy(), Uh[:b.nU])
    np.testing.assert_array_equal(P.cpu().numpy(), Ph)
    b.sync()


def test_context_outlives_its_dependents():
    """Closing a context before its systems and batches (as garbage collection may) keeps the C
    context alive until the last dependent is closed."""
    p = W.two_level(0.9, N=10)
    ctx = M.Context(0)
    s = M.System(ctx, p)
    b = M.Batch(ctx, [s], M.MMF_FP64, 2)
    ctx.close()
    assert ctx.h is not None
    b.set_times(0.0, W.time_grid(p, 2)[None, :])
    b.run()
    assert (b.sync() == 0).all()
    s.close()
    assert ctx.h is not None
    b.close()
    assert ctx.h is None


def test_dev_calls_check_their_state():
    p = W.two_level(0.9, N=10)
    ctx = M.Context(0)
    s = M.System(ctx, p)
    s.build(M.MMF_FP64)
    with pytest.raises(M.MmfError) as ei:
        s.quasienergies_dev(1 << 20, 0)  # before mmf_diagonalise: refused before any copy
    assert ei.value.code == M.MMF_ERR_STATE
    assert M.lib().mmf_quasienergies_dev(s.h, None, None) == M.MMF_ERR_ARG
