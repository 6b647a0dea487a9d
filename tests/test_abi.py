"""The C ABI library builds, loads and exports every function include/mmf.h declares; host-side
argument checks work without a GPU.  No GPU compute here."""

import ctypes
import subprocess

import numpy as np
import pytest

from paper_2005_03426_gb300 import build as B
from paper_2005_03426_gb300 import mmf as M


def _has_gpu():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.lib()


def test_header_declares_the_boundary():
    names = M.header_symbols()
    for required in ["mmf_ctx_create", "mmf_sys_create", "mmf_add_mode", "mmf_add_coupling",
                     "mmf_build", "mmf_diagonalise", "mmf_quasienergies", "mmf_eigenvectors",
                     "mmf_time_evolution", "mmf_transition_avg", "mmf_micromotion",
                     "mmf_time_evolution_operator", "mmf_batch_create", "mmf_batch_run",
                     "mmf_strerror"]:
        assert required in names
    assert set(names) == set(M._SIGS), "binding signatures must cover exactly the header"


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    for name in M.header_symbols():
        assert name in exported, name
        assert hasattr(lib, name)
    # internal kernels and helpers stay hidden
    assert not any(s.startswith("_Z") and "k_hetrd" in s for s in exported)


def test_strerror(lib):
    assert lib.mmf_strerror(0) == b"ok"
    assert b"budget" in lib.mmf_strerror(M.MMF_ERR_BUDGET)
    assert lib.mmf_strerror(12345) == b"unknown status"


def test_host_argument_checks(lib):
    h = ctypes.c_void_p()
    H0 = np.eye(2, dtype=np.complex128)
    assert lib.mmf_sys_create(None, 2, H0.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)) == M.MMF_ERR_ARG
    assert lib.mmf_ctx_create(0, 0, None, None) == M.MMF_ERR_ARG
    assert lib.mmf_dim(None) == -1
    assert lib.mmf_batch_size(None, 0) == -1
    assert lib.mmf_sys_destroy(None) == M.MMF_ERR_ARG


@pytest.mark.skipif(_has_gpu(), reason="checks the no-GPU failure mode")
def test_no_gpu_fails_loudly(lib):
    h = ctypes.c_void_p()
    rc = lib.mmf_ctx_create(0, 0, None, ctypes.byref(h))
    assert rc == M.MMF_ERR_CUDA
    assert lib.mmf_last_error()
    with pytest.raises(M.MmfError):
        M.Context(0)
