"""The tcgen05 GEMM engine against an FP64 reference (exact products, so only the FP32
accumulation order differs): full tiles, ragged edges, several K chunks, one to three products
in one accumulator, TF32 and BF16."""

import ctypes

import pytest

from paper_2005_03426_gb300 import mmf as M

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("shape", [(128, 128, 32), (128, 128, 256), (200, 300, 100), (1, 129, 7),
                                   (513, 257, 1030)])
@pytest.mark.parametrize("products", [1, 3])
def test_tensor_core_gemm(kind, shape, products):
    m, n, k = shape
    err, ref = ctypes.c_double(), ctypes.c_double()
    rc = M.lib().mmf_selftest_tensor_cores(m, n, k, kind, products, ctypes.byref(err), ctypes.byref(ref))
    assert rc == 0, M.lib().mmf_last_error()
    assert ref.value > 0
    # exact products, FP32 accumulation: error grows with the number of accumulated terms
    assert err.value <= 1e-5 * ref.value * max(1.0, k * products / 256.0), (err.value, ref.value)
