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


@pytest.mark.parametrize("n", [1, 37, 64, 129, 300, 1323, 2049, 4100])
def test_gram_on_tensor_cores_is_fp64_accurate(n):
    """The mixed path's Gram product by exact integer slicing on the BF16 tensor cores against an
    FP64 reference: sizes below, at and across the 128 x 64 tiles, the K-chunking (2n > 1024)
    and entries spread over six orders of magnitude.  Bound: 2^-38 per entry for columns of
    norm <= sqrt(n)/2 (each slice pair is exact; only the truncation to 40 bits below each
    column's largest entry and the dropped slice pairs remain)."""
    err, ref = ctypes.c_double(0), ctypes.c_double(0)
    rc = M.lib().mmf_selftest_gram(n, ctypes.byref(err), ctypes.byref(ref))
    assert rc == 0, M.lib().mmf_last_error()
    assert ref.value > 0
    assert err.value <= 2.0 ** -40 * max(1.0, ref.value) * 4


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("shape", [(128, 128, 32), (300, 256, 640), (1323, 256, 2688), (200, 96, 2646),
                                   (1, 32, 5)])
def test_split_tf32_products(mode, shape):
    """The split-TF32 product (two TF32 pieces per FP32 operand, three products in one FP32
    accumulator) on operands with full FP32 mantissas, in the three output modes (store, subtract
    in place, TF32 pieces as the next product's operand), against FP64: within a few FP32 roundings
    per accumulated term of sum_k |a_k b_k|, as a sequential FP32 dot product is."""
    m, n, k = shape
    if mode == 2 and n % 32:
        pytest.skip("operand mode needs N a multiple of 32")
    err, err32 = ctypes.c_double(), ctypes.c_double()
    rc = M.lib().mmf_selftest_split_tf32(m, n, k, mode, ctypes.byref(err), ctypes.byref(err32))
    assert rc == 0, M.lib().mmf_last_error()
    print(f"split TF32 {shape} mode {mode}: {err.value:.3e} (sequential FP32 {err32.value:.3e})")
    assert err.value <= 2.0 ** -24 * (8 + k / 16.0)


@pytest.mark.parametrize("n,count", [(2, 1), (33, 3), (64, 2), (129, 2), (300, 2), (457, 1), (200, 90)])
def test_householder_reduction_trailing_update(n, count):
    """The FP32 Householder reduction with its trailing update (A -= V W^H + W V^H after each
    32-column panel) on the tensor cores in split TF32 and on the FP32 units: Q^H A Q rebuilt in
    FP64 from the stored reflectors equals tridiag(e, d, e) within FP32 backward error of the
    reduction.  Sizes: below one panel, one 64-column block, a ragged 128-row tile, several
    panels, and 90 systems (one CTA per system instead of two)."""
    errs = {}
    for tc in (0, 1):
        err, ref = ctypes.c_double(), ctypes.c_double()
        rc = M.lib().mmf_selftest_hetrd(n, count, tc, ctypes.byref(err), ctypes.byref(ref))
        assert rc == 0, M.lib().mmf_last_error()
        errs[tc] = err.value / ref.value
    print(f"n = {n} x {count}: |Q^H A Q - T| / |A| = {errs[0]:.3e} (FP32 units), {errs[1]:.3e} (tensor cores)")
    for tc in (0, 1):
        assert errs[tc] <= 2.0 ** -24 * 4 * n
    # the split-TF32 products carry a few units of FP32 rounding each, as the FP32 units' do
    assert errs[1] <= 4 * errs[0] + 2.0 ** -24 * 8
