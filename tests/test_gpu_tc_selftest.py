"""Tensor-core building block of the split-precision products: one bfloat16 tcgen05.mma
chain (canonical K-major layout without swizzle, FP32 accumulator in tensor memory)
against the float64 product on the host.

The split contractions rely on two facts checked here with in-bounds operands: the layout
the descriptors describe is the one the operands are written in (any other reading gives
a different product), and FP32 accumulation of integer products is exact while every
partial sum stays below 2^24.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(A, B, reps):
    """A (128 x 64) and B (64 x 64, row n = column n of the factor) hold bfloat16 values."""
    from paper_2311_18715_gb300._lib import check, load_library

    lib = load_library()
    dev = torch.device("cuda", 0)
    a = torch.from_numpy(A).to(dev, torch.bfloat16).contiguous()
    b = torch.from_numpy(B).to(dev, torch.bfloat16).contiguous()
    d = torch.full((128, 64), float("nan"), dtype=torch.float32, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    check(lib, lib.odmd_tc_selftest(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(d.data_ptr()),
                                    C.c_void_p(st.data_ptr()), reps))
    # the operands as the device saw them (bfloat16), in float64
    a64 = a.float().double().cpu().numpy()
    b64 = b.float().double().cpu().numpy()
    return d.double().cpu().numpy(), reps * (a64 @ b64.T)


def test_small_integer_product_exact():
    rng = np.random.default_rng(0)
    A = rng.integers(-8, 9, (128, 64)).astype(np.float32)
    B = rng.integers(-8, 9, (64, 64)).astype(np.float32)
    got, want = _run(A, B, 1)
    assert np.array_equal(got, want)


def test_layout_distinguishes_every_row_and_column():
    """A is the identity on its first 64 rows and B has distinct integers everywhere: a
    misplaced core matrix or row moves some entry of D."""
    A = np.zeros((128, 64), dtype=np.float32)
    A[:64, :64] = np.eye(64)
    A[64:, :] = np.eye(64)[::-1]
    B = (np.arange(64 * 64, dtype=np.float32).reshape(64, 64) % 251) - 125
    got, want = _run(A, B, 1)
    assert np.array_equal(got, want)


def test_integer_accumulation_exact_below_2_24():
    """Products of digits up to 128 summed over K = 64 and 15 repetitions: every partial sum
    is an integer below 2^24, so an FP32 accumulator must hold it exactly."""
    rng = np.random.default_rng(1)
    A = rng.integers(100, 129, (128, 64)).astype(np.float32)
    B = rng.integers(100, 129, (64, 64)).astype(np.float32)
    reps = 15
    got, want = _run(A, B, reps)
    assert want.max() < 2 ** 24
    assert np.array_equal(got, want)


def test_normal_operands_within_fp32_accumulation():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((64, 64)).astype(np.float32)
    got, want = _run(A, B, 3)
    bound = 3 * 64 * 2.0 ** -22 * np.abs(A).max() * np.abs(B).max()
    assert np.max(np.abs(got - want)) <= bound
