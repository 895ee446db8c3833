"""The library's radix sort (the Morton-order sort before every tree build,
Sect. 4.2, and the pair sorts of the collision queue, Sect. 5) against
numpy's stable sort, element by element: ragged sizes around the 2048-key
tile, more tiles than resident blocks (several tiles per block), a device
count below the buffer capacity, heavy duplicates (stability), nearly sorted,
reversed and constant inputs, and the top key bit."""
import numpy as np
import pytest

from paper_1110_4876_gb300 import rb

pytestmark = pytest.mark.gpu


def _check(keys, key_bits, cap=None, with_vals=True):
    vals = np.arange(len(keys), dtype=np.uint32)[::-1].copy() if with_vals else None
    k, v = rb.rb_sort_pairs_u64(keys, vals, key_bits=key_bits, cap=cap)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(k, keys[order])
    if with_vals:
        np.testing.assert_array_equal(v, vals[order])


@pytest.mark.parametrize("n", [1, 2, 31, 2047, 2048, 2049, 100_003])
def test_ragged_sizes_with_duplicates(n):
    rng = np.random.default_rng(n)
    # few distinct high parts: long runs of equal digits in the top passes
    keys = (rng.integers(0, 7, n, dtype=np.uint64) << np.uint64(40)) | \
           rng.integers(0, 1 << 20, n, dtype=np.uint64)
    _check(keys, 43)


def test_more_tiles_than_resident_blocks():
    """3M keys are 1465 tiles: more than one wave of resident blocks, so
    blocks take several tiles and look back across them."""
    rng = np.random.default_rng(7)
    keys = rng.integers(0, 1 << 63, 3_000_000, dtype=np.uint64)
    keys[::3] = keys[1::3][: len(keys[::3])]   # duplicates: stability matters
    _check(keys, 64)


@pytest.mark.parametrize("cap_extra", [1, 5000, 400_000])
def test_count_below_capacity(cap_extra):
    """The count is read on the device (as in the pair sorts), the buffers
    and the grid are sized for cap."""
    rng = np.random.default_rng(cap_extra)
    keys = rng.integers(0, 1 << 24, 250_001, dtype=np.uint64)
    _check(keys, 24, cap=250_001 + cap_extra)


def test_nearly_sorted_reversed_and_constant():
    rng = np.random.default_rng(3)
    base = np.sort(rng.integers(0, 1 << 62, 500_000, dtype=np.uint64))
    swap = rng.integers(0, len(base) - 1, 5000)
    near = base.copy()
    near[swap], near[swap + 1] = base[swap + 1], base[swap]   # a step's worth of drift
    _check(near, 64)
    _check(base[::-1].copy(), 64)
    _check(np.full(300_000, 0x0123456789abcdef, dtype=np.uint64), 64)


def test_top_bit_and_keys_only():
    rng = np.random.default_rng(11)
    keys = rng.integers(0, 1 << 62, 70_000, dtype=np.uint64)
    keys[::2] |= np.uint64(1) << np.uint64(63)
    _check(keys, 64, with_vals=False)
