"""Scratch sizes of the two in-place orientations (host arithmetic, no GPU):
row bands (Sec. 3.2) take two bands of max(o, 256) rows of packed bits;
column bands (the exchanged axes of Sec. 3.3) take one band of H rows whose
width is the smallest multiple of 256 columns with 7 B / 8 >= l - 1, i.e.
the first band's packed bytes end left of where the second band's windows
begin."""
import pytest


@pytest.fixture(scope="module")
def lib():
    import paper_1905_13038_gb300 as bz
    bz.build()
    return bz._load()


def test_row_band_scratch(lib):
    assert lib.bz_inplace_scratch_bytes(4096, 3072, 15, 0) == 2 * 256 * 384
    assert lib.bz_inplace_scratch_bytes(4096, 3072, 511, 0) == 2 * 256 * 384  # o = 256
    assert lib.bz_inplace_scratch_bytes(100, 3072, 15, 0) == 2 * 100 * 384    # one band of H rows
    assert lib.bz_inplace_scratch_bytes(4096, 3071, 15, 8) == 2 * 8 * 384
    assert lib.bz_inplace_scratch_bytes(4096, 3072, 17, 8) == -1              # o = 9 > 8


def test_column_band_width_follows_the_window(lib):
    # l = ceil(w / 2); 256-column bands hold while l - 1 <= 224
    for w, B in [(1, 256), (31, 256), (449, 256), (450, 256), (451, 512), (511, 512)]:
        l = (w + 1) // 2
        assert (7 * B // 8 >= l - 1) and (B == 256 or 7 * 256 // 8 < l - 1)
        assert lib.bz_inplace_cols_scratch_bytes(4096, 3072, w, 0) == 4096 * B // 8, w
    assert lib.bz_inplace_cols_scratch_bytes(4096, 3072, 31, 768) == 4096 * 96
    assert lib.bz_inplace_cols_scratch_bytes(4096, 3072, 451, 256) == -1   # too narrow for l = 226
    assert lib.bz_inplace_cols_scratch_bytes(4096, 3072, 31, 300) == -1    # not a multiple of 256
    assert lib.bz_inplace_cols_scratch_bytes(4096, 100, 31, 0) == 4096 * 13  # one band narrower than 256
    assert lib.bz_inplace_cols_scratch_bytes(4096, 3072, 512, 0) == -1


def test_orientation_with_the_smaller_scratch(lib):
    """Theta(min{H, W}) (Sec. 3.3): column bands take less scratch on pages
    less than about twice as tall as wide, row bands on taller ones."""
    for H, W, cols_smaller in [(4096, 3072, True), (3072, 4096, True), (8192, 3072, False),
                               (512, 65536, True), (65536, 512, False)]:
        r = lib.bz_inplace_scratch_bytes(H, W, 31, 0)
        c = lib.bz_inplace_cols_scratch_bytes(H, W, 31, 0)
        assert (c < r) == cols_smaller, (H, W, r, c)
