"""Host-side 2-bit genotype packing (SSNAL_EN_I2_GENO layout), no GPU."""
import numpy as np
import pytest

import paper_2006_03970_gb300 as pkg


@pytest.mark.parametrize("n,m", [(1, 1), (3, 63), (4, 64), (5, 65), (7, 300)])
def test_pack_layout_and_round_trip(n, m):
    rng = np.random.default_rng(n * m)
    codes = rng.integers(0, 3, size=(n, m)).astype(np.int8)
    pk = pkg.pack_codes_2bit(codes)
    lda = (m + 63) // 64 * 64
    assert pk.dtype == np.uint8 and pk.shape == (n, lda // 4)
    for j in range(n):
        for i in range(m):  # row i of column j: bits 2 (i mod 4) of byte i / 4
            assert (pk[j, i // 4] >> (2 * (i % 4))) & 3 == codes[j, i]
    unpacked = np.stack([(pk >> (2 * q)) & 3 for q in range(4)], axis=-1).reshape(n, lda)
    assert np.array_equal(unpacked[:, :m], codes) and not unpacked[:, m:].any()


def test_pack_rejects_codes_outside_two_bits():
    with pytest.raises(ValueError):
        pkg.pack_codes_2bit(np.array([[0, 4]]))
