"""The resort step's radix sort (Sec. 2.3 re-binning; Sec. 3.3 resort) through
the C ABI: the permutation equals numpy's stable argsort bit for bit, for
ragged sizes, one to four digit passes, many equal keys and the cell keys of
an LJ box."""
import numpy as np
import pytest

import synth

le = pytest.importorskip("paper_2109_11083_gb300")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n, bits, distinct", [(1, 1, 2), (33, 5, 32), (4096, 9, 512),
                                               (4097, 18, 216000), (70001, 18, 7),
                                               (250000, 24, 1 << 24), (65536, 32, 1 << 32)])
def test_sort_equals_stable_argsort(n, bits, distinct):
    g = np.random.default_rng(n + bits)
    keys = g.integers(0, min(distinct, 1 << bits), size=n, dtype=np.uint64).astype(np.uint32)
    order, sk = le.le_sort_cell_keys(keys, bits)
    want = np.argsort(keys, kind="stable").astype(np.uint32)
    assert np.array_equal(order, want)
    assert np.array_equal(sk, keys[want])


def test_sort_of_cell_keys_of_an_lj_box():
    pos, box = synth.lj_box(20000, 0.8442, 3)
    nc = int(box // 2.8)
    c = np.minimum((pos / (box / nc)).astype(np.int64), nc - 1)
    keys = (c[:, 0] + nc * (c[:, 1] + nc * c[:, 2])).astype(np.uint32)
    bits = int(np.ceil(np.log2(nc ** 3)))
    order, _ = le.le_sort_cell_keys(keys, bits)
    assert np.array_equal(order, np.argsort(keys, kind="stable"))


def test_sort_rejects_keys_wider_than_bits():
    with pytest.raises(le.LEError) as e:
        le.le_sort_cell_keys(np.array([0, 8], dtype=np.uint32), 3)
    assert e.value.status == 1
