"""Host-side checks that need no GPU: the C-ABI library loads, exports every
entry point that include/le.h declares, and rejects bad arguments before any
device work."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            names += re.findall(r"LE_API\s+[\w\s\*]+?\b(le_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2109_11083_gb300 as le
    return le


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("le_create", "le_set_particles", "le_step", "le_forces", "le_stress",
                 "le_velocity_profile", "le_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing
    assert set(lib.exported_symbols()) <= set(declared_symbols())


def test_argument_checks_reject_bad_boxes_without_a_gpu(lib):
    p = lib.le_default_params()
    assert p.dt == 0.005 and p.profile_bins == 20 and p.fene_k == 30.0
    with pytest.raises(lib.LEError) as e:
        lib.le_create([5.0, 5.0, 5.0], 0.1, 2.5, 0.3, p)     # rc + skin >= L/2
    assert e.value.status == 4
    with pytest.raises(lib.LEError) as e:
        lib.le_create([10.0, 10.0, -1.0], 0.1, 2.5, 0.3, p)
    assert e.value.status == 1
    p.profile_bins = 0
    with pytest.raises(lib.LEError) as e:
        lib.le_create([10.0, 10.0, 10.0], 0.1, 2.5, 0.3, p)
    assert e.value.status == 1


def test_degenerate_sizes_are_refused_on_the_host(lib):
    """No particles, more than the 2^24 that a list entry can index, and a sort
    key wider than its stated bit count are argument errors, found before any
    device work; the largest indexable system is accepted."""
    p = lib.le_default_params()
    box = [20.0, 20.0, 20.0]
    for n in (0, -5, (1 << 24) + 1):
        with pytest.raises(lib.LEError) as e:
            lib.le_estimate_device_bytes(box, 0.1, 2.5, 0.3, p, n)
        assert e.value.status == 1
    small = lib.le_estimate_device_bytes(box, 0.1, 2.5, 0.3, p, 1000)
    largest = lib.le_estimate_device_bytes([270.0] * 3, 0.1, 2.5, 0.3, p, 1 << 24)
    assert 0 < small < largest
    with pytest.raises(lib.LEError) as e:
        lib.le_sort_cell_keys(np.zeros(0, np.uint32), 8)
    assert e.value.status == 1
    with pytest.raises(lib.LEError) as e:
        lib.le_sort_cell_keys(np.array([3, 300], np.uint32), 8)   # 300 needs 9 bits
    assert e.value.status == 1


def test_slot_encoding_gives_distinct_codes_below_the_end_marker():
    """The neighbour-slot code is four bit fields (x-cell offset -3..4 in 3
    bits, y and z offsets -1..1 in 2 bits each, across-the-face flag in 1
    bit): 144 distinct 8-bit codes, all below the 255 end-of-bonds marker and
    leaving 24 bits for the particle index."""
    seen = set()
    for cross in (0, 1):
        for dcz in (-1, 0, 1):
            for dcy in (-1, 0, 1):
                for k in range(-3, 5):
                    s = (k + 3) | ((dcy + 1) << 3) | ((dcz + 1) << 5) | (cross << 7)
                    assert 0 <= s < 255
                    seen.add(s)
    assert len(seen) == 144


def test_fp32_peak_rejects_missing_outputs_without_a_gpu(lib):
    """The FMA-peak measurement aid checks its arguments before any device work."""
    assert lib.lib().le_fp32_peak(None, None) == 1
