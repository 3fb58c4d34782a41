"""Host-side helpers of bench.py: the oracle baseline's crops and the L2 statement of a
workload line (no GPU)."""
import numpy as np

import bench


def test_crops_are_disjoint_cubes_of_a_large_field():
    sp = np.arange(128 ** 3, dtype=np.int64).reshape(128, 128, 128)
    parts = bench.crops(sp, 16)
    assert len(parts) == 8   # the 128^3 field holds eight disjoint 64^3 crops
    seen = set()
    for c in parts:
        assert c.shape == (bench.CROP,) * 3
        ids = set(c.ravel().tolist())
        assert not ids & seen
        seen |= ids


def test_small_field_is_taken_whole_once_per_process():
    sp = np.arange(32 ** 3, dtype=np.int64).reshape(32, 32, 32)
    parts = bench.crops(sp, 5)
    assert len(parts) == 5
    for c in parts:
        assert np.array_equal(c, sp)
    assert "independent runs of the whole 32x32x32 field" in bench.crop_desc(sp, 5, 5 * sp.size)
    big = np.zeros((128, 128, 128), dtype=np.uint16)
    assert "disjoint 64^3 crops" in bench.crop_desc(big, 8, 8 * 64 ** 3)


def test_l2_statement_follows_the_resident_bytes():
    assert bench.l2_statement(256 ** 3).startswith("inputs larger than L2")
    assert bench.l2_statement(128 ** 3).startswith("inputs smaller than L2")
    assert bench.l2_statement(32 ** 3).startswith("inputs smaller than L2")
    # the threshold sits where the resident bytes reach the L2 size
    n = int(bench.L2_BYTES / bench.RESIDENT_BYTES_PER_SITE)
    assert bench.l2_statement(n - 1000).startswith("inputs smaller")
    assert bench.l2_statement(n + 1000).startswith("inputs larger")
