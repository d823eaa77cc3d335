"""Host-side checks of the shared-memory layout of the small-grid kernel
(gs_small.cuh), restated here from its definition: element (y, x) of the
field at y nx + (x ^ rev4(y)), rev4 reversing the low four bits of y.

* The map is a permutation of [0, nx ny) that keeps every row in place, so
  a row pass and a column pass address every element exactly once.
* Within a half-warp (16 lanes, 8-byte accesses) the row accesses (T_x lanes
  per row on consecutive rows) and the column accesses (T_y consecutive rows
  per column, consecutive columns) fall on 16 distinct 8-byte banks, for
  every shape the kernel is built for.
"""

import pytest

SMALL_MAX_PIXELS = 8192
SHAPES = [(lx, ly) for lx in range(5, 9) for ly in range(5, 9) if (1 << (lx + ly)) <= SMALL_MAX_PIXELS]


def rev4(y):
    return int(f"{y & 15:04b}"[::-1], 2)


def fo(nx, y, x):
    return y * nx + (x ^ rev4(y))


def test_the_shapes_are_the_instantiated_ones():
    assert sorted(SHAPES) == sorted([(5, 5), (5, 6), (5, 7), (5, 8), (6, 5), (6, 6), (6, 7), (7, 5), (7, 6),
                                     (8, 5)])


@pytest.mark.parametrize("lx,ly", SHAPES)
def test_layout_is_a_row_preserving_permutation(lx, ly):
    nx, ny = 1 << lx, 1 << ly
    seen = set()
    for y in range(ny):
        row = {fo(nx, y, x) for x in range(nx)}
        assert row == set(range(y * nx, (y + 1) * nx))
        seen |= row
    assert len(seen) == nx * ny


def _lanes(T):
    """(group, thread-in-group) of the 16 lanes of each half-warp."""
    for half in range(2):
        yield [((16 * half + l) // T, (16 * half + l) % T) for l in range(16)]


@pytest.mark.parametrize("lx,ly", SHAPES)
def test_row_and_column_accesses_are_bank_conflict_free(lx, ly):
    nx, ny = 1 << lx, 1 << ly
    tx, ty = nx >> 5, ny >> 5
    nt = min(256, nx * ny // 32)
    for warp in range(nt // 32):
        for lanes in _lanes(tx):  # row pass: group g owns row l0 + g, lane t reads x = t + T i
            for i in range(32):
                banks = [fo(nx, warp * (32 // tx) + g, t + tx * i) % 16 for g, t in lanes]
                assert len(set(banks)) == 16, ("row", lx, ly, warp, i)
        for lanes in _lanes(ty):  # column pass: group g owns column g, lane t reads y = t + T i
            for i in range(32):
                banks = [fo(nx, t + ty * i, warp * (32 // ty) + g) % 16 for g, t in lanes]
                assert len(set(banks)) == 16, ("column", lx, ly, warp, i)


def test_rev4_is_the_bit_reversal_of_the_low_four_bits():
    for y in range(64):
        assert rev4(y) == rev4(y % 16) < 16
    assert [rev4(y) for y in range(16)] == [0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15]
