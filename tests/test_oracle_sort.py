"""Oracle pins of the cell sort (Alg. 1 / Alg. 2's particles-by-cell order):
brute force on small inputs -- the stable order by insertion, the offsets
by counting -- and the out-of-range rule."""

import numpy as np

import oracle as O


def _insertion_order(key):
    """Stable order by straight insertion: an element moves left only past
    strictly larger keys."""
    order = []
    for i in range(len(key)):
        j = len(order)
        while j > 0 and key[order[j - 1]] > key[i]:
            j -= 1
        order.insert(j, i)
    return order


def test_small_inputs_against_insertion_sort_and_counting():
    rng = np.random.default_rng(0)
    for trial in range(40):
        n_cells = int(rng.integers(1, 9))
        n = int(rng.integers(0, 60))
        cell_of = rng.integers(-2, n_cells + 2, size=n)
        perm, off = O.sort_by_cell(cell_of, n_cells)
        key = [c if 0 <= c < n_cells else n_cells for c in cell_of]
        assert list(perm) == _insertion_order(key)
        for c in range(n_cells + 1):
            assert off[c] == sum(1 for k in key if k < c)


def test_empty_cells_and_all_outside():
    perm, off = O.sort_by_cell(np.array([3, 3, 0]), 5)
    assert list(perm) == [2, 0, 1] and list(off) == [0, 1, 1, 1, 3, 3]
    perm, off = O.sort_by_cell(np.array([-1, 7, 5]), 5)
    assert list(perm) == [0, 1, 2] and list(off) == [0] * 6
    perm, off = O.sort_by_cell(np.array([], dtype=np.int64), 3)
    assert perm.size == 0 and list(off) == [0, 0, 0, 0]
