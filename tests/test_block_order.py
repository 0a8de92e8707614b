"""Host replay of the block order of the reverse steps.

Odd-parity steps of undivided grids take the grid's blocks in chunks of 64
from its end, each chunk in order (`grid_block` in the kernels).  The formula is
replayed here for grid sizes around the chunk size and at the bench sizes: it
must be a permutation of the blocks, ascending within every chunk, and start
on the grid's last chunk."""

import numpy as np
import pytest

K = 64


def grid_block(b, nb):
    c = b // K
    w = b - c * K
    hi = nb - c * K
    return np.where(hi > K, hi - K, 0) + w


@pytest.mark.parametrize("nb", [1, 2, 63, 64, 65, 127, 128, 129, 1000, 65536, 65537, 405126])
def test_reverse_order_is_a_permutation(nb):
    b = np.arange(nb, dtype=np.int64)
    lb = grid_block(b, nb)
    assert np.array_equal(np.sort(lb), b)
    # the first blocks taken are the grid's last ones, in ascending order
    first = lb[: min(K, nb)]
    assert first[-1] == nb - 1 and np.all(np.diff(first) == 1)
    # within each chunk the taken blocks ascend by one
    for c in range(0, nb, K):
        chunk = lb[c: c + K]
        assert np.all(np.diff(chunk) == 1)
