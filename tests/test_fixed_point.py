"""Host-side check of the fixed-point rounding the FP32 mass partials use.

The kernels turn x * 2^shift (|x| <= 4, shift <= 40, so |v| <= 2^42) into a
64-bit integer with float additions instead of a 64-bit conversion: adding
1.5 * 2^45 rounds v to a multiple of 2^22 whose quotient is the difference of
bit patterns, the exact remainder is rounded by adding 1.5 * 2^23.  The same
steps are replayed here in IEEE float32 arithmetic (numpy rounds every float32
addition to nearest even, as the kernels' __fadd_rn does) and compared with
the exact round-half-to-even of v, ties included.
"""

import numpy as np

F = np.float32


def _bits(a):
    return np.asarray(a, dtype=np.float32).view(np.int32).astype(np.int64)


def round_to_ll(v):
    v = np.asarray(v, dtype=np.float32)
    c, d = F(1.5 * 2.0 ** 45), F(1.5 * 2.0 ** 23)
    s = (v + c).astype(np.float32)
    k = _bits(s) - _bits(c)
    r = (v - (s - c).astype(np.float32)).astype(np.float32)
    j = _bits((r + d).astype(np.float32)) - _bits(d)
    return k * (1 << 22) + j


def exact_rne(v):
    return np.rint(np.asarray(v, dtype=np.float32).astype(np.float64)).astype(np.int64)


def test_random_values_over_the_whole_range():
    g = np.random.default_rng(7)
    e = g.uniform(-30.0, 42.0, 400000)
    v = (np.sign(g.uniform(-1, 1, e.size)) * 2.0 ** e).astype(np.float32)
    v = v[np.abs(v.astype(np.float64)) <= 2.0 ** 42]
    assert np.array_equal(round_to_ll(v), exact_rne(v))


def test_ties_and_edges():
    vals = []
    for m in range(0, 24):
        base = 2.0 ** m
        for off in (-1.5, -0.5, 0.5, 1.5, 2.5):
            vals += [base + off, -(base + off)]
    vals += [0.0, -0.0, 2.0 ** 42, -(2.0 ** 42), 2.0 ** 21, 2.0 ** 21 + 0.5, 2.0 ** 22 - 0.5,
             3.0 * 2.0 ** 21, 2.0 ** 41 + 2.0 ** 21, -(2.0 ** 41 + 2.0 ** 21), 4194303.5]
    v = np.array(vals, dtype=np.float32)
    v = v[v.astype(np.float64) == np.array(vals)]  # keep the exactly representable ones
    assert np.array_equal(round_to_ll(v), exact_rne(v))


def test_scaled_mole_fractions():
    # the kernels' inputs: x in [-4, 4] times 2^shift for every shift they use
    g = np.random.default_rng(11)
    x = g.uniform(-4.0, 4.0, 50000).astype(np.float32)
    for shift in range(8, 41):
        v = (x * F(2.0 ** shift)).astype(np.float32)
        assert np.array_equal(round_to_ll(v), exact_rne(v)), shift
