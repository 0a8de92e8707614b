"""Host-side checks of facts the CUDA per-node arithmetic relies on.

The kernels form Lambda_1 = K^{-1} B with K = I/c_s^2 + B/2 by Gauss-Jordan
elimination without pivoting.  That is safe if every pivot of K is bounded
away from zero; here the pivots are checked to be at least 1/c_s^2 for random
compositions (with vanishing species) and diffusivities over four decades,
using the oracle's B of Eq. 2-10.  The second test checks that the unpivoted
K^{-1} B equals the oracle's Lambda_1 of Eq. 3-26.
"""

import numpy as np
import pytest

import synthetic as sy

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _random_case(g, trial):
    n = int(g.integers(2, 9))
    lo, hi = (0.01, 0.12) if trial % 2 else (0.001, 10.0)
    D = np.ones((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            D[i, j] = D[j, i] = float(np.exp(g.uniform(np.log(lo), np.log(hi))))
    xi = g.uniform(0.0, 1.0, n)
    if trial % 3 == 0:
        xi[g.integers(0, n, size=int(g.integers(1, n)))] = 0.0
    if xi.sum() == 0.0:
        xi[0] = 1.0
    return xi / xi.sum(), D


def _unpivoted_pivots(K):
    A = K.copy()
    S = A.shape[0]
    piv = []
    for p in range(S):
        piv.append(A[p, p])
        for r in range(p + 1, S):
            A[r] -= A[r, p] / A[p, p] * A[p]
    return np.array(piv)


def test_unpivoted_pivots_bounded_below():
    import oracle

    g = sy.rng(2024)
    for trial in range(3000):
        xi, D = _random_case(g, trial)
        B = oracle.B_matrix(xi, D)
        for cs2 in (1.0 / 3.0, 0.25):
            K = np.eye(B.shape[0]) / cs2 + 0.5 * B
            assert _unpivoted_pivots(K).min() * cs2 >= 1.0 - 1e-12


def test_unpivoted_solve_equals_lambda1():
    import oracle

    g = sy.rng(7)
    for trial in range(300):
        xi, D = _random_case(g, trial)
        B = oracle.B_matrix(xi, D)
        lat = ("D2Q5", "D2Q9", "D3Q7")[trial % 3]
        cs2 = 0.25 if lat == "D3Q7" else 1.0 / 3.0
        S = B.shape[0]
        K = np.eye(S) / cs2 + 0.5 * B
        R = B.copy()
        A = K.copy()
        for p in range(S):  # Gauss-Jordan on [K | B] without row exchanges
            inv = 1.0 / A[p, p]
            A[p] *= inv
            R[p] *= inv
            for r in range(S):
                if r != p:
                    fac = A[r, p]
                    A[r] -= fac * A[p]
                    R[r] -= fac * R[p]
        if np.linalg.cond(B) > 1e12:
            continue
        L1, _ = oracle.lambdas(lat, xi, D)
        np.testing.assert_allclose(R, L1, rtol=1e-9, atol=1e-11)
