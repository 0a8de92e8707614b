"""Host-side helpers of the package's drivers and autograd wrapper that need no
GPU: unit conversion, the analytic erf solution of Sec. 4.1, the initial fields
of Secs. 4.2 and 4.3, and the packing of the D_ij pairs."""

import math

import numpy as np
import pytest

import theory as th


def test_lattice_units_put_the_largest_pair_at_d_max():
    from paper_1808_06787_gb300.scenarios import lattice_units

    pairs = {(1, 2): 0.833, (1, 3): 0.833, (2, 3): 0.168}
    dx = 1.0 / 200
    lat, dt = lattice_units(pairs, dx, d_max=0.1)
    assert max(lat.values()) == pytest.approx(0.1)
    assert dt == pytest.approx(0.1 * dx * dx / 0.833)
    for k, v in pairs.items():  # D_lattice = D dt / dx^2 for every pair
        assert lat[k] == pytest.approx(v * dt / dx ** 2)


def test_erf_solution_agrees_with_an_independent_form_and_solves_fick():
    from paper_1808_06787_gb300.scenarios import erf_solution

    X = np.linspace(-6, 6, 241)
    t, D, C0, C1 = 1.0, 0.05, 0.0, 1.0
    xi, J = erf_solution(X, t, D, C0, C1)
    xr, Jr = th.erf_solution(X, t, D, C0, C1)
    assert np.abs(xi - xr).max() <= 1e-15 and np.abs(J - Jr).max() <= 1e-15
    # J = -D d(xi)/dX (Fick) and d(xi)/dt = -dJ/dX, by central differences
    h = 1e-4
    xp, _ = erf_solution(X + h, t, D, C0, C1)
    xm, _ = erf_solution(X - h, t, D, C0, C1)
    assert np.abs(J + D * (xp - xm) / (2 * h)).max() <= 1e-8
    xt1, _ = erf_solution(X, t + h, D, C0, C1)
    xt0, _ = erf_solution(X, t - h, D, C0, C1)
    _, Jp = erf_solution(X + h, t, D, C0, C1)
    _, Jm = erf_solution(X - h, t, D, C0, C1)
    assert np.abs((xt1 - xt0) / (2 * h) + (Jp - Jm) / (2 * h)).max() <= 1e-7
    # far field: the two compositions
    assert xi[0] == pytest.approx(C0, abs=1e-12) and xi[-1] == pytest.approx(C1, abs=1e-12)


def test_relative_l2_is_the_error_norm_of_sec_4():
    from paper_1808_06787_gb300.scenarios import relative_l2

    a = np.array([3.0, 4.0])
    assert relative_l2(a, a) == 0.0
    assert relative_l2(a, np.zeros(2)) == pytest.approx(1.0)
    assert relative_l2(a, a * 1.1) == pytest.approx(0.1)


def test_duncan_toor_initial_field():
    from paper_1808_06787_gb300.scenarios import duncan_toor_initial

    nx, ny = 200, 4
    x = duncan_toor_initial(nx, ny)
    assert x.shape == (3, 1, ny, nx)
    assert np.abs(x.sum(axis=0) - 1.0).max() <= 1e-15
    X = (np.arange(nx) + 0.5) / nx
    # Sec. 4.2: xi_1 = 0.8 on the left quarter, a linear ramp to zero at x = 0.75,
    # zero beyond; xi_2 = 0.2 everywhere
    assert np.all(x[0, 0, :, X < 0.25] == 0.8)
    mid = (X >= 0.25) & (X < 0.75)
    assert np.allclose(x[0, 0, 0, mid], 1.6 * (0.75 - X[mid]))
    assert np.all(x[0, 0, :, X >= 0.75] == 0.0)
    assert np.all(x[1] == 0.2)
    assert np.all(x[:, :, 0, :] == x[:, :, -1, :])  # y-independent


def test_loschmidt_initial_field():
    from paper_1808_06787_gb300.scenarios import loschmidt_initial

    nx, ny = 6, 10
    x = loschmidt_initial(nx, ny)
    assert np.abs(x.sum(axis=0) - 1.0).max() <= 1e-15
    assert np.allclose(x[:, 0, : ny // 2, :], np.array([0.0, 0.509, 0.491])[:, None, None])
    assert np.allclose(x[:, 0, ny // 2:, :], np.array([0.515, 0.485, 0.0])[:, None, None])


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_pairs_pack_in_the_abi_order(n):
    from paper_1808_06787_gb300.autograd import n_from_pairs, pairs_to_matrix

    m = n * (n - 1) // 2
    assert n_from_pairs(m) == n
    vals = np.arange(1, m + 1, dtype=np.float64)
    D = pairs_to_matrix(vals, n)
    assert np.array_equal(D, D.T)
    # order (0,1), (0,2), .., (0,n-1), (1,2), .. as lbms_adjoint_reduce writes them
    k = 0
    for p in range(n):
        for q in range(p + 1, n):
            assert D[p, q] == vals[k]
            k += 1


def test_pair_count_must_be_triangular():
    from paper_1808_06787_gb300.autograd import n_from_pairs

    with pytest.raises(ValueError):
        n_from_pairs(4)
    assert math.comb(4, 2) == 6 and n_from_pairs(6) == 4
