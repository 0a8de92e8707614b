"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
printed in the paper (Remarks I-IV of Sec. 2, the D12 = D13 form of Sec. 4.2,
the moment matrix and equilibrium moments of Sec. 3), exact Fourier
amplification of the linear cases built in the two-relaxation-time pair form
(Sec. 3.1 states the MRT/TRT equivalence), the Chapman-Enskog continuum limit
(Eq. 3-26, second-order convergence), conservation laws, the mirror symmetry
of half-way bounce-back, and the numbers printed for the Duncan-Toor-like and
Loschmidt-tube problems (Secs. 4.2 and 4.3).
"""

import math

import numpy as np
import pytest
from scipy.linalg import expm

import synthetic as sy
import theory as th

pytestmark = pytest.mark.usefixtures("oracle_lib")

LATTICES = ["D2Q5", "D2Q9", "D3Q7", "D3Q15", "D1Q3", "D2Q4", "D3Q6"]


def _oracle():
    import oracle

    return oracle


def _rand_xi(g, n):
    x = g.uniform(0.05, 1.0, size=n)
    return x / x.sum()


# --------------------------------------------------------------------------
# Lattice tables and the moment matrix (Sec. 3.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat", LATTICES)
def test_lattice_tables_match_printed(lat):
    o = _oracle()
    Q, dim, c, w, opp, cs2 = o.lattice_info(lat)
    gc, gw = th.golden_lattice(lat)
    assert Q == gc.shape[0]
    np.testing.assert_array_equal(c, gc)
    np.testing.assert_allclose(w, gw, rtol=0, atol=1e-16)
    np.testing.assert_array_equal(opp, th.opposite(gc))
    assert abs(w.sum() - 1.0) < 1e-15


def test_d2q5_moment_matrix_and_equilibrium_moments():
    """M_0 of Eq. 3-14a and m^(0) = xi (1, 0, 0, 0, -2/3) of Sec. 3.2."""
    o = _oracle()
    M, Mi, group = o.moment_basis("D2Q5")
    M0, m0 = th.golden_M0()
    np.testing.assert_array_equal(M, M0)
    np.testing.assert_allclose(Mi @ M0, np.eye(5), atol=1e-15)
    _, w = th.golden_lattice("D2Q5")
    np.testing.assert_allclose(M @ w, m0, atol=1e-15)
    # first-order rows relax with lambda_1, second-order rows with lambda_2 (Eq. 3-14b)
    assert list(group) == [0, 1, 1, 2, 2]


@pytest.mark.parametrize("lat", LATTICES)
def test_moment_basis_groups_odd_even(lat):
    """Odd rows span the antisymmetric pair space, even rows the symmetric one."""
    o = _oracle()
    M, Mi, group = o.moment_basis(lat)
    c, _ = th.golden_lattice(lat)
    opp = th.opposite(c)
    for a in range(M.shape[0]):
        refl = M[a, opp]
        if group[a] == 1:
            np.testing.assert_allclose(refl, -M[a], atol=0)
        else:
            np.testing.assert_allclose(refl, M[a], atol=0)
    np.testing.assert_array_equal(M[0], np.ones(M.shape[1]))
    np.testing.assert_allclose(M @ Mi, np.eye(M.shape[0]), atol=1e-14)


# --------------------------------------------------------------------------
# Maxwell-Stefan matrices (Sec. 2, Remarks I-IV; Sec. 4.2)
# --------------------------------------------------------------------------

def test_remark_IV_ternary_B_det_and_Dtilde():
    o = _oracle()
    g = sy.rng(7)
    for _ in range(50):
        xi = _rand_xi(g, 3)
        D12, D13, D23 = g.uniform(0.01, 1.0, size=3)
        D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D13, (2, 3): D23})
        x1, x2, x3 = xi
        B_ref = np.array([
            [1 / D13 + x2 * (1 / D12 - 1 / D13), x1 * (1 / D13 - 1 / D12)],
            [x2 * (1 / D23 - 1 / D12), 1 / D23 + x1 * (1 / D12 - 1 / D23)],
        ])
        B = o.B_matrix(xi, D)
        np.testing.assert_allclose(B, B_ref, rtol=1e-13, atol=1e-13)
        det = x1 / (D12 * D13) + x2 / (D12 * D23) + x3 / (D13 * D23)
        assert det > 0
        assert abs(np.linalg.det(B) - det) <= 1e-11 * det
        Dt = o.Dtilde(xi, D)
        Dt1 = np.array([
            [1 / D23 + x1 * (1 / D12 - 1 / D23), x1 * (1 / D12 - 1 / D13)],
            [x2 * (1 / D12 - 1 / D23), 1 / D13 + x2 * (1 / D12 - 1 / D13)],
        ]) / det
        np.testing.assert_allclose(Dt, Dt1, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(Dt, th.ternary_Dtilde_closed(xi, D12, D13, D23),
                                   rtol=1e-11, atol=1e-13)


def test_remark_I_binary_is_fick():
    o = _oracle()
    for x1 in (0.0, 0.3, 0.9, 1.0):
        D = sy.D_from_pairs(2, {(1, 2): 0.37})
        B = o.B_matrix([x1, 1 - x1], D)
        np.testing.assert_allclose(B, [[1 / 0.37]], rtol=1e-15)
        np.testing.assert_allclose(o.Dtilde([x1, 1 - x1], D), [[0.37]], rtol=1e-15)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_remark_II_equal_diffusivities(n):
    o = _oracle()
    g = sy.rng(11)
    D = np.full((n, n), 0.21)
    for _ in range(10):
        xi = _rand_xi(g, n)
        np.testing.assert_allclose(o.B_matrix(xi, D), np.eye(n - 1) / 0.21, rtol=1e-14,
                                   atol=1e-13)
        np.testing.assert_allclose(o.Dtilde(xi, D), 0.21 * np.eye(n - 1), rtol=1e-13,
                                   atol=1e-14)


@pytest.mark.parametrize("n", [3, 4, 6])
def test_remark_III_dilute_species(n):
    """xi_i = 0: row i of B is diagonal and D~_ii = D_eff of Eq. 2-17."""
    o = _oracle()
    g = sy.rng(13)
    D = sy.random_D(n, lo=0.02, hi=0.9, seed=17)
    for i in range(n - 1):
        xi = _rand_xi(g, n)
        xi[i] = 0.0
        xi /= xi.sum()
        B = o.B_matrix(xi, D)
        Deff = 1.0 / sum(xi[k] / D[i, k] for k in range(n) if k != i)
        for j in range(n - 1):
            if j != i:
                assert B[i, j] == 0.0
        assert abs(B[i, i] - 1.0 / Deff) <= 1e-13 / Deff
        Dt = o.Dtilde(xi, D)
        row = np.zeros(n - 1)
        row[i] = Deff
        np.testing.assert_allclose(Dt[i], row, rtol=1e-12, atol=1e-14)


def test_special_form_D12_equals_D13():
    """The D12 = D13 form of D~ used for the Sec. 4.2 problem."""
    o = _oracle()
    g = sy.rng(19)
    D12, D23 = 0.833, 0.168
    D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D12, (2, 3): D23})
    for _ in range(20):
        xi = _rand_xi(g, 3)
        beta = 1.0 / (1.0 / D23 + xi[0] * (1.0 / D12 - 1.0 / D23))
        ref = np.array([[D12, 0.0], [beta * xi[1] * (1.0 - D12 / D23), beta]])
        np.testing.assert_allclose(o.Dtilde(xi, D), ref, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------------------
# Relaxation matrices (Eq. 3-26, Eq. 3-16)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("n", [2, 3, 5])
def test_lambda2_magic_product_and_srt(lat, n):
    """Eq. 3-16 makes (1/l1 - 1/2)(1/l2 - 1/2) = 3/16 on the diagonal."""
    o = _oracle()
    g = sy.rng(23)
    D = sy.random_D(n, seed=29)
    for _ in range(10):
        xi = _rand_xi(g, n)
        L1, L2 = o.lambdas(lat, xi, D, "magic")
        for i in range(n - 1):
            prod = (1 / L1[i, i] - 0.5) * (1 / L2[i, i] - 0.5)
            assert abs(prod - 3.0 / 16.0) < 1e-12
            for j in range(n - 1):
                if i != j:
                    assert L2[i, j] == L1[i, j]
        S1, S2 = o.lambdas(lat, xi, D, "srt")
        np.testing.assert_array_equal(S1, L1)
        np.testing.assert_array_equal(S2, S1)
        # stability: eigenvalues of Lambda_1 inside (0, 2)
        ev = np.linalg.eigvals(L1)
        assert np.all(ev.real > 0) and np.all(ev.real < 2)


@pytest.mark.parametrize("lat", LATTICES)
def test_lambda1_ternary_matches_closed_form_Dtilde(lat):
    o = _oracle()
    _c, _w = th.golden_lattice(lat)
    cs2 = th.cs2_of(_c, _w)
    g = sy.rng(31)
    for _ in range(10):
        xi = _rand_xi(g, 3)
        D12, D13, D23 = g.uniform(0.01, 0.12, size=3)
        D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D13, (2, 3): D23})
        L1, _ = o.lambdas(lat, xi, D)
        ref = th.lambda1_from_Dtilde(th.ternary_Dtilde_closed(xi, D12, D13, D23), cs2)
        np.testing.assert_allclose(L1, ref, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("lat", LATTICES)
@pytest.mark.parametrize("relax", ["magic", "srt"])
def test_collision_equals_pair_form(lat, relax):
    """M^{-1} Lambda M of Eq. 3-2 equals the odd/even pair form (Sec. 3.1)."""
    o = _oracle()
    c, w = th.golden_lattice(lat)
    g = sy.rng(37)
    for n in (2, 3, 5):
        D = sy.random_D(n, seed=41 + n)
        S = n - 1
        for _ in range(5):
            xi = _rand_xi(g, n)
            fs = np.outer(xi[:S], w) + 0.01 * g.standard_normal((S, w.size))
            xs = fs.sum(axis=1)
            xin = np.append(xs, 1.0 - xs.sum())
            L1, L2 = o.lambdas(lat, xin, D, relax)
            Om = th.collision_operator(c, L1, L2)
            W = th.equilibrium_map(w, S)
            f = fs.reshape(-1)
            ref = f - Om @ (f - W @ f)
            got = o.collide_node(lat, D, fs, relax).reshape(-1)
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)
            # the collision conserves each species' mole fraction (Eq. 3-15)
            np.testing.assert_allclose(got.reshape(S, -1).sum(axis=1), xs, atol=2e-16 * w.size)


# --------------------------------------------------------------------------
# Whole scheme: exact linear cases (Fourier amplification)
# --------------------------------------------------------------------------

CASES = [
    ("D2Q5", (24, 1, 1), (2, 0, 0)),
    ("D2Q5", (12, 10, 1), (1, 2, 0)),
    ("D2Q9", (16, 12, 1), (1, 1, 0)),
    ("D2Q9", (20, 1, 1), (3, 0, 0)),
    ("D3Q7", (8, 6, 5), (1, 1, 2)),
    ("D3Q15", (6, 5, 4), (1, 2, 1)),
    ("D3Q15", (9, 1, 1), (2, 0, 0)),
    ("D1Q3", (24, 1, 1), (3, 0, 0)),
    ("D2Q4", (14, 10, 1), (1, 2, 0)),
    ("D3Q6", (7, 6, 5), (1, 1, 1)),
]


@pytest.mark.parametrize("lat,dims,k", CASES)
@pytest.mark.parametrize("relax", ["magic", "srt"])
def test_binary_mode_exact(lat, dims, k, relax):
    """N = 2 is linear (B = 1/D): the oracle equals G(theta)^t exactly."""
    o = _oracle()
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    c, w = th.golden_lattice(lat)
    cs2 = th.cs2_of(c, w)
    Dv = 0.07
    D = sy.D_from_pairs(2, {(1, 2): Dv})
    eps = 0.1
    x0 = sy.small_mode([0.5, 0.5], [1.0, -1.0], eps, nx, ny, nz, k=k)
    steps = 60
    x, J = o.run(lat, D, x0, steps, flux=True)
    theta = th.theta_of(k, shape)
    l1 = 1.0 / (Dv / cs2 + 0.5)
    L1 = np.array([[l1]])
    L2 = th.magic_lambda2(L1) if relax == "magic" else L1.copy()
    if relax == "srt":
        x, J = o.run(lat, D, x0, steps, flux=True, relax="srt")
    xi_hat, m1_hat = th.predict_mode(c, w, L1, L2, theta, [eps], steps)
    pred = 0.5 + th.mode_field(xi_hat[0], theta, shape)
    np.testing.assert_allclose(x[0], pred, rtol=0, atol=2e-14)
    np.testing.assert_allclose(x[1], 1.0 - pred, rtol=0, atol=2e-14)
    # flux of the pre-collision state: J = (1 - l1/2) m_1 (equals -D~ grad xi of Eq. xix)
    dim = o.lattice_info(lat)[1]
    for a in range(dim):
        Jp = (1.0 - 0.5 * l1) * th.mode_field(m1_hat[0, a], theta, shape)
        np.testing.assert_allclose(J[0, a], Jp, rtol=0, atol=2e-15)
        np.testing.assert_allclose(J[1, a], -Jp, rtol=0, atol=2e-15)


@pytest.mark.parametrize("lat", LATTICES)
def test_ternary_linear_response_exact(lat):
    """Small-amplitude ternary mode: (x(+e) - x(-e)) / 2e equals the linear scheme
    about xi_bar with Lambda_1 from the closed-form D~ (Remark IV), to O(e^2)."""
    o = _oracle()
    c, w = th.golden_lattice(lat)
    cs2 = th.cs2_of(c, w)
    dims = {"D2Q5": (16, 6, 1), "D2Q9": (12, 8, 1), "D3Q7": (8, 4, 6), "D3Q15": (6, 4, 5),
            "D1Q3": (16, 1, 1), "D2Q4": (12, 6, 1), "D3Q6": (8, 4, 6)}[lat]
    k = {"D2Q5": (1, 1, 0), "D2Q9": (1, 1, 0), "D3Q7": (1, 0, 1), "D3Q15": (1, 1, 1),
         "D1Q3": (1, 0, 0), "D2Q4": (1, 1, 0), "D3Q6": (1, 0, 1)}[lat]
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    D12, D13, D23 = 0.10, 0.08, 0.02
    D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D13, (2, 3): D23})
    xbar = np.array([0.3, 0.25, 0.45])
    v = np.array([1.0, -0.4, -0.6])
    eps = 1e-4
    steps = 80
    xp, Jp = o.run(lat, D, sy.small_mode(xbar, v, eps, nx, ny, nz, k=k), steps, flux=True)
    xm, Jm = o.run(lat, D, sy.small_mode(xbar, v, -eps, nx, ny, nz, k=k), steps, flux=True)
    resp = (xp - xm) / (2 * eps)
    jresp = (Jp - Jm) / (2 * eps)
    L1 = th.lambda1_from_Dtilde(th.ternary_Dtilde_closed(xbar, D12, D13, D23), cs2)
    L2 = th.magic_lambda2(L1)
    theta = th.theta_of(k, shape)
    xi_hat, m1_hat = th.predict_mode(c, w, L1, L2, theta, v, steps)
    for s in range(2):
        np.testing.assert_allclose(resp[s], th.mode_field(xi_hat[s], theta, shape),
                                   rtol=0, atol=1e-7)
    np.testing.assert_allclose(resp.sum(axis=0), 0.0, atol=1e-9)
    # flux response: J = (I - Lambda_1/2) m_1 of the pre-collision state, which is
    # -D~ grad xi with the gradient of Eq. xix
    J_hat = (np.eye(2) - 0.5 * L1) @ m1_hat
    for s in range(2):
        for a in range(jresp.shape[1]):
            np.testing.assert_allclose(jresp[s, a], th.mode_field(J_hat[s, a], theta, shape),
                                       rtol=0, atol=1e-8)
    np.testing.assert_allclose(jresp.sum(axis=0), 0.0, atol=1e-10)


@pytest.mark.parametrize("lat", LATTICES)
def test_frozen_mode_is_linear_and_exact(lat):
    """Relaxation matrices frozen at xi_ref make the ternary scheme linear: a
    finite-amplitude mode equals the exact amplification G(theta)^t with
    Lambda_1 from the closed-form D~(xi_ref) of Remark IV, fluxes included."""
    o = _oracle()
    c, w = th.golden_lattice(lat)
    cs2 = th.cs2_of(c, w)
    dims = {"D2Q5": (16, 6, 1), "D2Q9": (12, 8, 1), "D3Q7": (8, 4, 6), "D3Q15": (6, 4, 5),
            "D1Q3": (16, 1, 1), "D2Q4": (12, 6, 1), "D3Q6": (8, 4, 6)}[lat]
    k = {"D2Q5": (1, 1, 0), "D2Q9": (1, 1, 0), "D3Q7": (1, 0, 1), "D3Q15": (1, 1, 1),
         "D1Q3": (1, 0, 0), "D2Q4": (1, 1, 0), "D3Q6": (1, 0, 1)}[lat]
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    D12, D13, D23 = 0.10, 0.08, 0.02
    D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D13, (2, 3): D23})
    xref = np.array([0.3, 0.25, 0.45])
    v = np.array([1.0, -0.4, -0.6])
    eps = 0.1  # far from the small-amplitude limit: exactness comes from linearity
    steps = 60
    x, J = o.run(lat, D, sy.small_mode(xref, v, eps, nx, ny, nz, k=k), steps, flux=True,
                 relax="frozen", xi_ref=xref)
    L1 = th.lambda1_from_Dtilde(th.ternary_Dtilde_closed(xref, D12, D13, D23), cs2)
    L2 = th.magic_lambda2(L1)
    theta = th.theta_of(k, shape)
    xi_hat, m1_hat = th.predict_mode(c, w, L1, L2, theta, eps * v, steps)
    for s in range(2):
        np.testing.assert_allclose(x[s], xref[s] + th.mode_field(xi_hat[s], theta, shape),
                                   rtol=0, atol=1e-14)
    J_hat = (np.eye(2) - 0.5 * L1) @ m1_hat
    for s in range(2):
        for a in range(J.shape[1]):
            np.testing.assert_allclose(J[s, a], th.mode_field(J_hat[s, a], theta, shape),
                                       rtol=0, atol=1e-14)


# --------------------------------------------------------------------------
# Continuum limit (Chapman-Enskog, Eq. 3-26; second-order convergence)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat", LATTICES)
def test_binary_continuum_decay_second_order(lat):
    """A sine mode decays as exp(-D |k|^2 t); the rate error falls ~4x per doubling."""
    o = _oracle()
    Dv = 0.05
    D = sy.D_from_pairs(2, {(1, 2): Dv})
    errs = []
    for nx in (32, 64):
        k = (1, 0, 0)
        x0 = sy.small_mode([0.5, 0.5], [1.0, -1.0], 0.1, nx, 1, 1, k=k)
        theta = 2 * math.pi / nx
        steps = int(round(0.5 / (Dv * theta ** 2)))
        x = o.run(lat, D, x0, steps)
        amp = 2.0 / nx * np.sum((x[0, 0, 0] - 0.5) * np.cos(theta * np.arange(nx)))
        Deff = -math.log(amp / 0.1) / (theta ** 2 * steps)
        errs.append(abs(Deff / Dv - 1.0))
    assert errs[0] < 0.02
    assert errs[1] < 0.005
    assert errs[0] / errs[1] > 3.0


def test_ternary_continuum_decay():
    """Small ternary mode follows exp(-|k|^2 D~(xi_bar) t) of Eq. 2-13 linearised."""
    o = _oracle()
    D12, D13, D23 = 0.10, 0.08, 0.02
    D = sy.D_from_pairs(3, {(1, 2): D12, (1, 3): D13, (2, 3): D23})
    xbar = np.array([0.3, 0.25, 0.45])
    v = np.array([1.0, -0.4, -0.6])
    nx, eps = 64, 1e-4
    theta = 2 * math.pi / nx
    Dt = th.ternary_Dtilde_closed(xbar, D12, D13, D23)
    steps = 1500
    xp = o.run("D2Q5", D, sy.small_mode(xbar, v, eps, nx), steps)
    xm = o.run("D2Q5", D, sy.small_mode(xbar, v, -eps, nx), steps)
    resp = (xp - xm)[:2, 0, 0] / (2 * eps)
    amp = 2.0 / nx * resp @ np.cos(theta * np.arange(nx))
    pred = expm(-theta ** 2 * Dt * steps) @ v[:2]
    np.testing.assert_allclose(amp, pred, rtol=0, atol=4e-3 * np.abs(v[:2]).max())


@pytest.mark.parametrize("lat,axis", [("D2Q5", 0), ("D2Q9", 1), ("D3Q7", 2), ("D3Q15", 1),
                                      ("D1Q3", 0), ("D2Q4", 1), ("D3Q6", 2)])
def test_local_gradient_is_second_order(lat, axis):
    """Eq. xix: the gradient read from the first moments of the populations
    equals the spectral derivative of the mole-fraction field to O(dx^2)."""
    o = _oracle()
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.08, (2, 3): 0.02})
    errs = []
    for nx in (32, 64):
        dims = [1, 1, 1]  # (nx, ny, nz)
        dims[axis] = nx
        dim = o.lattice_info(lat)[1]
        if dim > 1:
            dims[(axis + 1) % dim] = 2
        k = [0, 0, 0]
        k[axis] = 1
        x0 = sy.small_mode([0.3, 0.3, 0.4], [1.0, -0.4, -0.6], 0.02, *dims, k=tuple(k))
        x, G = o.run(lat, D, x0, 200, grad=True)
        ax = 3 - axis  # array axis of the field [n, nz, ny, nx]
        shape = [1, 1, 1, 1]
        shape[ax] = nx
        ik = (2j * np.pi * np.fft.fftfreq(nx)).reshape(shape)
        dxi = np.real(np.fft.ifft(np.fft.fft(x, axis=ax) * ik, axis=ax))
        errs.append(np.abs(G[:, axis] - dxi).max() / np.abs(dxi).max())
        # the other components vanish for a plane wave
        for a in range(G.shape[1]):
            if a != axis:
                assert np.abs(G[:, a]).max() < 1e-15
    assert errs[1] < 3e-3
    assert errs[0] / errs[1] > 3.8


def test_binary_flux_is_fick():
    """J_1 = -D d(xi_1)/dx (Remark I) for a slow mode, to O(k^2)."""
    o = _oracle()
    Dv, nx = 0.05, 64
    D = sy.D_from_pairs(2, {(1, 2): Dv})
    theta = 2 * math.pi / nx
    x, J = o.run("D2Q5", D, sy.small_mode([0.5, 0.5], [1, -1], 0.1, nx), 400, flux=True)
    X = np.arange(nx)
    amp = 2.0 / nx * np.sum((x[0, 0, 0] - 0.5) * np.cos(theta * X))
    Jref = Dv * amp * theta * np.sin(theta * X)
    np.testing.assert_allclose(J[0, 0, 0, 0], Jref, rtol=0, atol=3e-3 * np.abs(Jref).max())


# --------------------------------------------------------------------------
# Conservation and boundaries (Sec. 4: half-way bounce-back, periodic)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("lat,bc", [
    ("D2Q9", ("periodic", "periodic", "noflux", "noflux", "periodic", "periodic")),
    ("D2Q5", ("noflux",) * 4 + ("periodic",) * 2),
    ("D3Q7", ("noflux",) * 6),
    ("D3Q15", ("noflux", "noflux", "periodic", "periodic", "noflux", "noflux")),
    ("D1Q3", ("noflux", "noflux") + ("periodic",) * 4),
    ("D2Q4", ("noflux",) * 4 + ("periodic",) * 2),
    ("D3Q6", ("noflux",) * 6),
])
def test_mass_conservation_and_closure(lat, bc):
    o = _oracle()
    n = 4
    D = sy.random_D(n, seed=43)
    if lat in ("D3Q7", "D3Q15", "D3Q6"):
        x0 = sy.sin_modes(n, 9, 7, 6, amp=0.1, seed=44)
    elif lat == "D1Q3":
        x0 = sy.sin_modes(n, 37, 1, amp=0.1, seed=46)
    else:
        x0 = sy.sin_modes(n, 13, 11, amp=0.1, seed=45)
    x = o.run(lat, D, x0, 150, bc=bc)
    np.testing.assert_allclose(x.sum(axis=(1, 2, 3)), x0.sum(axis=(1, 2, 3)), rtol=1e-13)
    np.testing.assert_allclose(x.sum(axis=0), 1.0, atol=1e-14)


@pytest.mark.parametrize("lat", ["D2Q5", "D3Q7", "D1Q3", "D2Q4", "D3Q6"])
def test_bounce_back_equals_mirrored_periodic(lat):
    """Half-way bounce-back on [0, L) equals a periodic run of the mirrored field on
    [0, 2L) (exact for the axis-aligned lattices)."""
    o = _oracle()
    n = 3
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.08, (2, 3): 0.02})
    if lat in ("D2Q5", "D2Q4"):
        x0 = sy.sin_modes(n, 10, 7, amp=0.1, seed=47)
        axes = (3, 2)
    elif lat == "D1Q3":
        x0 = sy.sin_modes(n, 17, 1, amp=0.1, seed=49)
        axes = (3,)
    else:
        x0 = sy.sin_modes(n, 6, 5, 4, amp=0.1, seed=48)
        axes = (3, 2, 1)
    big = x0
    for ax in axes:
        big = np.concatenate([big, np.flip(big, axis=ax)], axis=ax)
    steps = 70
    closed = o.run(lat, D, x0, steps, bc=("noflux",) * 6)
    per = o.run(lat, D, big, steps)
    sl = tuple([slice(None)] + [slice(0, s) for s in x0.shape[1:]])
    np.testing.assert_allclose(closed, per[sl], rtol=0, atol=1e-14)


def test_d2q9_bounce_back_y_uniform():
    """D2Q9 with walls in x and y-uniform data equals the mirrored periodic run."""
    o = _oracle()
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.08, (2, 3): 0.02})
    x0 = sy.two_bulb(12, 5, 1, width=2.0)
    big = np.concatenate([x0, np.flip(x0, axis=3)], axis=3)
    bc = ("noflux", "noflux", "periodic", "periodic", "periodic", "periodic")
    closed = o.run("D2Q9", D, x0, 60, bc=bc)
    per = o.run("D2Q9", D, big, 60)
    np.testing.assert_allclose(closed, per[..., :12], rtol=0, atol=1e-14)


def test_d3q15_bounce_back_yz_uniform():
    """D3Q15 with walls in x and y/z-uniform data equals the mirrored periodic run
    (the diagonal populations (c_x, c_y, c_z) and (c_x, -c_y, -c_z) agree by symmetry,
    so bounce-back and mirror reflection give the same populations)."""
    o = _oracle()
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.08, (2, 3): 0.02})
    x0 = sy.two_bulb(10, 3, 2, width=2.0)
    big = np.concatenate([x0, np.flip(x0, axis=3)], axis=3)
    bc = ("noflux", "noflux") + ("periodic",) * 4
    closed = o.run("D3Q15", D, x0, 50, bc=bc)
    per = o.run("D3Q15", D, big, 50)
    np.testing.assert_allclose(closed, per[..., :10], rtol=0, atol=1e-14)


def test_closed_tube_3d_equals_1d():
    """x-only data in a closed D3Q7 box stays y/z-uniform and equals the 1-cell run."""
    o = _oracle()
    D = sy.D_from_pairs(3, {(1, 2): 0.1, (1, 3): 0.08, (2, 3): 0.02})
    x3 = sy.two_bulb(16, 4, 3)
    x1 = sy.two_bulb(16, 1, 1)
    a = o.run("D3Q7", D, x3, 90, bc=("noflux",) * 6)
    b = o.run("D3Q7", D, x1, 90, bc=("noflux",) * 6)
    np.testing.assert_allclose(a, np.broadcast_to(b, a.shape), rtol=0, atol=1e-15)


# --------------------------------------------------------------------------
# Numbers printed in the paper (Secs. 4.2 and 4.3)
# --------------------------------------------------------------------------

def test_duncan_toor_minimum():
    """xi_2 at x = 0.72 dips to 0.1581 at about t = 0.2 (Sec. 4.2)."""
    o = _oracle()
    P = th.golden_numbers()
    nx = int(P["duncan_toor.cells"])
    Dmax = max(P["duncan_toor.D12"], P["duncan_toor.D13"], P["duncan_toor.D23"])
    scale = 0.1 / Dmax  # lattice diffusivity of the fastest pair = 0.1
    D = sy.D_from_pairs(3, {(1, 2): P["duncan_toor.D12"] * scale,
                            (1, 3): P["duncan_toor.D13"] * scale,
                            (2, 3): P["duncan_toor.D23"] * scale})
    dt = scale / nx ** 2
    steps = int(round(0.3 / dt))
    snaps = np.arange(0, steps + 1, 200)
    x0 = sy.duncan_toor_1d(nx)
    bc = ("noflux", "noflux") + ("periodic",) * 4
    x, S = o.run("D2Q5", D, x0, steps, bc=bc, snapshots=snaps)
    X = (np.arange(nx) + 0.5) / nx
    x2 = np.array([np.interp(P["duncan_toor.probe_x"], X, s[1, 0, 0]) for s in S])
    i = int(np.argmin(x2))
    assert abs(x2[i] - P["duncan_toor.xi2_min"]) < 5e-4
    assert abs(snaps[i] * dt - P["duncan_toor.t_min"]) < 0.02
    # equilibria are the means of the initial field (mass conservation)
    assert abs(x0[0].mean() - P["duncan_toor.xi1_eq"]) < 1e-12
    assert abs(x[1].mean() - P["duncan_toor.xi2_eq"]) < 1e-12


def test_loschmidt_peak_time():
    """Bottom-half mean of xi_2 peaks at t* = 0.35 h (Sec. 4.3)."""
    o = _oracle()
    P = th.golden_numbers()
    n = int(P["loschmidt.cells"])
    Dmax = max(P["loschmidt.D12"], P["loschmidt.D13"], P["loschmidt.D23"])
    scale = 0.1 / Dmax
    D = sy.D_from_pairs(3, {(1, 2): P["loschmidt.D12"] * scale,
                            (1, 3): P["loschmidt.D13"] * scale,
                            (2, 3): P["loschmidt.D23"] * scale})
    dx = 2.0 / n  # tube [-L, L] with L = 1
    dt = scale * dx * dx
    t_ref = (100 * math.pi * math.sqrt(1.0 / 60.0)) ** 2  # seconds
    steps = int(round(1.0 / dt))
    snaps = np.arange(0, steps + 1, 100)
    bc = ("noflux", "noflux") + ("periodic",) * 4
    x0 = sy.loschmidt_1d(n)
    x, S = o.run("D2Q5", D, x0, steps, bc=bc, snapshots=snaps)
    bottom = S[:, 1, 0, 0, : n // 2].mean(axis=1)
    t_peak_h = snaps[int(np.argmax(bottom))] * dt * t_ref / 3600.0
    # printed to two digits: 0.35 h
    assert abs(t_peak_h - P["loschmidt.t_peak_hours"]) <= 0.005
    assert abs(x0[0].mean() - P["loschmidt.xi1_eq"]) < 1e-12
    assert abs(x0[1].mean() - P["loschmidt.xi2_eq"]) < 1e-12
