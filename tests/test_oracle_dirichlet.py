"""Pins of the oracle's Dirichlet (half-way anti-bounce-back) faces, Sec. 4.

* Table I: the relative L2 errors of xi_1 and J_1 of the two-component erf
  problem at t = 1, 5, 20 for MRT (Eq. 3-16) and SRT, as printed.
* Figs. 3 and 4: second-order convergence in space at t = 5 for several
  lambda_1^11.
* Steady states: a binary mixture between two Dirichlet walls relaxes to the
  exact linear profile (walls half-way), on every lattice and both relaxation
  modes; a ternary one converges at second order to the steady Maxwell-Stefan
  profile of Eq. 2-12 computed by shooting with the closed form of Remark IV.
"""

import math

import numpy as np
import pytest

import synthetic as sy
import theory as th

DIR_X = ("dirichlet", "dirichlet", "periodic", "periodic", "periodic", "periodic")


def _oracle():
    import oracle

    oracle.build()
    return oracle


def _erf_run(o, nx, lam1, relax, times, *, ny=1):
    """Errors (E(xi_1), E(J_1)) of the Sec. 4.1 problem at the given times."""
    P = th.golden_numbers()
    Dp, C0, C1 = P["erf.D"], P["erf.C0"], P["erf.C1"]
    dx = 12.0 / nx
    Dl = (1.0 / lam1 - 0.5) / 3.0  # Eq. 3-26 for one species, c_s^2 = 1/3
    dt = Dl * dx * dx / Dp
    X = -6.0 + (np.arange(nx) + 0.5) * dx
    x0 = sy.erf_step(nx, ny, C0=C0, C1=C1)
    D = np.array([[1.0, Dl], [Dl, 1.0]])
    xb = np.zeros((6, 2))
    xb[0] = (C0, 1.0 - C0)
    xb[1] = (C1, 1.0 - C1)
    out = []
    for t in times:
        steps = int(round(t / dt))
        x, J = o.run("D2Q5", D, x0, steps, bc=DIR_X, xb=xb, relax=relax, flux=True)
        xa, Ja = th.erf_solution(X, steps * dt, Dp, C0, C1)
        # lattice flux to physical units: J dx / dt
        out.append((th.rel_l2(np.broadcast_to(xa, x[0, 0].shape), x[0, 0]),
                    th.rel_l2(np.broadcast_to(Ja, x[0, 0].shape), J[0, 0, 0] * dx / dt)))
    return out


@pytest.mark.parametrize("relax,tag", [("magic", "mrt"), ("srt", "srt")])
def test_table_I_errors(relax, tag):
    """Table I to 0.3 % (the printed values have five digits)."""
    o = _oracle()
    P = th.golden_numbers()
    errs = _erf_run(o, int(P["erf.nx"]), P["erf.lambda1"], relax, (1, 5, 20))
    for (Ex, EJ), t in zip(errs, (1, 5, 20)):
        assert Ex == pytest.approx(P["erf.%s.Ex.t%d" % (tag, t)], rel=3e-3)
        assert EJ == pytest.approx(P["erf.%s.EJ.t%d" % (tag, t)], rel=3e-3)


def test_table_I_holds_on_the_full_2d_grid():
    """240 x 40 with periodic y gives the same errors as one row (y-uniform data)."""
    o = _oracle()
    P = th.golden_numbers()
    a = _erf_run(o, 240, 1.25, "magic", (1,), ny=int(P["erf.ny"]))[0]
    b = _erf_run(o, 240, 1.25, "magic", (1,), ny=1)[0]
    assert a == pytest.approx(b, rel=1e-10)
    assert a[0] == pytest.approx(P["erf.mrt.Ex.t1"], rel=3e-3)


@pytest.mark.parametrize("lam1", [0.8, 1.25, 1.6])
def test_second_order_convergence(lam1):
    o = _oracle()
    P = th.golden_numbers()
    nxs = (120, 240, 360, 480)  # dx = 1/10, 1/20, 1/30, 1/40
    errs = [_erf_run(o, nx, lam1, "magic", (5,))[0] for nx in nxs]
    logdx = np.log([12.0 / n for n in nxs])
    for comp in (0, 1):
        slope = np.polyfit(logdx, np.log([e[comp] for e in errs]), 1)[0]
        assert abs(slope - P["erf.convergence_slope"]) < 0.05


@pytest.mark.parametrize("lat,shape", [("D2Q5", (1, 3, 16)), ("D2Q9", (1, 3, 16)),
                                       ("D3Q7", (2, 2, 16)), ("D3Q15", (2, 2, 16)),
                                       ("D1Q3", (1, 1, 16)), ("D2Q4", (1, 3, 16)),
                                       ("D3Q6", (2, 2, 16))])
@pytest.mark.parametrize("relax", ["magic", "srt"])
def test_binary_linear_steady_state_is_exact(lat, shape, relax):
    o = _oracle()
    nz, ny, nx = shape
    Dl = 0.07
    D = np.array([[1.0, Dl], [Dl, 1.0]])
    x0 = np.full((2,) + shape, 0.5)
    xb = np.zeros((6, 2))
    xb[0] = (0.9, 0.1)
    xb[1] = (0.2, 0.8)
    x, J = o.run(lat, D, x0, 40000, bc=DIR_X, xb=xb, relax=relax, flux=True)
    X = (np.arange(nx) + 0.5) / nx
    lin = 0.9 + (0.2 - 0.9) * X
    np.testing.assert_allclose(x[0], np.broadcast_to(lin, shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(x[1], 1.0 - x[0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(J[0, 0], -Dl * (0.2 - 0.9) / nx, rtol=1e-10, atol=0)


def test_ternary_steady_state_converges_to_maxwell_stefan_profile():
    o = _oracle()
    d12, d13, d23 = 0.1, 0.08, 0.02
    D = sy.D_from_pairs(3, {(1, 2): d12, (1, 3): d13, (2, 3): d23})
    xL = np.array([0.1, 0.3, 0.6])
    xR = np.array([0.7, 0.25, 0.05])
    xb = np.zeros((6, 3))
    xb[0], xb[1] = xL, xR
    errs = []
    for nx in (16, 32):
        x0 = np.broadcast_to(((xL + xR) / 2)[:, None, None, None], (3, 1, 1, nx)).copy()
        steps = int(12 * nx * nx / d23)
        x = o.run("D2Q5", D, x0, steps, bc=DIR_X, xb=xb)
        X = (np.arange(nx) + 0.5) / nx
        ref, _ = th.ternary_steady_profile(xL, xR, d12, d13, d23, X)
        errs.append(np.abs(x[:, 0, 0, :] - ref).max())
    assert errs[1] < 2e-4
    assert errs[0] / errs[1] > 3.5  # second order


def test_uniform_dirichlet_state_is_a_fixed_point():
    o = _oracle()
    D = sy.random_D(4, seed=11)
    xb = np.tile([0.1, 0.2, 0.3, 0.4], (6, 1))
    x0 = np.broadcast_to(xb[0][:, None, None, None], (4, 3, 4, 5)).copy()
    bc = ("dirichlet", "dirichlet", "noflux", "dirichlet", "periodic", "periodic")
    for lat in ("D2Q5", "D2Q9"):
        x = o.run(lat, D, x0[:, :1], 50, bc=bc, xb=xb)
        np.testing.assert_allclose(x, x0[:, :1], rtol=0, atol=1e-15)
    x = o.run("D3Q7", D, x0, 50, bc=("dirichlet",) * 6, xb=xb)
    np.testing.assert_allclose(x, x0, rtol=0, atol=1e-15)


def test_dirichlet_arguments_are_checked():
    o = _oracle()
    D = sy.random_D(3)
    x0 = np.full((3, 1, 2, 4), 1.0 / 3.0)
    with pytest.raises(RuntimeError):
        o.run("D2Q5", D, x0, 1, bc=DIR_X)  # Dirichlet without compositions
    with pytest.raises(RuntimeError):
        o.run("D2Q5", D, x0, 1, bc=("dirichlet", "periodic") + ("periodic",) * 4,
              xb=np.zeros((6, 3)))  # periodic face without its partner
