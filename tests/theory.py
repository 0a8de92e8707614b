"""Independent predictions used to pin the oracle (test-only helpers).

Nothing here calls the oracle or the CUDA library.  The lattice tables are
read from ``tests/golden/lattices.txt`` (the velocities and weights printed in
Eqs. 3-7, 3-8 and 3-10), and the collision is built in the two-relaxation-time
pair form rather than through a moment matrix:

* odd (antisymmetric) part of f - f_eq of each opposite pair relaxes with
  Lambda_1, even (symmetric) part and the rest population relax with
  Lambda_2.  Sec. 3.1 states this equivalence of the MRT model with odd/even
  relaxation groups and the TRT model.

With that operator the scheme is linear whenever Lambda is constant, so a
single Fourier mode evolves exactly by the amplification matrix
G = diag(exp(-i theta . c_q)) (I - Omega (I - W)), with W the equilibrium map
f -> w_k sum_q f_q of Eq. 3-3 and the streaming of Eq. 3-13b.
"""

from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_lattice(name: str):
    """(c[Q,3] int, w[Q] float) for one lattice, from the golden table."""
    rows = []
    with open(os.path.join(GOLDEN, "lattices.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            if p[0] == name:
                rows.append((int(p[1]), int(p[2]), int(p[3]), int(p[4]), float(Fraction(p[5]))))
    rows.sort()
    c = np.array([[r[1], r[2], r[3]] for r in rows], dtype=np.int64)
    w = np.array([r[4] for r in rows])
    return c, w


def golden_numbers() -> dict:
    out = {}
    with open(os.path.join(GOLDEN, "paper_numbers.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = float(v)
    return out


def golden_M0():
    M, m0 = [], None
    with open(os.path.join(GOLDEN, "d2q5_M0.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p = line.split()
            vals = [float(Fraction(v)) for v in p[1:]]
            if p[0] == "M0":
                M.append(vals)
            else:
                m0 = vals
    return np.array(M), np.array(m0)


def opposite(c: np.ndarray) -> np.ndarray:
    Q = c.shape[0]
    opp = np.empty(Q, dtype=np.int64)
    for k in range(Q):
        opp[k] = [m for m in range(Q) if np.all(c[m] == -c[k])][0]
    return opp


def cs2_of(c, w) -> float:
    return float(np.sum(w * c[:, 0] ** 2))


def pair_projectors(c):
    """(P_odd, P_even) on R^Q: antisymmetric and symmetric parts over opposite pairs."""
    Q = c.shape[0]
    opp = opposite(c)
    Po = np.zeros((Q, Q))
    Pe = np.zeros((Q, Q))
    for k in range(Q):
        if opp[k] == k:
            Pe[k, k] = 1.0
        else:
            Po[k, k] += 0.5
            Po[k, opp[k]] -= 0.5
            Pe[k, k] += 0.5
            Pe[k, opp[k]] += 0.5
    return Po, Pe


def collision_operator(c, L1, L2):
    """Omega on R^{S Q} (index s*Q + k) in the pair form."""
    Po, Pe = pair_projectors(c)
    return np.kron(L1, Po) + np.kron(L2, Pe)


def equilibrium_map(w, S):
    Q = w.size
    return np.kron(np.eye(S), np.outer(w, np.ones(Q)))


def magic_lambda2(L1):
    """Eq. 3-16: off-diagonal = Lambda_1, diagonal 8 (l - 2) / (l - 8)."""
    L2 = L1.copy()
    for i in range(L1.shape[0]):
        l = L1[i, i]
        L2[i, i] = 8.0 * (l - 2.0) / (l - 8.0)
    return L2


def amplification(c, w, L1, L2, theta):
    """G(theta) for the linear scheme with constant Lambda_1, Lambda_2."""
    S = L1.shape[0]
    Q = w.size
    Om = collision_operator(c, L1, L2)
    W = equilibrium_map(w, S)
    coll = np.eye(S * Q) - Om @ (np.eye(S * Q) - W)
    shift = np.exp(-1j * (c @ np.asarray(theta, dtype=np.float64)))
    return np.kron(np.eye(S), np.diag(shift)) @ coll


def predict_mode(c, w, L1, L2, theta, amp_vec, steps):
    """Complex mode coefficients after ``steps`` steps from f = f_eq of ``amp_vec``.

    Returns (xi_hat[S], m1_hat[S, 3]) where the field is Re[hat * exp(i theta . x)].
    """
    S = L1.shape[0]
    Q = w.size
    F = np.kron(np.asarray(amp_vec[:S], dtype=np.float64), w).astype(np.complex128)
    G = amplification(c, w, L1, L2, theta)
    F = np.linalg.matrix_power(G, steps) @ F
    F = F.reshape(S, Q)
    xi = F.sum(axis=1)
    m1 = F @ c.astype(np.float64)
    return xi, m1


def ternary_Dtilde_closed(xi, D12, D13, D23):
    """Second closed form of D~ for three species, Remark IV (Eq. 2-19)."""
    x1, x2, x3 = xi
    den = x1 * D23 + x2 * D13 + x3 * D12
    return np.array([
        [D13 * (x1 * D23 + (1.0 - x1) * D12), x1 * D23 * (D13 - D12)],
        [x2 * D13 * (D23 - D12), D23 * (x2 * D13 + (1.0 - x2) * D12)],
    ]) / den


def lambda1_from_Dtilde(Dt, cs2):
    """Lambda_1 solving D~ = c_s^2 (Lambda_1^{-1} - I/2), Eq. 3-26."""
    S = Dt.shape[0]
    return np.linalg.inv(Dt / cs2 + 0.5 * np.eye(S))


def mode_field(hat, theta, shape):
    """Re[hat * exp(i theta . x)] on integer node positions, shape (nz, ny, nx)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ph = theta[0] * x + theta[1] * y + theta[2] * z
    return np.real(hat * np.exp(1j * ph))


def theta_of(k, shape):
    nz, ny, nx = shape
    return np.array([2 * math.pi * k[0] / nx, 2 * math.pi * k[1] / ny,
                     2 * math.pi * k[2] / nz if nz > 1 else 0.0])


def erf_solution(X, t, D, C0, C1):
    """Two-component step on the infinite line (Sec. 4.1, Eq. 4-2): xi_1 and J_1."""
    from scipy.special import erf

    X = np.asarray(X, dtype=np.float64)
    xi = 0.5 * (C0 + C1) + 0.5 * (C1 - C0) * erf(X / (2.0 * np.sqrt(D * t)))
    J = -0.5 * (C1 - C0) * np.sqrt(D / (np.pi * t)) * np.exp(-X * X / (4.0 * D * t))
    return xi, J


def rel_l2(a, n):
    """Relative L2 error E = ||a - n|| / ||a|| (Sec. 4)."""
    a = np.asarray(a)
    return float(np.sqrt(np.sum((a - n) ** 2) / np.sum(a ** 2)))


def ternary_steady_profile(xL, xR, D12, D13, D23, X):
    """Steady one-dimensional Maxwell-Stefan profile between two fixed compositions.

    With no sources the flux J is uniform and d(xi)/dX = -D~(xi)^{-1} J
    (Eq. 2-12 on [0, 1]); J is found by shooting from xL so that the profile ends
    at xR.  Uses the closed form of D~ of Remark IV, not the solver's B.
    """
    from scipy.integrate import solve_ivp
    from scipy.optimize import fsolve

    xL = np.asarray(xL, dtype=np.float64)
    xR = np.asarray(xR, dtype=np.float64)

    def rhs(_, y):
        xi = (y[0], y[1], 1.0 - y[0] - y[1])
        return -np.linalg.solve(ternary_Dtilde_closed(xi, D12, D13, D23), rhs.J)

    def shoot(J):
        rhs.J = np.asarray(J)
        sol = solve_ivp(rhs, (0.0, 1.0), xL[:2], rtol=1e-12, atol=1e-14)
        return sol.y[:, -1] - xR[:2]

    J0 = -ternary_Dtilde_closed(0.5 * (xL + xR), D12, D13, D23) @ (xR[:2] - xL[:2])
    J = fsolve(shoot, J0, xtol=1e-13)
    rhs.J = J
    sol = solve_ivp(rhs, (0.0, 1.0), xL[:2], rtol=1e-12, atol=1e-14, dense_output=True)
    y = sol.sol(np.asarray(X, dtype=np.float64))
    return np.vstack([y, 1.0 - y.sum(axis=0)]), J
