"""The benchmark problems of Sec. 4, run on the CUDA solver.

Each driver converts the problem's physical data to lattice units, runs the
solver through its C ABI and returns plain NumPy arrays of what the paper plots:

* ``erf_binary``   -- Sec. 4.1: two-component step between Dirichlet walls on
  [-6, 6] x [-1, 1]; profiles of xi_1 and J_1 (Figs. 1-2) and their relative L2
  errors against the erf solution of Eq. 4-2 (Table I, Figs. 3-4).
* ``duncan_toor``  -- Sec. 4.2: the ternary coupling problem on [0, 1]^2 with
  no-flux walls in x; xi, J and -d(xi)/dx at a probe (Figs. 5-7) and the fields
  at the end (Figs. 8-9).
* ``loschmidt``    -- Sec. 4.3: the CH4 / Ar / H2 Loschmidt tube on [-L, L]^2,
  no-flux at y = +-L, periodic in x; bottom and top averages of xi_1, xi_2 in
  hours (Figs. 11-12) and profiles along y (Figs. 13-14).

Lattice units: the grid spacing is the domain length over the node count and
the time step makes the largest lattice diffusivity ``d_max`` (0.1 by default),
dt = d_max dx^2 / max D_ij.  The paper does not give its time steps for
Secs. 4.2 and 4.3; in Sec. 4.1 it fixes lambda_1 = 1.25, i.e. a lattice
diffusivity (1/lambda_1 - 1/2) c_s^2 = 0.1.
"""

from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np
import torch

from .lbms import Solver

P, W, B = "periodic", "noflux", "dirichlet"


def _pairs_matrix(n: int, pairs: Dict[tuple, float]) -> np.ndarray:
    D = np.ones((n, n))
    for (i, j), v in pairs.items():
        D[i - 1, j - 1] = D[j - 1, i - 1] = float(v)
    return D


def lattice_units(pairs: Dict[tuple, float], dx: float, d_max: float = 0.1):
    """Lattice diffusivities {(i, j): D_ij dt / dx^2} and the time step dt that
    makes the largest of them ``d_max``."""
    dt = d_max * dx * dx / max(pairs.values())
    return {k: v * dt / (dx * dx) for k, v in pairs.items()}, dt


def erf_solution(X, t: float, D: float, C0: float, C1: float):
    """Eq. 4-2: xi_1 and J_1 of a step from C0 (x < 0) to C1 on the whole line."""
    X = np.asarray(X, dtype=np.float64)
    erf = np.vectorize(math.erf)
    xi = 0.5 * (C0 + C1) + 0.5 * (C1 - C0) * erf(X / (2.0 * math.sqrt(D * t)))
    J = -0.5 * (C1 - C0) * np.sqrt(D / (math.pi * t)) * np.exp(-X * X / (4.0 * D * t))
    return xi, J


def relative_l2(ref, num) -> float:
    """E(phi) of Sec. 4: ||phi_a - phi_n|| / ||phi_a|| over all nodes."""
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(np.sum((ref - num) ** 2) / np.sum(ref ** 2)))


def erf_binary(nx: int = 240, ny: int = 40, *, lambda1: float = 1.25, relax: str = "magic",
               times: Sequence[float] = (1.0, 5.0, 20.0), D: float = 0.05, C0: float = 0.9,
               C1: float = 0.1, dtype=torch.float64) -> dict:
    """Sec. 4.1.  Dirichlet walls at x = -6 (xi_1 = C0) and x = 6 (C1), periodic
    in y; lambda_1 = 1.25 sets the lattice diffusivity, hence dt.  Returns the
    node positions, and per time the xi_1 and J_1 (physical units) profiles of
    the first row with their errors E(xi_1), E(J_1)."""
    dx = 12.0 / nx
    d_lat = (1.0 / lambda1 - 0.5) / 3.0  # Eq. 3-26 for one species, c_s^2 = 1/3
    dt = d_lat * dx * dx / D
    X = -6.0 + (np.arange(nx) + 0.5) * dx
    x1 = np.where(X < 0.0, C0, C1)
    x0 = np.empty((2, 1, ny, nx))
    x0[0] = x1
    x0[1] = 1.0 - x1
    s = Solver("D2Q5", _pairs_matrix(2, {(1, 2): d_lat}), (nx, ny), bc=(B, B, P, P, P, P),
               relax=relax, dtype=dtype, boundary={0: (C0, 1.0 - C0), 1: (C1, 1.0 - C1)})
    s.set_state(torch.from_numpy(x0).to(dtype).to(s.device))
    out = {"X": X, "dt": dt, "t": [], "xi1": [], "J1": [], "E_xi1": [], "E_J1": []}
    done = 0
    for t in times:
        steps = int(round(t / dt))
        s.step(steps - done)
        done = steps
        x, J = s.moments(flux=True)
        xi = _host(x)[0, 0]
        Jx = _host(J)[0, 0, 0] * dx / dt  # lattice flux to physical
        xa, Ja = erf_solution(X, steps * dt, D, C0, C1)
        out["t"].append(steps * dt)
        out["xi1"].append(xi[0])
        out["J1"].append(Jx[0])
        out["E_xi1"].append(relative_l2(np.broadcast_to(xa, xi.shape), xi))
        out["E_J1"].append(relative_l2(np.broadcast_to(Ja, Jx.shape), Jx))
    for k in ("t", "xi1", "J1", "E_xi1", "E_J1"):
        out[k] = np.asarray(out[k])
    return out


def duncan_toor_initial(nx: int, ny: int) -> np.ndarray:
    """Initial field of Sec. 4.2 on cell centres of [0, 1]^2 (x-dependent only)."""
    X = (np.arange(nx) + 0.5) / nx
    x1 = np.where(X < 0.25, 0.8, np.where(X < 0.75, 1.6 * (0.75 - X), 0.0))
    out = np.empty((3, 1, ny, nx))
    out[0] = x1
    out[1] = 0.2
    out[2] = 1.0 - out[0] - out[1]
    return out


def _host(t: torch.Tensor) -> np.ndarray:
    """Solver output copied to the host as float64 (analysis happens there)."""
    return t.cpu().numpy().astype(np.float64)


def _probe(field_row: np.ndarray, X: np.ndarray, x: float) -> float:
    return float(np.interp(x, X, field_row))


def duncan_toor(nx: int = 200, ny: int = 200, *, t_end: float = 1.0, samples: int = 200,
                probe_x: float = 0.72, d_max: float = 0.1, dtype=torch.float64) -> dict:
    """Sec. 4.2: D12 = D13 = 0.833, D23 = 0.168 on [0, 1]^2, no flux at x = 0, 1,
    periodic in y.  Returns times and, at x = probe_x, xi_i, J_i (physical
    units) and -d(xi_i)/dx of Eq. xix for i = 1, 2, 3 (arrays [samples + 1, 3]),
    and the final xi, J, -d(xi)/dx rows along x."""
    dx = 1.0 / nx
    pairs, dt = lattice_units({(1, 2): 0.833, (1, 3): 0.833, (2, 3): 0.168}, dx, d_max)
    s = Solver("D2Q5", _pairs_matrix(3, pairs), (nx, ny), bc=(W, W, P, P, P, P), dtype=dtype)
    s.set_state(torch.from_numpy(duncan_toor_initial(nx, ny)).to(dtype).to(s.device))
    X = (np.arange(nx) + 0.5) * dx
    total = int(round(t_end / dt))
    marks = np.unique(np.round(np.linspace(0, total, samples + 1)).astype(np.int64))
    out = {"t": [], "xi": [], "J": [], "neg_grad": [], "dt": dt, "X": X}
    done = 0
    for m in marks:
        s.step(int(m - done))
        done = int(m)
        x, J = s.moments(flux=True)
        G = s.gradient()
        xr = _host(x)[:, 0, 0]
        Jr = _host(J)[:, 0, 0, 0] * dx / dt
        Gr = -_host(G)[:, 0, 0, 0] / dx
        out["t"].append(m * dt)
        out["xi"].append([_probe(r, X, probe_x) for r in xr])
        out["J"].append([_probe(r, X, probe_x) for r in Jr])
        out["neg_grad"].append([_probe(r, X, probe_x) for r in Gr])
    out["final"] = {"xi": xr, "J": Jr, "neg_grad": Gr}
    for k in ("t", "xi", "J", "neg_grad"):
        out[k] = np.asarray(out[k])
    return out


LOSCHMIDT_L_CM = 100.0 * math.pi * math.sqrt(1.0 / 60.0)  # tube half-length L_ref, cm
LOSCHMIDT_T_REF_S = LOSCHMIDT_L_CM ** 2  # t_ref = L_ref^2 s / cm^2


def loschmidt_initial(nx: int, ny: int) -> np.ndarray:
    """Sec. 4.3: top half (y > 0) CH4 / Ar = 0.515 / 0.485, bottom half Ar / H2 =
    0.509 / 0.491, on cell centres of [-L, L]^2 (y-dependent only)."""
    out = np.empty((3, 1, ny, nx))
    top = np.array([0.515, 0.485, 0.0])
    bottom = np.array([0.0, 0.509, 0.491])
    out[:, 0, : ny // 2, :] = bottom[:, None, None]
    out[:, 0, ny // 2:, :] = top[:, None, None]
    return out


def loschmidt(nx: int = 200, ny: int = 200, *, t_end_hours: float = 1.0, samples: int = 200,
              d_max: float = 0.1, dtype=torch.float64) -> dict:
    """Sec. 4.3: dimensionless D12 = 0.2157, D13 = 0.7716, D23 = 0.8335 on
    [-1, 1]^2, no flux at y = +-1, periodic in x.  Returns times in hours and the
    bottom (y < 0) and top (y > 0) averages of xi_1, xi_2 (arrays [samples + 1, 2]),
    and the final xi profiles along y."""
    dx = 2.0 / ny
    pairs, dt = lattice_units({(1, 2): 0.2157, (1, 3): 0.7716, (2, 3): 0.8335}, dx, d_max)
    s = Solver("D2Q5", _pairs_matrix(3, pairs), (nx, ny), bc=(P, P, W, W, P, P), dtype=dtype)
    s.set_state(torch.from_numpy(loschmidt_initial(nx, ny)).to(dtype).to(s.device))
    total = int(round(t_end_hours * 3600.0 / LOSCHMIDT_T_REF_S / dt))
    marks = np.unique(np.round(np.linspace(0, total, samples + 1)).astype(np.int64))
    out = {"hours": [], "bottom": [], "top": [], "dt": dt}
    done = 0
    for m in marks:
        s.step(int(m - done))
        done = int(m)
        x = _host(s.moments())[:, 0]  # [n, ny, nx]
        half = ny // 2
        out["hours"].append(m * dt * LOSCHMIDT_T_REF_S / 3600.0)
        out["bottom"].append(x[:2, :half].mean(axis=(1, 2)))
        out["top"].append(x[:2, half:].mean(axis=(1, 2)))
    out["Y"] = -1.0 + (np.arange(ny) + 0.5) * dx
    out["final_profile"] = x[:, :, 0]
    for k in ("hours", "bottom", "top"):
        out[k] = np.asarray(out[k])
    return out
