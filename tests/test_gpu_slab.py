"""Slab decomposition on one GPU: a grid split into slabs along its split axis
(each slab a handle with LBMS_HALO cut faces, halo exchange by device copies in
lbms_slab_step) evolves bit for bit as the undivided grid -- mole fractions,
fluxes and local gradients, FP32 (stochastic rounding keyed by the node's global
index) and FP64 -- and matches the oracle at the parity tolerances.  Cases cover
every lattice, closed, wrapping and Dirichlet split axes, walls and periodic
faces on the other axes (diagonal links that cross a cut and a wrap or a wall
at once), and slabs one layer thick.
"""

import numpy as np
import pytest

import synthetic as sy

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")

P, W, DI = "periodic", "noflux", "dirichlet"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [
    # lattice, n, grid, faces, parts
    ("D3Q7", 3, (13, 11, 12), (P, P, W, W, W, W), 2),
    ("D3Q7", 3, (13, 11, 12), (W, W, P, P, P, P), 3),
    ("D3Q7", 4, (9, 8, 3), (P, P, P, P, P, P), 3),  # slabs of one layer, wrapping
    ("D2Q9", 4, (17, 23, 1), (P, P, P, P, P, P), 3),
    ("D2Q9", 5, (19, 16, 1), (W, W, W, W, P, P), 2),
    ("D2Q5", 3, (20, 18, 1), (P, P, W, W, P, P), 4),
    ("D3Q15", 3, (7, 6, 9), (W, W, P, P, P, P), 2),
    ("D3Q15", 2, (6, 7, 8), (P, P, W, W, W, W), 3),
    ("D1Q3", 3, (41, 1, 1), (W, W, P, P, P, P), 3),
    ("D1Q3", 5, (30, 1, 1), (P, P, P, P, P, P), 2),
    ("D2Q4", 3, (15, 14, 1), (W, W, P, P, P, P), 2),
    ("D3Q6", 3, (8, 7, 10), (P, P, W, W, W, W), 2),
]


def _run_pair(lattice, n, grid, bc, parts, dtype, steps, boundary=None):
    from paper_1808_06787_gb300 import SlabSolver, Solver

    D = sy.random_D(n, seed=300 + n)
    x0 = sy.sin_modes(n, *grid, amp=0.1, seed=310 + n)
    whole = Solver(lattice, D, grid, bc=bc, dtype=dtype, boundary=boundary)
    whole.set_state(torch.from_numpy(x0).to(dtype).cuda())
    slabs = SlabSolver(lattice, D, grid, parts, bc=bc, dtype=dtype, boundary=boundary)
    slabs.set_state(torch.from_numpy(x0).to(dtype).cuda())
    whole.step(steps)
    slabs.step(steps)
    return D, x0, whole, slabs


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-n%d-%dx%dx%d-p%d" % ((c[0], c[1]) + c[2] + (c[4],)))
def test_slabs_equal_the_undivided_grid_bit_for_bit(case, dtype):
    lattice, n, grid, bc, parts = case
    _, _, whole, slabs = _run_pair(lattice, n, grid, bc, parts, dtype, 57)
    assert slabs.steps_done == whole.steps_done == 57
    xw, Jw = whole.moments(flux=True)
    xs, Js = slabs.moments(flux=True)
    assert torch.equal(xs, xw)
    assert torch.equal(Js, Jw)
    assert torch.equal(slabs.gradient(), whole.gradient())
    mw, ms = whole.mass(), slabs.mass()
    tol = 1e-13 if dtype == torch.float64 else 1e-9
    assert np.all(np.abs(ms - mw) <= tol * np.abs(mw) + 1e-12), (ms, mw)
    assert slabs.status() == 0 and whole.status() == 0


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_slabs_with_dirichlet_ends_equal_the_undivided_grid(dtype):
    """A split axis closed by two Dirichlet faces (held by the end slabs)."""
    bnd = {2: [0.2, 0.5, 0.3], 3: [0.5, 0.25, 0.25]}
    _, _, whole, slabs = _run_pair("D2Q5", 3, (16, 21, 1), (P, P, DI, DI, P, P), 3, dtype, 40,
                                   boundary=bnd)
    xw, Jw = whole.moments(flux=True)
    xs, Js = slabs.moments(flux=True)
    assert torch.equal(xs, xw) and torch.equal(Js, Jw)


@pytest.mark.parametrize("dtype,tol_x,tol_j", [(torch.float32, 2e-5, 1e-6), (torch.float64, 1e-12, 1e-13)],
                         ids=["f32", "f64"])
def test_slabs_match_the_oracle(dtype, tol_x, tol_j):
    import oracle

    lattice, n, grid, bc = "D2Q9", 4, (23, 26, 1), (W, W, P, P, P, P)
    D, x0, _, slabs = _run_pair(lattice, n, grid, bc, 3, dtype, 301)
    x, J = slabs.moments(flux=True)
    xo, Jo = oracle.run(lattice, D, x0, 301, bc=bc, flux=True)
    assert np.abs(x.double().cpu().numpy() - xo).max() <= tol_x
    assert np.abs(J.double().cpu().numpy() - Jo).max() <= tol_j
    m0 = x0.sum(axis=(1, 2, 3))
    assert np.all(np.abs(slabs.mass() - m0) <= 1e-6 * m0)


def test_halo_buffers_and_errors():
    from paper_1808_06787_gb300 import LbmsError, SlabSolver, Solver
    from paper_1808_06787_gb300.lbms import lbms_slab_step

    D = sy.random_D(3, seed=5)
    slabs = SlabSolver("D3Q15", D, (6, 5, 8), 2, bc=(P, P, W, W, W, W))
    slabs.set_state(torch.from_numpy(sy.sin_modes(3, 6, 5, 8, amp=0.1, seed=6)).float().cuda())
    lower = slabs.slabs[0]
    send, recv = lower.halo_buffers(5)  # the lower slab's top face is a cut
    assert tuple(send.shape) == (5, 2, 30) and tuple(recv.shape) == (5, 2, 30)
    # set_state packed the send buffer: the top layer's upward populations
    f = lower.get_state().view(2, 15, 4, 5, 6)
    up = [k for k in range(15) if k in (5, 7, 10, 11, 13)]  # c_z = +1 in the device order
    for j, k in enumerate(up):
        assert torch.equal(send[j], f[:, k, 3].reshape(2, 30))
    with pytest.raises(LbmsError, match="not an LBMS_HALO face"):
        lower.halo_buffers(4)  # the grid's own wall
    with pytest.raises(LbmsError, match="one step per call"):
        lower.step(2)
    # slabs that are not neighbours of one grid
    other = Solver("D3Q15", D, (6, 5, 4), bc=(P, P, W, W, W, W))
    with pytest.raises(LbmsError, match="pair of cuts"):
        lbms_slab_step([lower._h, other._h], 1)
    with pytest.raises(LbmsError):
        lower.set_state_raw(lower.get_state(), 0)
    slabs.step(3)
    assert slabs.status() == 0
