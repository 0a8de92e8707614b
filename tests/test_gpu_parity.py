"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances (max-abs over all nodes and species): mole fractions 1e-12 in the
FP64 build and 2e-5 in the FP32 build; fluxes 1e-13 (FP64) and 1e-6 (FP32),
since |J| stays below ~1e-2 in these workloads and the FP32 flux carries the
rounding of the O(0.1) populations it is formed from.  Per-species mass drift
in FP32 must stay below 1e-6 relative.
"""

import math

import numpy as np
import pytest

import synthetic as sy

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")

TOL_X = {torch.float64: 1e-12, torch.float32: 2e-5}
TOL_J = {torch.float64: 1e-13, torch.float32: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1808_06787_gb300 as p

    p.load()


def gpu_run(lattice, D, x0, steps, *, bc="periodic", relax="magic", dtype=torch.float32,
            flux=True, chunked_steps=None):
    from paper_1808_06787_gb300 import Solver

    n, nz, ny, nx = x0.shape
    s = Solver(lattice, D, (nx, ny, nz), bc=bc, relax=relax, dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    if chunked_steps:
        for c in chunked_steps:
            s.step(c)
    else:
        s.step(steps)
    out = s.moments(flux=flux)
    x, J = out if flux else (out, None)
    res = dict(x=x.double().cpu().numpy(), mass=s.mass(), status=s.status(), solver=s)
    if flux:
        res["J"] = J.double().cpu().numpy()
    return res


def oracle_run(lattice, D, x0, steps, *, bc="periodic", relax="magic", flux=True):
    import oracle

    bcs = (bc,) * 6 if isinstance(bc, str) else bc
    return oracle.run(lattice, D, x0, steps, bc=bcs, relax=relax, flux=flux)


P, W = "periodic", "noflux"

SMALL = [
    # lattice, n, (nx, ny, nz), faces
    ("D2Q5", 3, (37, 23, 1), (P, P, P, P, P, P)),
    ("D2Q5", 2, (33, 5, 1), (W, W, P, P, P, P)),
    ("D2Q5", 8, (21, 17, 1), (P, P, W, W, P, P)),
    ("D2Q9", 5, (29, 19, 1), (P, P, W, W, P, P)),
    ("D2Q9", 4, (17, 16, 1), (W, W, W, W, P, P)),
    ("D2Q9", 7, (12, 10, 1), (P, P, P, P, P, P)),
    ("D3Q7", 3, (13, 11, 9), (W, W, W, W, W, W)),
    ("D3Q7", 4, (16, 9, 7), (P, P, W, W, W, W)),
    ("D3Q7", 2, (5, 4, 3), (P, P, P, P, P, P)),
    ("D3Q7", 6, (1, 1, 40), (P, P, P, P, W, W)),
    ("D2Q5", 3, (1, 1, 1), (P, P, P, P, P, P)),
    ("D3Q15", 3, (9, 7, 6), (W, W, P, P, W, W)),
    ("D3Q15", 5, (7, 6, 5), (P, P, P, P, P, P)),
    ("D3Q15", 2, (6, 5, 4), (W, W, W, W, W, W)),
    ("D1Q3", 4, (53, 1, 1), (W, W, P, P, P, P)),
    ("D1Q3", 8, (40, 1, 1), (P, P, P, P, P, P)),
    ("D2Q4", 3, (23, 17, 1), (W, W, P, P, P, P)),
    ("D2Q4", 6, (15, 12, 1), (P, P, P, P, P, P)),
    ("D3Q6", 3, (11, 9, 7), (W, W, W, W, W, W)),
    ("D3Q6", 4, (8, 7, 6), (P, P, W, W, P, P)),
]


def _small_input(lattice, n, dims, seed):
    nx, ny, nz = dims
    x0 = sy.sin_modes(n, nx, ny, nz, amp=0.1, seed=seed)
    D = sy.random_D(n, seed=seed + 1)
    return x0, D


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", SMALL, ids=lambda c: "%s-n%d-%dx%dx%d" % ((c[0], c[1]) + c[2]))
def test_parity_small_grids(case, dtype):
    lattice, n, dims, bc = case
    x0, D = _small_input(lattice, n, dims, 100 + n)
    steps = 301
    g = gpu_run(lattice, D, x0, steps, bc=bc, dtype=dtype)
    x, J = oracle_run(lattice, D, x0, steps, bc=bc)
    assert g["status"] == 0
    assert np.abs(g["x"] - x).max() <= TOL_X[dtype]
    assert np.abs(g["J"] - J).max() <= TOL_J[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("lattice", ["D2Q5", "D2Q9", "D3Q7"])
def test_parity_srt(lattice, dtype):
    dims = (19, 14, 6) if lattice == "D3Q7" else (31, 22, 1)
    x0, D = _small_input(lattice, 3, dims, 7)
    bc = (W, W, P, P, W, W)
    g = gpu_run(lattice, D, x0, 120, bc=bc, relax="srt", dtype=dtype)
    x, J = oracle_run(lattice, D, x0, 120, bc=bc, relax="srt")
    assert np.abs(g["x"] - x).max() <= TOL_X[dtype]
    assert np.abs(g["J"] - J).max() <= TOL_J[dtype]


def test_dilute_species_and_zero_composition():
    """Species that vanish on part of the domain (two-bulb) and a binary run."""
    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    x0 = sy.two_bulb(40, 6, 1, width=1.0)
    for dtype in (torch.float64, torch.float32):
        g = gpu_run("D2Q5", D, x0, 400, bc=(W, W, P, P, P, P), dtype=dtype)
        x, J = oracle_run("D2Q5", D, x0, 400, bc=(W, W, P, P, P, P))
        assert np.abs(g["x"] - x).max() <= TOL_X[dtype]
        assert np.abs(g["J"] - J).max() <= TOL_J[dtype]


def test_flux_is_zero_at_t0_and_time_levels():
    D = sy.random_D(3, seed=5)
    x0 = sy.sin_modes(3, 16, 12, amp=0.1, seed=6)
    for steps in (0, 1, 2):
        g = gpu_run("D2Q9", D, x0, steps, dtype=torch.float64)
        x, J = oracle_run("D2Q9", D, x0, steps)
        assert np.abs(g["x"] - x).max() <= 1e-14
        assert np.abs(g["J"] - J).max() <= 1e-15


def test_d2q5_fp64_128sq_full_size():
    """128 x 128 periodic ternary D2Q5, FP64, 2000 steps, seeded sine modes."""
    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    x0 = sy.sin_modes(3, 128, 128, amp=0.05, seed=1001)
    g = gpu_run("D2Q5", D, x0, 2000, dtype=torch.float64)
    x, J = oracle_run("D2Q5", D, x0, 2000)
    assert np.abs(g["x"] - x).max() <= 1e-12
    assert np.abs(g["J"] - J).max() <= 1e-13
    m0 = x0.sum(axis=(1, 2, 3))
    assert np.all(np.abs(g["mass"] - m0) <= 1e-12 * m0)


def test_d3q7_fp32_256cube_tube_full_size():
    """256^3 closed tube, FP32, 20000 steps: every node against the oracle's
    one-cell-wide run (x-only data stays y/z-uniform in a closed box)."""
    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    n = 256
    steps = 20000
    x0 = sy.two_bulb(n, n, n)
    from paper_1808_06787_gb300 import Solver

    s = Solver("D3Q7", D, (n, n, n), bc="noflux", dtype=torch.float32)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    s.step(steps)
    x = s.moments()
    ref = oracle_run("D3Q7", D, sy.two_bulb(n, 1, 1), steps, bc="noflux", flux=False)
    err = (x.double() - torch.from_numpy(ref).cuda()).abs().max().item()
    assert err <= 2e-5, err
    m1 = s.mass()
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0) + 1e-9), (m0, m1)
    assert s.status() == 0
    # the middle species was uniform and shows reverse/osmotic diffusion
    mid = ref[1, 0, 0]
    assert mid.max() - mid.min() > 1e-3


def _window_oracle(lattice, D, x0, cx, cy, T):
    """Oracle value at (cx, cy) after T steps, from a periodic window that holds
    the whole dependency cone of that node."""
    w = 2 * T + 3
    n, _, ny, nx = x0.shape
    ix = (np.arange(w) - w // 2 + cx) % nx
    iy = (np.arange(w) - w // 2 + cy) % ny
    win = x0[:, :, iy][:, :, :, ix]
    x = oracle_run(lattice, D, win, T, flux=False)
    return x[:, 0, w // 2, w // 2]


def test_d2q9_fp32_2048sq_n5_full_size():
    """2048^2 periodic D2Q9, N = 5, FP32: sampled nodes after 12 steps against the
    oracle on their dependency cones; mass, closure and flags after 10000 steps."""
    n = 5
    D = sy.random_D(n, seed=1003)
    x0 = sy.gaussian_blobs(n, 2048, 2048, seed=1003)
    from paper_1808_06787_gb300 import Solver

    s = Solver("D2Q9", D, (2048, 2048, 1), dtype=torch.float32)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    T = 12
    s.step(T)
    x = s.moments().double().cpu().numpy()
    g = sy.rng(77)
    pts = [(0, 0), (2047, 2047), (1024, 0)] + [tuple(g.integers(0, 2048, size=2)) for _ in range(6)]
    for (cx, cy) in pts:
        ref = _window_oracle("D2Q9", D, x0, int(cx), int(cy), T)
        assert np.abs(x[:, 0, cy, cx] - ref).max() <= 2e-6
    s.step(10000 - T)
    xt = s.moments()
    assert (xt.double().sum(dim=0) - 1.0).abs().max().item() <= 1e-6
    m1 = s.mass()
    assert np.all(np.abs(m1 - m0) <= 1e-6 * np.abs(m0)), (m0, m1)
    assert s.status() == 0


def test_host_buffers_match_device_buffers():
    """Pageable host inputs/outputs go through the chunked staging path (the
    fields here exceed the 16 MiB staging area, so several chunks are used);
    pinned host buffers are read and written by the kernels in place; results
    equal the device path bit for bit."""
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(3, seed=9)
    x0 = sy.sin_modes(3, 1024, 1000, amp=0.05, seed=10)
    x0t = torch.from_numpy(x0)
    a = Solver("D2Q5", D, (1024, 1000), dtype=torch.float64)
    a.set_state(x0t.cuda())
    a.step(7)
    xa, Ja = a.moments(flux=True)
    b = Solver("D2Q5", D, (1024, 1000), dtype=torch.float64)
    b.set_state(x0t.clone())  # pageable host
    b.step(7)
    xb = torch.empty(b.field_shape, dtype=torch.float64).pin_memory()
    Jb = torch.empty(b.flux_shape, dtype=torch.float64)
    b.moments(xb, Jb)
    assert torch.equal(xa.cpu(), xb) and torch.equal(Ja.cpu(), Jb)
    c = Solver("D2Q5", D, (1024, 1000), dtype=torch.float64)
    c.set_state(x0t.clone().pin_memory())
    c.step(7)
    xc = c.moments()
    assert torch.equal(xa, xc)
    xp = torch.empty(c.field_shape, dtype=torch.float64).pin_memory()
    Jp = torch.empty(c.flux_shape, dtype=torch.float64).pin_memory()
    c.moments(xp, Jp)  # both outputs pinned: written by the moments kernel in place
    assert torch.equal(xa.cpu(), xp) and torch.equal(Ja.cpu(), Jp)
    # a pinned input may be overwritten as soon as set_state returns
    x0p = x0t.clone().pin_memory()
    d = Solver("D2Q5", D, (1024, 1000), dtype=torch.float64)
    d.set_state(x0p)
    x0p.fill_(0.0)
    d.step(7)
    assert torch.equal(xa, d.moments())


def test_graph_replay_equals_single_steps_and_is_deterministic():
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(4, seed=3)
    x0 = torch.from_numpy(sy.sin_modes(4, 40, 30, amp=0.1, seed=4)).float().cuda()
    a = Solver("D2Q9", D, (40, 30), bc=(W, W, P, P, P, P))
    a.set_state(x0)
    a.step(101)  # graph replays of 32 steps plus single launches
    b = Solver("D2Q9", D, (40, 30), bc=(W, W, P, P, P, P))
    b.set_state(x0)
    for _ in range(101):
        b.step(1)
    assert a.steps_done == b.steps_done == 101
    assert torch.equal(a.moments(), b.moments())
    ma, mb = a.mass(), b.mass()
    assert np.array_equal(ma, mb)
    assert np.array_equal(a.mass(), ma)


@pytest.mark.parametrize("lattice,grid,n", [("D2Q9", (40, 30), 4), ("D2Q5", (2048, 1024), 3),
                                            ("D3Q7", (128, 128, 128), 3), ("D2Q9", (512, 384), 5)])
def test_call_graphs_equal_single_steps(lattice, grid, n):
    """Calls of up to 64 steps replay one graph per (length, buffer parity), the
    four most recent kept; longer calls take the 32/16/8/4/2-step graphs.  A
    sequence of calls of mixed lengths (cache hits from both parities, evictions,
    lengths above 64, single steps) equals the same number of single steps bit
    for bit, fields and masses, on the one-node and the two-nodes-per-thread
    kernels (the 2^21-node grids)."""
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(n, seed=31)
    nx, ny = grid[0], grid[1]
    nz = grid[2] if len(grid) == 3 else 1
    x0 = sy.sin_modes(n, nx, ny, amp=0.1, seed=32) if nz == 1 else sy.two_bulb(nx, ny, nz, width=4.0)
    x0 = torch.from_numpy(x0).float().cuda()
    bc = (W, W, P, P, P, P)
    calls = [5, 20, 3, 64, 7, 20, 11, 2, 33, 64, 20, 65, 1, 6, 20]
    a = Solver(lattice, D, grid, bc=bc)
    a.set_state(x0)
    for c in calls:
        a.step(c)
    b = Solver(lattice, D, grid, bc=bc)
    b.set_state(x0)
    for _ in range(sum(calls)):
        b.step(1)
    assert a.steps_done == b.steps_done == sum(calls)
    assert torch.equal(a.moments(), b.moments())
    assert np.array_equal(a.mass(), b.mass())
    assert a.status() == b.status() == 0


def test_call_graphs_follow_a_new_reference_composition():
    """The captured graphs hold the kernel arguments: changing the frozen
    mode's reference composition between two calls of the same length must
    take effect in the second call."""
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(3, seed=33)
    x0 = torch.from_numpy(sy.sin_modes(3, 48, 40, amp=0.05, seed=34)).double().cuda()
    ref1 = np.array([0.3, 0.3, 0.4])
    ref2 = np.array([0.5, 0.2, 0.3])

    def run(single):
        s = Solver("D2Q5", D, (48, 40), dtype=torch.float64, relax="frozen")
        s.set_state(x0)
        for ref in (ref1, ref2):
            s.set_reference(ref)
            if single:
                for _ in range(20):
                    s.step(1)
            else:
                s.step(20)
        return s.moments()

    assert torch.equal(run(False), run(True))


def test_mass_matches_field_sum():
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(5, seed=12)
    x0 = sy.gaussian_blobs(5, 300, 200, sigma=9, seed=13)
    s = Solver("D2Q9", D, (300, 200), dtype=torch.float64)
    s.set_state(torch.from_numpy(x0).cuda())
    m_init = s.mass()  # standalone mass kernel
    np.testing.assert_allclose(m_init, x0.sum(axis=(1, 2, 3)), rtol=1e-13)
    s.step(50)
    m_fused = s.mass()  # partials written by the last step
    x = s.moments().cpu().numpy()
    np.testing.assert_allclose(m_fused, x.sum(axis=(1, 2, 3)), rtol=1e-12)
    np.testing.assert_allclose(m_fused, m_init, rtol=1e-12)


def test_mass_fp32_fixed_point_is_exact_to_its_resolution():
    """FP32 masses are exact sums of the nodes' values rounded to 2^-k, so they
    match an FP64 sum of the FP32 moments within cells * 2^-(k+1)."""
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(4, seed=21)
    x0 = sy.gaussian_blobs(4, 512, 384, sigma=20, seed=22)
    s = Solver("D2Q9", D, (512, 384), bc=(P, P, W, W, P, P))
    s.set_state(torch.from_numpy(x0).float().cuda())
    cells = 512 * 384
    k = 59 - math.ceil(math.log2(cells))
    for steps in (0, 37):
        s.step(steps)
        m = s.mass()
        x = s.moments().double()
        # the mass uses xi = sum_k f_k; the moments kernel computes the same sums
        ref = x.sum(dim=(1, 2, 3)).cpu().numpy()
        assert np.all(np.abs(m - ref) <= cells * 2.0 ** -(k + 1) + 1e-9 * np.abs(ref))
        assert np.array_equal(s.mass(), m)


def test_status_flags():
    from paper_1808_06787_gb300 import Solver, lbms

    D = sy.random_D(3, seed=2)
    x0 = sy.sin_modes(3, 16, 16, amp=0.05, seed=2)
    bad = x0.copy()
    bad[0, 0, 3, 3] += 0.01
    s = Solver("D2Q5", D, (16, 16))
    s.set_state(torch.from_numpy(bad).float().cuda())
    assert s.status() & lbms.FLAG_INIT
    s.set_state(torch.from_numpy(x0).float().cuda())
    assert s.status() == 0
    nan = x0.copy()
    nan[1, 0, 5, 7] = np.nan
    s.set_state(torch.from_numpy(nan).float().cuda())
    s.step(3)
    fl = s.status()
    assert fl & lbms.FLAG_INIT and fl & lbms.FLAG_NONFINITE


def test_invalid_calls_report_errors():
    from paper_1808_06787_gb300 import LbmsError, Solver

    D = sy.random_D(3, seed=2)
    s = Solver("D2Q5", D, (8, 8))
    with pytest.raises(LbmsError):
        s.step(-1)
    with pytest.raises(ValueError):
        s.set_state(torch.zeros((3, 1, 8, 9), device="cuda"))


# Local gradients of Eq. xix: grad = -D~^{-1} J, so the flux tolerances scale
# by 1 / min D_ij (0.01 for the seeded diffusivities): 1e-11 (FP64), 1e-4 (FP32).
TOL_G = {torch.float64: 1e-11, torch.float32: 1e-4}


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", SMALL[:9] + SMALL[11:14] + SMALL[16:], ids=lambda c: "%s-n%d-%dx%dx%d" % ((c[0], c[1]) + c[2]))
def test_gradient_parity(case, dtype):
    import oracle

    from paper_1808_06787_gb300 import Solver

    lattice, n, dims, bc = case
    x0, D = _small_input(lattice, n, dims, 500 + n)
    steps = 123
    s = Solver(lattice, D, dims, bc=bc, dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    assert float(s.gradient().abs().max()) == 0.0  # t = 0: no gradient yet
    s.step(steps)
    G = s.gradient().double().cpu().numpy()
    host = torch.empty(s.flux_shape, dtype=dtype).pin_memory()
    s.gradient(out=host)
    _, Jo, Go = oracle.run(lattice, D, x0, steps, bc=bc, flux=True, grad=True)
    assert np.abs(G - Go).max() <= TOL_G[dtype]
    assert np.array_equal(host.double().numpy(), G)
    # the species' gradients close to zero, and J = -D~ grad node by node is
    # checked through the oracle's own flux
    assert np.abs(G.sum(axis=0)).max() <= 10 * TOL_G[dtype]
    x, J = s.moments(flux=True)
    assert np.abs(J.double().cpu().numpy() - Jo).max() <= TOL_J[dtype]


def test_population_view_follows_raw_state_loads():
    """Solver.populations() views the current buffer, also after a raw load at an
    odd step count (lbms_populations)."""
    from paper_1808_06787_gb300 import Solver

    dims = (12, 10, 1)
    s = Solver("D2Q5", sy.random_D(3, seed=3), dims, dtype=torch.float64)
    s.set_state(torch.from_numpy(sy.sin_modes(3, *dims, amp=0.1, seed=4)).cuda())
    s.step(3)
    f = s.get_state()
    s.set_state_raw(f, 7)
    assert torch.equal(s.populations().reshape(f.shape), f)
    s.step(1)
    assert torch.equal(s.populations().reshape(f.shape), s.get_state())


def test_d3q15_tube_full_size_window():
    """D3Q15 256^3 closed ternary tube (bench workload `tube15`), FP32: after T steps
    the nodes near the interface depend only on nodes within T cells along x, so
    the oracle on an x-window of the full y-z cross-section gives them exactly."""
    from paper_1808_06787_gb300 import Solver
    import oracle

    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    N, T, half = 256, 24, 40
    s = Solver("D3Q15", D, (N, N, N), bc="noflux", dtype=torch.float32)
    x0 = sy.two_bulb(N, N, N, width=4.0)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    s.step(T)
    x = s.moments()[:, :, :, N // 2 - 8:N // 2 + 8].double().cpu().numpy()
    # the window's own faces (no-flux) are more than T cells from the compared nodes
    win = x0[:, :, :, N // 2 - half:N // 2 + half]
    ref = oracle.run("D3Q15", D, win, T, bc=("noflux",) * 6)[:, :, :, half - 8:half + 8]
    assert np.abs(x - ref).max() <= 2e-5
    assert np.all(np.abs(s.mass() - m0) <= 1e-6 * np.abs(m0))
    assert s.status() == 0


def test_d1q3_line_full_size_window():
    """D1Q3 line of 2^26 nodes (bench workload `line`), FP32: the interface region
    after T steps against the oracle on a window of 2T + 128 nodes, and mass."""
    from paper_1808_06787_gb300 import Solver
    import oracle

    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    N, T = 1 << 26, 500
    s = Solver("D1Q3", D, (N, 1, 1), bc=("noflux", "noflux") + ("periodic",) * 4,
               dtype=torch.float32)
    x0 = sy.two_bulb(N, 1, 1, width=4.0)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    s.step(T)
    half = T + 64
    x = s.moments()[:, :, :, N // 2 - 32:N // 2 + 32].double().cpu().numpy()
    win = x0[:, :, :, N // 2 - half:N // 2 + half]
    ref = oracle.run("D1Q3", D, win, T, bc=("noflux", "noflux") + ("periodic",) * 4)
    assert np.abs(x - ref[:, :, :, half - 32:half + 32]).max() <= 2e-5
    assert np.all(np.abs(s.mass() - m0) <= 1e-6 * np.abs(m0))
    assert s.status() == 0


def test_d3q6_tube_full_size_window():
    """D3Q6 256^3 closed ternary tube (bench workload `tube6`, no rest velocity),
    FP32: the interface region after T steps against the oracle on an x-window of
    the full y-z cross-section (a node depends only on nodes within T cells), and mass."""
    from paper_1808_06787_gb300 import Solver
    import oracle

    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    N, T, half = 256, 24, 40
    s = Solver("D3Q6", D, (N, N, N), bc="noflux", dtype=torch.float32)
    x0 = sy.two_bulb(N, N, N, width=4.0)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    s.step(T)
    x = s.moments()[:, :, :, N // 2 - 8:N // 2 + 8].double().cpu().numpy()
    win = x0[:, :, :, N // 2 - half:N // 2 + half]
    ref = oracle.run("D3Q6", D, win, T, bc=("noflux",) * 6)[:, :, :, half - 8:half + 8]
    assert np.abs(x - ref).max() <= 2e-5
    assert np.all(np.abs(s.mass() - m0) <= 1e-6 * np.abs(m0))
    assert s.status() == 0


def test_d2q4_plane_full_size_window():
    """D2Q4 8192^2 ternary two-bulb plane (bench workload `plane4`, no rest velocity;
    no-flux x faces, periodic y), FP32: the interface region after T steps against
    the oracle on an x-window of all 8192 rows, and mass."""
    from paper_1808_06787_gb300 import Solver
    import oracle

    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    N, T, half = 8192, 24, 40
    bc = ("noflux", "noflux") + ("periodic",) * 4
    s = Solver("D2Q4", D, (N, N, 1), bc=bc, dtype=torch.float32)
    x0 = sy.two_bulb(N, N, 1, width=4.0)
    s.set_state(torch.from_numpy(x0).float().cuda())
    m0 = s.mass()
    s.step(T)
    x = s.moments()[:, :, :, N // 2 - 8:N // 2 + 8].double().cpu().numpy()
    win = x0[:, :, :, N // 2 - half:N // 2 + half]
    ref = oracle.run("D2Q4", D, win, T, bc=bc)[:, :, :, half - 8:half + 8]
    assert np.abs(x - ref).max() <= 2e-5
    assert np.all(np.abs(s.mass() - m0) <= 1e-6 * np.abs(m0))
    assert s.status() == 0


FROZEN_CASES = [
    ("D2Q5", 3, (24, 18, 1), (P, P, W, W, P, P)),
    ("D2Q9", 4, (17, 13, 1), (P, P, P, P, P, P)),
    ("D3Q7", 3, (11, 9, 7), (W, W, P, P, W, W)),
    ("D3Q15", 3, (8, 7, 6), (P, P, P, P, P, P)),
    ("D1Q3", 5, (41, 1, 1), (W, W, P, P, P, P)),
    ("D2Q4", 3, (20, 14, 1), (W, W, P, P, P, P)),
    ("D3Q6", 3, (9, 8, 7), (P, P, P, P, W, W)),
]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", FROZEN_CASES, ids=lambda c: "%s-n%d" % (c[0], c[1]))
def test_frozen_mode_parity(case, dtype):
    """LBMS_RELAX_FROZEN (relaxation matrices at a fixed reference composition)
    against the oracle's frozen mode: fields, fluxes and gradients."""
    import oracle

    from paper_1808_06787_gb300 import LbmsError, Solver

    lattice, n, dims, bc = case
    x0, D = _small_input(lattice, n, dims, 700 + n)
    xref = np.full(n, 1.0 / n)
    s = Solver(lattice, D, dims, bc=bc, relax="frozen", dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    with pytest.raises(LbmsError, match="set_reference"):
        s.step(1)
    s.set_reference(xref)
    s.step(211)
    x, J = s.moments(flux=True)
    G = s.gradient()
    xo, Jo, Go = oracle.run(lattice, D, x0, 211, bc=bc, relax="frozen", xi_ref=xref,
                            flux=True, grad=True)
    assert np.abs(x.double().cpu().numpy() - xo).max() <= TOL_X[dtype]
    assert np.abs(J.double().cpu().numpy() - Jo).max() <= TOL_J[dtype]
    assert np.abs(G.double().cpu().numpy() - Go).max() <= TOL_G[dtype]
    assert s.status() == 0
    with pytest.raises(LbmsError):
        s.set_reference(np.full(n, 0.5))  # does not sum to one
    assert s.adjoint_scratch is not None
    with pytest.raises(LbmsError, match="adjoint"):
        s.adjoint_scratch()
