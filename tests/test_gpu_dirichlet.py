"""Dirichlet faces (half-way anti-bounce-back, Sec. 4) on the GPU, through the C ABI.

1. Parity with the FP64 oracle on small grids of every lattice, with Dirichlet
   faces mixed with no-flux and periodic ones (D2Q9 corners included), in both
   relaxation modes: mole fractions 1e-12 (FP64) / 2e-5 (FP32), fluxes
   1e-13 / 1e-6.
2. The two-component erf problem of Sec. 4.1 at its full 240 x 40 size: the
   GPU reproduces the oracle's fields and the errors of Table I.
3. Properties at any size: the exact linear steady state between two walls,
   and a composition changed between steps takes effect in stream order.
4. One adjoint step with Dirichlet faces is the transpose of the step's
   derivative (the anti-bounce-back enters with a factor -1).
5. Argument checks that need a live handle.
"""

import numpy as np
import pytest

import synthetic as sy

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")

TOL_X = {torch.float64: 1e-12, torch.float32: 2e-5}
TOL_J = {torch.float64: 1e-13, torch.float32: 1e-6}
P, W, B = "periodic", "noflux", "dirichlet"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1808_06787_gb300 as p

    p.load()


def _compositions(n, seed):
    g = sy.rng(seed)
    xb = g.uniform(0.05, 1.0, size=(6, n))
    return xb / xb.sum(axis=1, keepdims=True)


def _boundary(bc, xb):
    return {f: xb[f] for f in range(6) if bc[f] == B}


def gpu_run(lattice, D, x0, steps, bc, xb, *, relax="magic", dtype=torch.float64):
    from paper_1808_06787_gb300 import Solver

    n, nz, ny, nx = x0.shape
    s = Solver(lattice, D, (nx, ny, nz), bc=bc, relax=relax, dtype=dtype,
               boundary=_boundary(bc, xb))
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    s.step(steps)
    x, J = s.moments(flux=True)
    return x.double().cpu().numpy(), J.double().cpu().numpy(), s


CASES = [
    # lattice, n, (nx, ny, nz), faces
    ("D2Q5", 2, (33, 5, 1), (B, B, P, P, P, P)),
    ("D2Q5", 3, (24, 19, 1), (B, W, B, B, P, P)),
    ("D2Q9", 3, (21, 17, 1), (B, B, P, P, P, P)),
    ("D2Q9", 5, (19, 13, 1), (B, B, W, B, P, P)),
    ("D2Q9", 4, (11, 9, 1), (B, B, B, B, P, P)),
    ("D3Q7", 3, (13, 9, 7), (B, B, W, W, B, W)),
    ("D3Q7", 4, (9, 8, 10), (P, P, P, P, B, B)),
    ("D3Q15", 3, (9, 7, 6), (B, B, W, W, B, W)),
    ("D1Q3", 3, (40, 1, 1), (B, B, P, P, P, P)),
    ("D2Q4", 3, (22, 15, 1), (B, W, B, B, P, P)),
    ("D3Q6", 3, (9, 8, 7), (B, B, W, W, B, W)),
]


@pytest.mark.parametrize("relax", ["magic", "srt"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-n%d-%dx%dx%d" % ((c[0], c[1]) + c[2]))
def test_parity_dirichlet(case, dtype, relax):
    import oracle

    lattice, n, dims, bc = case
    x0 = sy.sin_modes(n, *dims, amp=0.1, seed=300 + n)
    D = sy.random_D(n, seed=301 + n)
    xb = _compositions(n, 302 + n)
    steps = 257
    x, J, s = gpu_run(lattice, D, x0, steps, bc, xb, relax=relax, dtype=dtype)
    xo, Jo = oracle.run(lattice, D, x0, steps, bc=bc, relax=relax, flux=True, xb=xb)
    assert s.status() == 0
    assert np.abs(x - xo).max() <= TOL_X[dtype]
    assert np.abs(J - Jo).max() <= TOL_J[dtype]


def _erf_case(lam1):
    import theory as th

    Pn = th.golden_numbers()
    nx, ny = int(Pn["erf.nx"]), int(Pn["erf.ny"])
    Dp, C0, C1 = Pn["erf.D"], Pn["erf.C0"], Pn["erf.C1"]
    dx = 12.0 / nx
    Dl = (1.0 / lam1 - 0.5) / 3.0
    dt = Dl * dx * dx / Dp
    D = np.array([[1.0, Dl], [Dl, 1.0]])
    xb = np.zeros((6, 2))
    xb[0] = (C0, 1.0 - C0)
    xb[1] = (C1, 1.0 - C1)
    x0 = sy.erf_step(nx, ny, C0=C0, C1=C1)
    X = -6.0 + (np.arange(nx) + 0.5) * dx
    return Pn, D, xb, x0, X, dx, dt


@pytest.mark.parametrize("relax,tag", [("magic", "mrt"), ("srt", "srt")])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32], ids=["f64", "f32"])
def test_table_I_on_the_gpu(relax, tag, dtype):
    """Sec. 4.1 on 240 x 40: fields equal the oracle's; errors as in Table I."""
    import oracle
    import theory as th

    from paper_1808_06787_gb300 import Solver

    Pn, D, xb, x0, X, dx, dt = _erf_case(1.25)
    bc = (B, B, P, P, P, P)
    s = Solver("D2Q5", D, (x0.shape[3], x0.shape[2]), bc=bc, relax=relax, dtype=dtype,
               boundary={0: xb[0], 1: xb[1]})
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    done = 0
    for t in (1, 5, 20):
        steps = int(round(t / dt))
        s.step(steps - done)
        done = steps
        x, J = s.moments(flux=True)
        x = x.double().cpu().numpy()
        J = J.double().cpu().numpy()
        xo, Jo = oracle.run("D2Q5", D, x0[:, :, :1], steps, bc=bc, relax=relax, flux=True, xb=xb)
        assert np.abs(x - xo).max() <= TOL_X[dtype]
        assert np.abs(J - Jo).max() <= TOL_J[dtype]
        xa, Ja = th.erf_solution(X, steps * dt, Pn["erf.D"], Pn["erf.C0"], Pn["erf.C1"])
        Ex = th.rel_l2(np.broadcast_to(xa, x[0, 0].shape), x[0, 0])
        EJ = th.rel_l2(np.broadcast_to(Ja, x[0, 0].shape), J[0, 0, 0] * dx / dt)
        if dtype == torch.float64:
            assert Ex == pytest.approx(Pn["erf.%s.Ex.t%d" % (tag, t)], rel=3e-3)
            assert EJ == pytest.approx(Pn["erf.%s.EJ.t%d" % (tag, t)], rel=3e-3)
        else:  # FP32 rounding (~1e-7 per node) adds little to the discretisation error
            assert abs(Ex - Pn["erf.%s.Ex.t%d" % (tag, t)]) <= 1e-6
    assert s.status() == 0


def test_second_order_convergence_on_the_gpu():
    """Figs. 3 and 4: errors at t = 5 for dx = 1/10 .. 1/40 fall with slope 2."""
    import theory as th

    from paper_1808_06787_gb300 import Solver

    Pn = th.golden_numbers()
    Dp, C0, C1 = Pn["erf.D"], Pn["erf.C0"], Pn["erf.C1"]
    lam1 = 1.25
    errs = []
    nxs = (120, 240, 360, 480)
    for nx in nxs:
        dx = 12.0 / nx
        Dl = (1.0 / lam1 - 0.5) / 3.0
        dt = Dl * dx * dx / Dp
        steps = int(round(5.0 / dt))
        s = Solver("D2Q5", np.array([[1.0, Dl], [Dl, 1.0]]), (nx, 4), bc=(B, B, P, P, P, P),
                   dtype=torch.float64, boundary={0: (C0, 1 - C0), 1: (C1, 1 - C1)})
        s.set_state(torch.from_numpy(sy.erf_step(nx, 4, C0=C0, C1=C1)).cuda())
        s.step(steps)
        x, J = s.moments(flux=True)
        X = -6.0 + (np.arange(nx) + 0.5) * dx
        xa, Ja = th.erf_solution(X, steps * dt, Dp, C0, C1)
        errs.append((th.rel_l2(xa, x[0, 0, 1].cpu().numpy()),
                     th.rel_l2(Ja, J[0, 0, 0, 1].cpu().numpy() * dx / dt)))
    logdx = np.log([12.0 / n for n in nxs])
    for comp in (0, 1):
        slope = np.polyfit(logdx, np.log([e[comp] for e in errs]), 1)[0]
        assert abs(slope - Pn["erf.convergence_slope"]) < 0.05


@pytest.mark.parametrize("lattice,dims", [("D2Q5", (16, 3, 1)), ("D2Q9", (16, 3, 1)),
                                          ("D3Q7", (16, 2, 2)), ("D3Q15", (16, 2, 2)),
                                          ("D1Q3", (16, 1, 1)), ("D2Q4", (16, 3, 1)),
                                          ("D3Q6", (16, 2, 2))])
def test_linear_steady_state_and_stream_ordered_boundary_change(lattice, dims):
    from paper_1808_06787_gb300 import Solver

    nx = dims[0]
    Dl = 0.07
    D = np.array([[1.0, Dl], [Dl, 1.0]])
    bc = (B, B, P, P, P, P)
    s = Solver(lattice, D, dims, bc=bc, dtype=torch.float64,
               boundary={0: (0.9, 0.1), 1: (0.2, 0.8)})
    x0 = np.full((2, dims[2], dims[1], nx), 0.5)
    s.set_state(torch.from_numpy(x0).cuda())
    s.step(40000)
    X = (np.arange(nx) + 0.5) / nx
    x, J = s.moments(flux=True)
    x = x.cpu().numpy()
    np.testing.assert_allclose(x[0], np.broadcast_to(0.9 - 0.7 * X, x[0].shape), rtol=0, atol=1e-12)
    np.testing.assert_allclose(J[0, 0].cpu().numpy(), Dl * 0.7 / nx, rtol=1e-10, atol=0)
    # new composition on the high face; queued steps see it in stream order
    s.set_boundary(1, (0.6, 0.4))
    s.step(40000)
    x = s.moments().cpu().numpy()
    np.testing.assert_allclose(x[0], np.broadcast_to(0.9 - 0.3 * X, x[0].shape), rtol=0, atol=1e-12)


@pytest.mark.parametrize("lattice,n,dims,bc", [
    ("D2Q5", 3, (21, 13, 1), (B, B, P, P, P, P)),
    ("D2Q9", 4, (17, 11, 1), (B, W, B, B, P, P)),
    ("D3Q7", 3, (9, 7, 6), (B, B, W, W, B, B)),
    ("D3Q15", 3, (7, 6, 5), (B, B, W, W, P, P)),
    ("D1Q3", 2, (30, 1, 1), (B, W, P, P, P, P)),
    ("D2Q4", 3, (16, 12, 1), (B, B, W, W, P, P)),
    ("D3Q6", 3, (8, 7, 6), (P, P, B, W, B, B)),
])
def test_adjoint_step_with_dirichlet_faces_is_a_transpose(lattice, n, dims, bc):
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(n, seed=71 + n)
    xb = _compositions(n, 72 + n)
    kw = dict(bc=bc, dtype=torch.float64, boundary=_boundary(bc, xb))
    s = Solver(lattice, D, dims, **kw)
    s.set_state(torch.from_numpy(sy.sin_modes(n, *dims, amp=0.1, seed=73 + n)).cuda())
    s.step(3)
    f = s.get_state()
    g = torch.Generator(device="cpu").manual_seed(9)
    v = torch.randn(f.shape, generator=g, dtype=torch.float64).cuda() * 1e-2
    w = torch.randn(f.shape, generator=g, dtype=torch.float64).cuda()

    def one(sv, ff):
        sv.set_state_raw(ff, 0)
        sv.step(1)
        return sv.get_state()

    eps = 1e-6
    Jv = (one(s, f + eps * v) - one(s, f - eps * v)) / (2 * eps)
    lam_out = torch.empty_like(w)
    gacc = s.adjoint_scratch()
    s.adjoint_step(f, w, lam_out, gacc)
    lhs, rhs = float((Jv * w).sum()), float((v * lam_out).sum())
    assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-12), (lhs, rhs)
    gD = s.adjoint_reduce(gacc)
    h = 1e-6
    Dp, Dm = D.copy(), D.copy()
    Dp[0, 1] = Dp[1, 0] = D[0, 1] + h
    Dm[0, 1] = Dm[1, 0] = D[0, 1] - h
    fd = float(((one(Solver(lattice, Dp, dims, **kw), f) -
                 one(Solver(lattice, Dm, dims, **kw), f)) * w).sum()) / (2 * h)
    assert abs(gD[0] - fd) <= 1e-6 * max(abs(fd), 1e-9) + 1e-9


def test_boundary_arguments_are_checked():
    from paper_1808_06787_gb300 import LbmsError, Solver

    s = Solver("D2Q5", sy.random_D(3), (8, 4), bc=(B, W, P, P, P, P), dtype=torch.float64)
    s.set_state(torch.full((3, 1, 4, 8), 1.0 / 3.0, dtype=torch.float64).cuda())
    with pytest.raises(LbmsError, match="no composition"):
        s.step(1)
    with pytest.raises(LbmsError, match="not a Dirichlet face"):
        s.set_boundary(1, (0.2, 0.3, 0.5))
    with pytest.raises(LbmsError, match="not a Dirichlet face"):
        s.set_boundary(6, (0.2, 0.3, 0.5))
    with pytest.raises(LbmsError, match="sums to"):
        s.set_boundary(0, (0.2, 0.3, 0.6))
    with pytest.raises(LbmsError, match="not a mole fraction"):
        s.set_boundary(0, (1.2, -0.5, 0.3))
    s.set_boundary(0, (0.2, 0.3, 0.5))
    s.step(5)
    assert s.status() == 0
    # batches: a Dirichlet face must have its composition before the first step
    from paper_1808_06787_gb300 import BatchSolver

    bt = BatchSolver("D2Q5", np.stack([sy.random_D(3)]), np.array([[8, 8, 1]]),
                     bcs=[(B, B, P, P, P, P)], dtype=torch.float32)
    with pytest.raises(LbmsError, match="no composition set"):
        bt.step(1)
    with pytest.raises(LbmsError, match="sums to"):
        bt.set_boundary(0, 0, (0.2, 0.3, 0.6))
    with pytest.raises(LbmsError, match="out of range"):
        bt.set_boundary(1, 0, (0.2, 0.3, 0.5))


def test_gradient_with_dirichlet_faces_matches_finite_differences():
    """simulate() with Dirichlet faces (RunSpec.boundary), FP64: dL/dD against
    fourth-order central differences of the forward."""
    from paper_1808_06787_gb300 import RunSpec, Solver, simulate

    dims, steps = (24, 16, 1), 150
    bc = (B, B, P, P, P, P)
    xb = _compositions(3, 91)
    boundary = _boundary(bc, xb)
    x0 = torch.from_numpy(sy.sin_modes(3, *dims, amp=0.1, seed=92)).cuda()
    target = torch.from_numpy(sy.sin_modes(3, *dims, amp=0.1, seed=93)).cuda()
    d0 = np.array([0.07, 0.05, 0.02])

    def loss_of(d):
        D = sy.D_from_pairs(3, {(1, 2): d[0], (1, 3): d[1], (2, 3): d[2]})
        s = Solver("D2Q5", D, dims, bc=bc, dtype=torch.float64, boundary=boundary)
        s.set_state(x0)
        s.step(steps)
        return float(((s.moments() - target) ** 2).sum())

    dp = torch.tensor(d0, dtype=torch.float64, requires_grad=True)
    spec = RunSpec("D2Q5", dims, steps, bc=bc, dtype=torch.float64, boundary=boundary)
    loss = ((simulate(x0.clone(), dp, spec) - target) ** 2).sum()
    loss.backward()
    h = 1e-4
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (8 * (loss_of(d0 + e) - loss_of(d0 - e)) - (loss_of(d0 + 2 * e) - loss_of(d0 - 2 * e))) / (12 * h)
        assert abs(float(dp.grad[k]) - fd) <= 1e-6 * abs(fd) + 1e-12, (k, float(dp.grad[k]), fd)
