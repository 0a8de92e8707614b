"""Adjoint kernels and the differentiable solver (gradients with respect to
the binary diffusivities and the initial field).

1. One adjoint step is the transpose of the derivative of one forward step:
   <J v, w> = <v, J^T w> with J v from central differences of the FP64
   forward step, and the same for the derivative with respect to D_ij.
2. Whole runs: the adjoint gradient of L = sum (x(T) - x*)^2 against central
   finite differences of the FP64 CPU oracle on a 64 x 64 copy of the
   512 x 512 workload (D pairs; the initial field along random directions),
   and at full size against central differences of the GPU forward.
"""

import math

import numpy as np
import pytest

import synthetic as sy

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")

P, W = "periodic", "noflux"
D_START = (0.10, 0.08, 0.02)
D_TARGET = (0.09, 0.07, 0.02)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _one_step(s, f, step=0):
    s.set_state_raw(f, step)
    s.step(1)
    return s.get_state()


@pytest.mark.parametrize("lattice,n,dims,bc", [
    ("D2Q5", 3, (21, 13, 1), (W, W, P, P, P, P)),
    ("D2Q9", 4, (17, 11, 1), (P, P, W, W, P, P)),
    ("D3Q7", 5, (9, 7, 6), (W, W, P, P, W, W)),
    ("D2Q9", 2, (12, 9, 1), (P,) * 6),
    ("D3Q15", 4, (7, 6, 5), (W, W, P, P, W, W)),
    ("D1Q3", 3, (33, 1, 1), (W, W, P, P, P, P)),
])
def test_adjoint_step_is_transpose_of_step_derivative(lattice, n, dims, bc):
    from paper_1808_06787_gb300 import Solver

    D = sy.random_D(n, seed=31 + n)
    s = Solver(lattice, D, dims, bc=bc, dtype=torch.float64)
    x0 = sy.sin_modes(n, *dims, amp=0.1, seed=40 + n)
    s.set_state(torch.from_numpy(x0).cuda())
    s.step(3)  # a state off equilibrium
    f = s.get_state()
    g = torch.Generator(device="cpu").manual_seed(5)
    v = torch.randn(f.shape, generator=g, dtype=torch.float64).cuda() * 1e-2
    w = torch.randn(f.shape, generator=g, dtype=torch.float64).cuda()  # lambda is FP64
    eps = 1e-6
    Jv = (_one_step(s, f + eps * v) - _one_step(s, f - eps * v)) / (2 * eps)
    lam_out = torch.empty_like(w)
    gacc = s.adjoint_scratch()
    s.adjoint_step(f, w, lam_out, gacc)
    lhs = float((Jv * w).sum())
    rhs = float((v * lam_out).sum())
    assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-12), (lhs, rhs)
    # derivative with respect to each D pair of L = <w, step(f; D)>
    gD = s.adjoint_reduce(gacc)
    k = 0
    for p_ in range(n):
        for q in range(p_ + 1, n):
            h = 1e-6
            Dp, Dm = D.copy(), D.copy()
            Dp[p_, q] = Dp[q, p_] = D[p_, q] + h
            Dm[p_, q] = Dm[q, p_] = D[p_, q] - h
            sp = Solver(lattice, Dp, dims, bc=bc, dtype=torch.float64)
            sm = Solver(lattice, Dm, dims, bc=bc, dtype=torch.float64)
            fd = float(((_one_step(sp, f) - _one_step(sm, f)) * w).sum()) / (2 * h)
            assert abs(gD[k] - fd) <= 1e-6 * max(abs(fd), 1e-9) + 1e-9, (p_, q, gD[k], fd)
            k += 1


def _oracle_loss(D3, x0, target, steps):
    import oracle

    D = sy.D_from_pairs(3, {(1, 2): D3[0], (1, 3): D3[1], (2, 3): D3[2]})
    x = oracle.run("D2Q5", D, x0, steps)
    return float(((x - target) ** 2).sum())


def _fd4(fun, h):
    """Fourth-order central difference of fun at 0 (error O(h^4))."""
    return (8.0 * (fun(h) - fun(-h)) - (fun(2 * h) - fun(-2 * h))) / (12.0 * h)


def _gradients_64(dtype, steps, target):
    from paper_1808_06787_gb300 import RunSpec, simulate

    x0 = sy.sin_modes(3, 64, 64, amp=0.05, seed=1005)
    x0t = torch.from_numpy(x0).to(dtype).cuda().requires_grad_(True)
    dp = torch.tensor(D_START, dtype=torch.float64, requires_grad=True)
    spec = RunSpec("D2Q5", (64, 64, 1), steps, dtype=dtype)
    xT = simulate(x0t, dp, spec)
    loss = ((xT.double() - torch.from_numpy(target).cuda()) ** 2).sum()
    loss.backward()
    return x0, x0t.grad.double().cpu().numpy(), dp.grad.numpy(), spec


def _target_64(steps):
    import oracle

    x0 = sy.sin_modes(3, 64, 64, amp=0.05, seed=1005)
    return oracle.run("D2Q5", sy.D_from_pairs(3, {(1, 2): D_TARGET[0], (1, 3): D_TARGET[1],
                                                  (2, 3): D_TARGET[2]}), x0, steps)


def test_fp64_gradient_matches_oracle_finite_differences_64():
    """64 x 64 copy of the 512 x 512 workload, 4000 steps: the FP64 adjoint
    differentiates the map the FP64 oracle evaluates, so they agree to the error
    of the fourth-order finite differences (h = 1e-4)."""
    steps = 4000
    target = _target_64(steps)
    x0, gx, gD, spec = _gradients_64(torch.float64, steps, target)
    assert spec.stats["checkpoints"] == math.ceil(steps / math.ceil(math.sqrt(steps)))
    assert np.all(gx[2] == 0.0)
    checks = []
    for k in range(3):
        def fun(d, k=k):
            dd = list(D_START)
            dd[k] += d
            return _oracle_loss(dd, x0, target, steps)

        checks.append(("D pair %d" % k, gD[k], _fd4(fun, 1e-4)))
    for k_mode in ((1, 0, 0), (0, 1, 0), (1, 2, 0)):
        # a bounded mode moving species 1 against species 2 (sum_sigma v = 0)
        v = sy.small_mode([0.0, 0.0, 0.0], [1.0, -1.0, 0.0], 1.0, 64, 64, k=k_mode)
        checks.append(("x0 direction %s" % (k_mode,), float((gx * v).sum()),
                       _fd4(lambda e: _oracle_loss(D_START, x0 + e * v, target, steps), 1e-4)))
    for name, ad, fd in checks:
        print(name, ad, fd, abs(ad - fd) / abs(fd))
    for name, ad, fd in checks:
        assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-14, (name, ad, fd)


def test_fp32_gradient_close_to_fp64_gradient_64():
    """The FP32 solver (FP64 adjoint state) against the FP64 gradient checked
    above.  Its accuracy is that of the FP32 forward trajectory: late in the run
    the non-equilibrium part f - w xi that the D derivative multiplies is ~1e-6
    of f, and the final-state error (~1e-7) is a visible part of the slow-mode
    misfit the initial-field gradient is built from."""
    steps = 4000
    target = _target_64(steps)
    _, gx64, gD64, _ = _gradients_64(torch.float64, steps, target)
    _, gx32, gD32, _ = _gradients_64(torch.float32, steps, target)
    rel_D = np.abs(gD32 - gD64) / np.abs(gD64)
    rel_x = np.linalg.norm(gx32 - gx64) / np.linalg.norm(gx64)
    print("FP32 vs FP64: D", rel_D, "x0 (norm)", rel_x)
    assert np.all(rel_D <= 2e-3), rel_D
    assert rel_x <= 5e-2, rel_x


def test_adjoint_512sq_full_size_gradient_vs_finite_differences():
    """512 x 512, 4000 steps, FP32: adjoint dL/dD against central differences
    (h = 1e-4) of the GPU forward; target generated with D* = (0.09, 0.07, 0.02)."""
    from paper_1808_06787_gb300 import RunSpec, Solver, simulate

    steps = 4000
    x0 = sy.sin_modes(3, 512, 512, amp=0.05, seed=1005)
    x0t = torch.from_numpy(x0).float().cuda()

    def forward(d3):
        s = Solver("D2Q5", sy.D_from_pairs(3, {(1, 2): d3[0], (1, 3): d3[1], (2, 3): d3[2]}),
                   (512, 512), dtype=torch.float32)
        s.set_state(x0t)
        s.step(steps)
        return s.moments().double()

    target = forward(D_TARGET)
    dp = torch.tensor(D_START, dtype=torch.float64, requires_grad=True)
    xT = simulate(x0t.clone().requires_grad_(True), dp, RunSpec("D2Q5", (512, 512, 1), steps))
    loss = ((xT.double() - target) ** 2).sum()
    loss.backward()
    gD = dp.grad.numpy()
    h = 1e-4
    for k in range(3):
        up, dn = list(D_START), list(D_START)
        up[k] += h
        dn[k] -= h
        fd = (float(((forward(up) - target) ** 2).sum()) - float(((forward(dn) - target) ** 2).sum())) / (2 * h)
        assert abs(gD[k] - fd) <= 1e-2 * abs(fd) + 1e-9, (k, gD[k], fd)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_recompute_is_bit_identical_and_leaves_the_handle_alone(dtype):
    from paper_1808_06787_gb300 import Solver

    n, dims = 3, (24, 20, 1)
    s = Solver("D2Q5", sy.random_D(n, seed=81), dims, bc=(W, W, P, P, P, P), dtype=dtype)
    s.set_state(torch.from_numpy(sy.sin_modes(n, *dims, amp=0.1, seed=82)).to(dtype).cuda())
    s.step(5)
    ck = s.get_state()
    ref = []
    for _ in range(7):
        s.step(1)
        ref.append(s.get_state())
    out = torch.empty((7,) + tuple(s.state_shape), dtype=dtype, device="cuda")
    s.recompute(ck, 5, 7, out)
    for j in range(7):
        assert torch.equal(out[j], ref[j]), j
    # the handle continues from its own state and step count
    s.step(3)
    after = s.get_state()
    s2 = Solver("D2Q5", sy.random_D(n, seed=81), dims, bc=(W, W, P, P, P, P), dtype=dtype)
    s2.set_state_raw(ref[-1], 12)
    s2.step(3)
    assert torch.equal(after, s2.get_state())


def _pack_pairs(w64):
    hi = w64.float()
    lo = (w64 - hi.double()).float()
    return torch.stack([hi, lo], dim=-1).contiguous()


def test_fp32_adjoint_state_keeps_48_bits():
    """A lambda uniform over directions and nodes is a fixed point of the adjoint
    step; the float-pair state reproduces it far below FP32 resolution."""
    from paper_1808_06787_gb300 import Solver

    n, dims = 3, (21, 13, 1)
    s = Solver("D2Q5", sy.random_D(n, seed=83), dims, dtype=torch.float32)
    s.set_state(torch.from_numpy(sy.sin_modes(n, *dims, amp=0.1, seed=84)).float().cuda())
    s.step(4)
    f = s.get_state()
    c = torch.tensor([1.0 / 3.0 + 1e-9, -2.0 / 7.0], dtype=torch.float64)
    w = c.view(2, 1, 1).expand(s.state_shape).contiguous().cuda()
    lam = _pack_pairs(w)
    out = s.adjoint_state()
    s.adjoint_step(f, lam, out, s.adjoint_scratch())
    got = s.adjoint_value(out)
    assert float((got - w).abs().max()) <= 1e-13


def test_fp32_adjoint_step_matches_fp64_step():
    from paper_1808_06787_gb300 import Solver

    n, dims = 3, (21, 13, 1)
    D = sy.random_D(n, seed=85)
    s64 = Solver("D2Q5", D, dims, bc=(W, W, P, P, P, P), dtype=torch.float64)
    s64.set_state(torch.from_numpy(sy.sin_modes(n, *dims, amp=0.1, seed=86)).cuda())
    s64.step(4)
    f64 = s64.get_state()
    s32 = Solver("D2Q5", D, dims, bc=(W, W, P, P, P, P), dtype=torch.float32)
    g = torch.Generator(device="cpu").manual_seed(87)
    # a smooth large part plus small deviations, as in a backward sweep
    w = (0.5 + 1e-3 * torch.randn(s64.state_shape, generator=g, dtype=torch.float64)).cuda()
    o64 = torch.empty_like(w)
    ga64, ga32 = s64.adjoint_scratch(), s32.adjoint_scratch()
    s64.adjoint_step(f64, w, o64, ga64)
    o32 = s32.adjoint_state()
    s32.adjoint_step(f64.float(), _pack_pairs(w), o32, ga32)
    diff = (s32.adjoint_value(o32) - o64).abs().max()
    # FP32 Jacobian on deviations of ~1e-3 (and FP32 populations): ~1e-9
    assert float(diff) <= 2e-8
    np.testing.assert_allclose(s32.adjoint_reduce(ga32), s64.adjoint_reduce(ga64), rtol=2e-3, atol=0)
