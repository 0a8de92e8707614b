"""Adjoint kernels and the differentiable solver (gradients with respect to
the binary diffusivities and the initial field).

1. One adjoint step is the transpose of the derivative of one forward step:
   <J v, w> = <v, J^T w> with J v from central differences of the FP64
   forward step, and the same for the derivative with respect to D_ij.
2. Whole runs: the adjoint gradient of L = sum (x(T) - x*)^2 against central
   finite differences of the FP64 CPU oracle on a 64 x 64 copy of the
   512 x 512 workload (D pairs; the initial field along bounded modes), in
   FP64 and in FP32 (the FP32 bound follows from the FP32 forward error and
   the adjoint's arithmetic), and at full size against central differences of
   the GPU forward in FP64 and FP32.
3. The adjoint entry points refuse host buffers.
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
    ("D2Q4", 3, (15, 13, 1), (W, W, P, P, P, P)),
    ("D2Q4", 5, (12, 11, 1), (P,) * 6),
    ("D3Q6", 4, (8, 7, 6), (P, P, W, W, W, W)),
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


def _Dm(d3):
    return sy.D_from_pairs(3, {(1, 2): d3[0], (1, 3): d3[1], (2, 3): d3[2]})


def _fd4(fun, h):
    """Fourth-order central difference of fun at 0 (error O(h^4)); fun may return
    a scalar or an array."""
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
    return (x0, x0t.grad.double().cpu().numpy(), dp.grad.numpy(), spec,
            xT.detach().double().cpu().numpy())


STEPS_64 = 4000
H_FD = 1e-4
X0_MODES = ((1, 0, 0), (0, 1, 0), (1, 2, 0))


@pytest.fixture(scope="module")
def oracle_fd_64():
    """The FP64 oracle on the 64 x 64 copy of the 512 x 512 adjoint workload
    (4000 steps): target field (from D*), final field at the starting point, and
    for each parameter -- the three D pairs, then three bounded initial-field
    modes moving species 1 against species 2 -- fourth-order central differences
    (h = 1e-4) of the loss and of the final field."""
    import oracle

    x0 = sy.sin_modes(3, 64, 64, amp=0.05, seed=1005)
    target = oracle.run("D2Q5", _Dm(D_TARGET), x0, STEPS_64)
    base = oracle.run("D2Q5", _Dm(D_START), x0, STEPS_64)
    params = []
    for k in range(3):
        def final(e, k=k):
            dd = list(D_START)
            dd[k] += e
            return oracle.run("D2Q5", _Dm(dd), x0, STEPS_64)

        params.append(("D pair %d" % k, final, None))
    for mode in X0_MODES:
        v = sy.small_mode([0.0, 0.0, 0.0], [1.0, -1.0, 0.0], 1.0, 64, 64, k=mode)
        params.append(("x0 direction %s" % (mode,),
                       lambda e, v=v: oracle.run("D2Q5", _Dm(D_START), x0 + e * v, STEPS_64), v))
    out = []
    for name, final, v in params:
        fields = {e: final(e) for e in (H_FD, -H_FD, 2 * H_FD, -2 * H_FD)}
        dx = _fd4(lambda e: fields[e], H_FD)
        dL = _fd4(lambda e: float(((fields[e] - target) ** 2).sum()), H_FD)
        out.append((name, v, dL, dx))
    return dict(x0=x0, target=target, base=base, params=out)


def _adjoint_values(gD, gx, params):
    return [gD[i] if v is None else float((gx * v).sum()) for i, (_, v, _, _) in enumerate(params)]


def test_fp64_gradient_matches_oracle_finite_differences_64(oracle_fd_64):
    """64 x 64 copy of the 512 x 512 workload, 4000 steps: the FP64 adjoint
    differentiates the map the FP64 oracle evaluates, so they agree to the error
    of the fourth-order finite differences (h = 1e-4)."""
    o = oracle_fd_64
    _, gx, gD, spec, _ = _gradients_64(torch.float64, STEPS_64, o["target"])
    assert spec.stats["checkpoints"] == math.ceil(STEPS_64 / math.ceil(math.sqrt(STEPS_64)))
    assert np.all(gx[2] == 0.0)
    ad = _adjoint_values(gD, gx, o["params"])
    for (name, _, fd, _), a in zip(o["params"], ad):
        print(name, a, fd, abs(a - fd) / abs(fd))
    for (name, _, fd, _), a in zip(o["params"], ad):
        assert abs(a - fd) <= 1e-6 * abs(fd) + 1e-14, (name, a, fd)


# Arithmetic allowance of the FP32 adjoint (float-pair lambda, FP32 Jacobian on the
# deviation of lambda from its direction mean, compensated FP32 sums): each of the
# T = 4000 backward steps rounds the deviation it maps at the FP32 unit roundoff
# u = 2^-24, so the accumulated relative error of a gradient component is of order
# T u = 2.4e-4; the allowance takes four times that.
FP32_ADJOINT_ARITH = 4 * STEPS_64 * 2.0 ** -24


def test_fp32_gradient_matches_oracle_fd_64_within_forward_error_bound(oracle_fd_64):
    """The FP32 solver's gradient against fourth-order differences of the FP64
    oracle.  The FP32 forward ends at x32(T) = x(T) + dx instead of x(T); to first
    order that moves the gradient of L = |x(T) - x*|^2 along any parameter p by
    2 <dx, dx(T)/dp>, which the oracle's differences of the final field give.  So
    the FP32 gradient must equal (oracle difference + that shift) to within the
    adjoint's own arithmetic allowance, and must differ from the oracle difference
    by no more than |shift| + that allowance."""
    o = oracle_fd_64
    _, gx, gD, _, x32 = _gradients_64(torch.float32, STEPS_64, o["target"])
    dx = x32 - o["base"]
    print("FP32 forward error at T: max %.3g, norm %.3g" % (np.abs(dx).max(), np.linalg.norm(dx)))
    ad = _adjoint_values(gD, gx, o["params"])
    for (name, _, fd, dxdp), a in zip(o["params"], ad):
        shift = 2.0 * float((dx * dxdp).sum())
        resid = a - (fd + shift)
        print("%-24s adjoint %.9g  oracle FD %.9g  shift %.3g  rel |ad-fd| %.3g  rel resid %.3g"
              % (name, a, fd, shift, abs(a - fd) / abs(fd), abs(resid) / abs(fd)))
        assert abs(resid) <= FP32_ADJOINT_ARITH * abs(fd), (name, a, fd, shift)
        assert abs(a - fd) <= abs(shift) + FP32_ADJOINT_ARITH * abs(fd), (name, a, fd, shift)


def test_fp32_initial_field_gradient_error_is_the_propagated_forward_error_64(oracle_fd_64):
    """The whole initial-field gradient: FP32 minus FP64 (the FP64 gradient is
    pinned to the oracle above) is, to first order, the FP64 adjoint applied to
    the FP32 forward error, g32 - g64 = 2 J^T (x32(T) - x64(T)) with J = dx(T)/dx0;
    the FP64 adjoint seeded with 2 (x32 - x64) gives that vector.  After removing
    it, what is left must be within the FP32 adjoint's arithmetic allowance."""
    from paper_1808_06787_gb300 import RunSpec, simulate

    o = oracle_fd_64
    _, gx64, _, _, x64 = _gradients_64(torch.float64, STEPS_64, o["target"])
    _, gx32, _, _, x32 = _gradients_64(torch.float32, STEPS_64, o["target"])
    x0t = torch.from_numpy(o["x0"]).cuda().requires_grad_(True)
    dp = torch.tensor(D_START, dtype=torch.float64, requires_grad=True)
    xT = simulate(x0t, dp, RunSpec("D2Q5", (64, 64, 1), STEPS_64, dtype=torch.float64))
    (xT * torch.from_numpy(2.0 * (x32 - x64)).cuda()).sum().backward()
    pred = x0t.grad.cpu().numpy()
    err = np.linalg.norm(gx32 - gx64) / np.linalg.norm(gx64)
    resid = np.linalg.norm(gx32 - gx64 - pred) / np.linalg.norm(gx64)
    print("x0 gradient FP32 vs FP64 (norm): %.3g; after removing the propagated forward "
          "error: %.3g" % (err, resid))
    assert resid <= FP32_ADJOINT_ARITH, (err, resid)
    assert err <= np.linalg.norm(pred) / np.linalg.norm(gx64) + FP32_ADJOINT_ARITH


def test_adjoint_512sq_full_size_gradient_vs_finite_differences():
    """512 x 512, 4000 steps, FP32 (the bench's adjoint workload): adjoint dL/dD
    against central differences of the GPU forward.

    (a) FP64 forward (pinned to the oracle at 1e-12), h = 1e-4: as in the 64 x 64
    test, the FP32 gradient equals the difference plus the first-order shift
    2 <x32(T) - x64(T), dx(T)/dD> within the FP32 adjoint's arithmetic allowance.
    (b) FP32 forward: its loss carries rounding noise nu (estimated from loss
    changes under perturbations far too small to matter, minus the adjoint's
    prediction of them), so the step is chosen as h = max(1e-4, 1e3 nu / |g|),
    where the noise adds at most nu / h to the difference; the truncation error
    is estimated from the differences at h and 2h (Richardson)."""
    from paper_1808_06787_gb300 import RunSpec, Solver, simulate

    steps = 4000
    x0 = sy.sin_modes(3, 512, 512, amp=0.05, seed=1005)

    def forward(d3, dtype):
        s = Solver("D2Q5", _Dm(d3), (512, 512), dtype=dtype)
        s.set_state(torch.from_numpy(x0).to(dtype).cuda())
        s.step(steps)
        x = s.moments().double()
        s.close()
        return x

    target = forward(D_TARGET, torch.float32)
    dp = torch.tensor(D_START, dtype=torch.float64, requires_grad=True)
    xT = simulate(torch.from_numpy(x0).float().cuda().requires_grad_(True), dp,
                  RunSpec("D2Q5", (512, 512, 1), steps))
    loss = ((xT.double() - target) ** 2).sum()
    loss.backward()
    gD = dp.grad.numpy()
    x32 = xT.detach().double()
    x64 = forward(D_START, torch.float64)
    L32 = lambda d3: float(((forward(d3, torch.float32) - target) ** 2).sum())
    L64 = lambda d3: float(((forward(d3, torch.float64) - target) ** 2).sum())
    for k in range(3):
        def at(e, k=k):
            d = list(D_START)
            d[k] += e
            return d

        # (a)
        h = 1e-4
        xp, xm = forward(at(h), torch.float64), forward(at(-h), torch.float64)
        fd64 = (float(((xp - target) ** 2).sum()) - float(((xm - target) ** 2).sum())) / (2 * h)
        shift = 2.0 * float(((x32 - x64) * (xp - xm) / (2 * h)).sum())
        resid = gD[k] - (fd64 + shift)
        print("D pair %d: adjoint %.9g  FP64 FD %.9g  shift %.3g  rel resid %.3g"
              % (k, gD[k], fd64, shift, abs(resid) / abs(fd64)))
        # central differences at h = 1e-4 carry O(h^2) truncation: estimated by
        # Richardson from h and 2h
        fd64_2h = (L64(at(2 * h)) - L64(at(-2 * h))) / (4 * h)
        trunc = abs(fd64_2h - fd64) / 3.0
        assert abs(resid) <= FP32_ADJOINT_ARITH * abs(fd64) + trunc, (k, gD[k], fd64, shift, trunc)
        # (b)
        L0 = L32(D_START)
        nu = max(abs(L32(at(e)) - L0 - e * gD[k]) for e in (1e-9, -1e-9, 2e-9, -2e-9))
        hb = max(1e-4, 1e3 * nu / abs(gD[k]))
        fd = (L32(at(hb)) - L32(at(-hb))) / (2 * hb)
        fd2 = (L32(at(2 * hb)) - L32(at(-2 * hb))) / (4 * hb)
        tol = nu / hb + abs(fd2 - fd) / 3.0 + abs(shift) + FP32_ADJOINT_ARITH * abs(fd)
        print("D pair %d: noise %.3g  h %.3g  FP32 FD %.9g  |ad - fd| %.3g  tol %.3g"
              % (k, nu, hb, fd, abs(gD[k] - fd), tol))
        assert abs(gD[k] - fd) <= tol, (k, gD[k], fd, tol)


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


def test_adjoint_entry_points_refuse_host_buffers():
    from paper_1808_06787_gb300 import LbmsError, Solver

    dims = (12, 10, 1)
    s = Solver("D2Q5", sy.random_D(3, seed=5), dims, dtype=torch.float64)
    s.set_state(torch.from_numpy(sy.sin_modes(3, *dims, amp=0.1, seed=6)).cuda())
    s.step(2)
    f = s.get_state()
    lam, lam2, gacc = s.adjoint_state(), s.adjoint_state(), s.adjoint_scratch()
    host = lambda t: torch.zeros(t.shape, dtype=t.dtype)
    with pytest.raises(LbmsError, match="device memory"):
        s.adjoint_step(host(f), lam, lam2, gacc)
    with pytest.raises(LbmsError, match="device memory"):
        s.adjoint_step(f, host(lam), lam2, gacc)
    with pytest.raises(LbmsError, match="device memory"):
        s.adjoint_step(f, lam, lam2, host(gacc))
    with pytest.raises(LbmsError, match="device memory"):
        s.adjoint_seed(host(torch.zeros(s.field_shape, dtype=torch.float64)), lam)
    with pytest.raises(LbmsError, match="device memory"):
        s.adjoint_reduce(host(gacc))
    # the device path still works after the refusals
    s.adjoint_seed(torch.ones(s.field_shape, dtype=torch.float64, device="cuda"), lam)
    s.adjoint_step(f, lam, lam2, gacc)
    assert np.all(np.isfinite(s.adjoint_reduce(gacc)))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("count", [1, 2, 5])
def test_adjoint_steps_equal_single_adjoint_steps(dtype, count):
    """lbms_adjoint_steps (a segment in one call) = `count` calls of
    lbms_adjoint_step, bit for bit, including the gradient accumulator."""
    from paper_1808_06787_gb300 import Solver

    n, dims = 3, (23, 17, 1)
    s = Solver("D2Q5", sy.random_D(n, seed=91), dims, bc=(W, W, P, P, P, P), dtype=dtype)
    s.set_state(torch.from_numpy(sy.sin_modes(n, *dims, amp=0.1, seed=92)).to(dtype).cuda())
    s.step(3)
    states = [s.get_state()]
    for _ in range(count - 1):
        s.step(1)
        states.append(s.get_state())
    rest = torch.stack(states[1:]) if count > 1 else None
    g = torch.Generator(device="cpu").manual_seed(93)
    seed_x = (1e-2 * torch.randn(s.field_shape, generator=g, dtype=torch.float64)).to(dtype).cuda()
    lam0 = s.adjoint_state()
    s.adjoint_seed(seed_x, lam0)
    # reference: single steps from the last state back to the first
    a, b = lam0.clone(), s.adjoint_state()
    ga = s.adjoint_scratch()
    for j in range(count - 1, -1, -1):
        s.adjoint_step(states[j], a, b, ga)
        a, b = b, a
    # one call
    la, lb = lam0.clone(), s.adjoint_state()
    gb = s.adjoint_scratch()
    s.adjoint_steps(states[0], rest, count, la, lb, gb)
    out = lb if count % 2 else la
    assert torch.equal(out, a)
    assert torch.equal(gb, ga)


@pytest.mark.parametrize("lattice,dims,bc", [("D2Q4", (24, 20, 1), (W, W, P, P, P, P)),
                                             ("D3Q6", (10, 9, 8), (P, P, W, W, W, W))])
def test_gradient_without_rest_velocity_matches_oracle_differences(lattice, dims, bc):
    """Whole-run gradients on the lattices without a rest velocity (FP64, 300
    steps) against fourth-order differences of the FP64 oracle."""
    import oracle

    from paper_1808_06787_gb300 import RunSpec, simulate

    n, steps = 3, 300
    x0 = sy.sin_modes(n, *dims, amp=0.1, seed=97)
    # a target far from the start, so that the misfit (and the gradient) stand
    # well above the rounding noise of the loss
    target = oracle.run(lattice, _Dm((0.05, 0.12, 0.04)), x0, steps, bc=bc)
    x0t = torch.from_numpy(x0).cuda().requires_grad_(True)
    dp = torch.tensor(D_START, dtype=torch.float64, requires_grad=True)
    xT = simulate(x0t, dp, RunSpec(lattice, dims, steps, bc=bc, dtype=torch.float64))
    ((xT - torch.from_numpy(target).cuda()) ** 2).sum().backward()
    loss = lambda d3, x: float(((oracle.run(lattice, _Dm(d3), x, steps, bc=bc) - target) ** 2).sum())
    fds = []
    for k in range(3):
        def fun(e, k=k):
            d = list(D_START)
            d[k] += e
            return loss(d, x0)

        fds.append(_fd4(fun, 1e-4))
    # the differences' rounding noise is set by the loss, the same for every
    # component: the bound is relative to the largest component
    scale = max(abs(v) for v in fds)
    for k, fd in enumerate(fds):
        assert abs(dp.grad[k].item() - fd) <= 1e-6 * scale + 1e-14, (k, dp.grad[k].item(), fd)
    v = sy.small_mode([0.0, 0.0, 0.0], [1.0, -1.0, 0.0], 1.0, *dims, k=(1, 1, 0))
    fd = _fd4(lambda e: loss(D_START, x0 + e * v), 1e-4)
    ad = float((x0t.grad.cpu().numpy() * v).sum())
    assert abs(ad - fd) <= 1e-6 * abs(fd) + 1e-14, (ad, fd)
