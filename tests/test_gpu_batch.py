"""Batched solves (many independent grids in one node space).

Every instance of a batch must evolve exactly as a single solve of its grid
(same kernels' arithmetic, same stochastic-rounding keys), whatever step
schedule the batch runs with; the single-solve path is itself checked against
the FP64 oracle in test_gpu_parity.py, and a few instances are checked against
the oracle here directly.
"""

import numpy as np
import pytest

import synthetic as sy

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

torch = pytest.importorskip("torch")

P, W = "periodic", "noflux"


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mixed_batch(lattice, n, dtype, seed=5):
    g = sy.rng(seed)
    if lattice in ("D3Q7", "D3Q15", "D3Q6"):
        grids = [(9, 7, 5), (1, 1, 1), (16, 4, 3), (13, 13, 2), (3, 40, 1)]
    elif lattice == "D1Q3":
        grids = [(33, 1, 1), (1, 1, 1), (640, 1, 1), (51, 1, 1), (300, 1, 1), (7, 1, 1)]
    else:
        grids = [(33, 17, 1), (1, 1, 1), (64, 64, 1), (50, 3, 1), (5, 91, 1), (128, 20, 1)]
    Ds, bcs, x0s = [], [], []
    for i, gr in enumerate(grids):
        Ds.append(sy.random_D(n, seed=seed * 100 + i))
        bcs.append([(P,) * 6, (W, W, P, P, W, W), (P, P, W, W, P, P), (W,) * 6][i % 4])
        x0s.append(sy.sin_modes(n, *gr, amp=0.08, seed=seed * 1000 + i))
    return grids, Ds, bcs, x0s


def _single(lattice, D, x0, steps, bc, dtype):
    from paper_1808_06787_gb300 import Solver

    n, nz, ny, nx = x0.shape
    s = Solver(lattice, D, (nx, ny, nz), bc=bc, dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    s.step(steps)
    x, J = s.moments(flux=True)
    return x, J, s.mass()


@pytest.mark.parametrize("lattice,n", [("D2Q5", 3), ("D2Q9", 5), ("D3Q7", 4), ("D3Q15", 3),
                                       ("D1Q3", 3), ("D2Q4", 3), ("D2Q4", 4), ("D3Q6", 3)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_equals_single_solves_bitwise(lattice, n, dtype):
    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs, x0s = _mixed_batch(lattice, n, dtype)
    b = BatchSolver(lattice, Ds, grids, bcs=bcs, dtype=dtype)
    b.set_state([torch.from_numpy(x) for x in x0s])
    steps = 77
    b.step(steps)
    x, J = b.moments(flux=True)
    xs, Js = b.unpack(x), b.unpack(J, flux=True)
    mass = b.mass()
    assert b.status() == 0
    for i in range(len(grids)):
        xr, Jr, mr = _single(lattice, Ds[i], x0s[i], steps, bcs[i], dtype)
        assert torch.equal(xs[i], xr), i
        assert torch.equal(Js[i], Jr), i
        assert np.array_equal(mass[i], mr), i


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_every_schedule_gives_the_same_result(dtype):
    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs, x0s = _mixed_batch("D2Q5", 3, dtype, seed=9)
    # enough instances for several L2 groups even at the largest budget
    g = sy.rng(3)
    for i in range(40):
        L = int(g.integers(200, 600))
        grids.append((L, L, 1))
        Ds.append(sy.random_D(3, seed=700 + i))
        bcs.append((P,) * 6)
        x0s.append(sy.sin_modes(3, L, L, amp=0.05, seed=900 + i))
    ref = None
    # every schedule with both kernel shapes (the two-nodes-per-thread shape
    # exists for FP32 only)
    from paper_1808_06787_gb300 import LbmsError

    for cand in range(14):
        b = BatchSolver("D2Q5", Ds, grids, bcs=bcs, dtype=dtype)
        if cand >= 7 and dtype == torch.float64:
            with pytest.raises(LbmsError, match="two-nodes-per-thread"):
                b.set_schedule(cand)
            b.close()
            continue
        b.set_schedule(cand)
        assert b.schedule == cand
        b.set_state([torch.from_numpy(x) for x in x0s])
        b.step(71)
        x = b.moments()
        m = b.mass()
        if ref is None:
            ref = (x, m)
        else:
            assert torch.equal(x, ref[0]), cand
            assert np.array_equal(m, ref[1]), cand
        b.close()


def test_batch_instances_against_oracle():
    import oracle

    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs = sy.batch_instances(6, lo=20, hi=40, seed=44)
    x0s = [sy.batch_field(i, int(grids[i][0]), seed=44) for i in range(6)]
    b = BatchSolver("D2Q5", Ds, grids, bcs=bcs, dtype=torch.float32)
    b.set_state([torch.from_numpy(x) for x in x0s])
    b.step(500)
    xs = b.unpack(b.moments())
    for i in range(6):
        ref = oracle.run("D2Q5", Ds[i], x0s[i], 500, bc=bcs[i])
        assert np.abs(xs[i].double().cpu().numpy() - ref).max() <= 2e-5, i


def test_batch_host_buffers_and_offsets():
    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs, x0s = _mixed_batch("D2Q9", 4, torch.float64, seed=13)
    a = BatchSolver("D2Q9", Ds, grids, bcs=bcs, dtype=torch.float64)
    flat = a.pack([torch.from_numpy(x) for x in x0s])
    a.set_state(flat.cuda())
    a.step(9)
    xa, Ja = a.moments(flux=True)
    b = BatchSolver("D2Q9", Ds, grids, bcs=bcs, dtype=torch.float64)
    b.set_state(flat.clone())  # pageable host source, packed through the staging area
    b.step(9)
    xb, Jb = b.moments(flux=True, out_device="cpu")  # pinned outputs, written in place
    assert torch.equal(xa.cpu(), xb) and torch.equal(Ja.cpu(), Jb)
    c = BatchSolver("D2Q9", Ds, grids, bcs=bcs, dtype=torch.float64)
    fp = flat.clone().pin_memory()
    c.set_state(fp)  # pinned host source, read by the init kernel in place
    fp.fill_(0.0)
    c.step(9)
    xc, Jc = c.moments(flux=True)
    assert torch.equal(xa, xc) and torch.equal(Ja, Jc)


def test_tuner_picks_a_valid_schedule():
    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs = sy.batch_instances(64, seed=8)
    b = BatchSolver("D2Q5", Ds, grids, bcs=bcs)
    chosen, times = b.tune(trial_steps=8)
    assert 0 <= chosen < 14 and b.schedule == chosen
    assert np.all(times > 0) and times[chosen] == times.min()
    # a batch without the two-nodes-per-thread kernel reports those candidates as -1
    b64 = BatchSolver("D2Q5", Ds, grids, bcs=bcs, dtype=torch.float64)
    chosen, times = b64.tune(trial_steps=4)
    assert 0 <= chosen < 7 and np.all(times[7:] == -1.0) and np.all(times[:7] > 0)


def test_batch_4096_uneven_d2q5_instances_full_size():
    """4096 ternary D2Q5 instances, sides uniform in [32, 256], 5000 steps, FP32:
    per-instance mass drift, flags, and sampled instances against single solves."""
    from paper_1808_06787_gb300 import BatchSolver

    count = 4096
    grids, Ds, bcs = sy.batch_instances(count)
    b = BatchSolver("D2Q5", Ds, grids, bcs=bcs, dtype=torch.float32)
    flat = torch.empty(int(b.offsets[-1]), dtype=torch.float32)
    for i in range(count):
        flat[int(b.offsets[i]):int(b.offsets[i + 1])] = torch.from_numpy(
            sy.batch_field(i, int(grids[i][0])).reshape(-1)).float()
    b.set_state(flat.cuda())
    m0 = b.mass()
    b.step(5000)
    m1 = b.mass()
    assert b.status() == 0
    assert np.max(np.abs(m1 - m0) / np.abs(m0)) <= 1e-6
    xs = b.unpack(b.moments())
    for i in (0, 1, 2047, 4095):
        x0 = sy.batch_field(i, int(grids[i][0]))
        xr, _, _ = _single("D2Q5", Ds[i], x0, 5000, bcs[i], torch.float32)
        assert torch.equal(xs[i], xr), i
    # two sampled instances (a periodic sine and a no-flux tanh one) against the oracle
    import oracle

    for i in (0, 1):
        x0 = sy.batch_field(i, int(grids[i][0]))
        ref = oracle.run("D2Q5", Ds[i], x0, 5000, bc=bcs[i])
        assert np.abs(xs[i].double().cpu().numpy().reshape(ref.shape) - ref).max() <= 2e-5, i


@pytest.mark.parametrize("lattice", ["D2Q5", "D2Q4", "D3Q7", "D1Q3"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batch_with_dirichlet_faces_equals_single_solves(lattice, dtype):
    """Instances with Dirichlet faces (per-instance compositions) evolve bit for
    bit as single solves with the same faces and compositions, with both kernel
    shapes where the two-nodes-per-thread kernel exists."""
    from paper_1808_06787_gb300 import BatchSolver, LbmsError, Solver

    DI = "dirichlet"
    n = 3
    if lattice == "D3Q7":
        grids = [(9, 7, 5), (6, 5, 8), (12, 3, 4)]
        bcs = [(DI, DI, P, P, W, W), (W, W, DI, W, P, P), (P, P, P, P, DI, DI)]
    elif lattice == "D1Q3":
        grids = [(40, 1, 1), (77, 1, 1), (9, 1, 1)]
        bcs = [(DI, DI, P, P, P, P), (DI, W, P, P, P, P), (W, DI, P, P, P, P)]
    else:
        grids = [(30, 17, 1), (21, 40, 1), (64, 9, 1)]
        bcs = [(DI, DI, P, P, P, P), (W, W, DI, W, P, P), (DI, W, DI, DI, P, P)]
    Ds = [sy.random_D(n, seed=600 + i) for i in range(3)]
    x0s = [sy.sin_modes(n, *gr, amp=0.08, seed=610 + i) for i, gr in enumerate(grids)]
    comps = sy.rng(620)
    boundary = {}
    for i, bc in enumerate(bcs):
        for f, kind in enumerate(bc):
            if kind == DI:
                c = comps.uniform(0.1, 1.0, size=n)
                boundary[(i, f)] = c / c.sum()
    shapes = [0, 7] if (dtype == torch.float32 and lattice in ("D2Q5", "D2Q4", "D1Q3")) else [0]
    steps = 61
    for cand in shapes:
        b = BatchSolver(lattice, Ds, grids, bcs=bcs, dtype=dtype)
        with pytest.raises(LbmsError, match="no composition set"):
            b.step(1)
        for (i, f), c in boundary.items():
            b.set_boundary(i, f, c)
        b.set_schedule(cand)
        b.set_state([torch.from_numpy(x) for x in x0s])
        b.step(steps)
        x, J = b.moments(flux=True)
        xs, Js = b.unpack(x), b.unpack(J, flux=True)
        for i in range(3):
            bnd = {f: c for (j, f), c in boundary.items() if j == i}
            s = Solver(lattice, Ds[i], grids[i], bc=bcs[i], dtype=dtype, boundary=bnd)
            s.set_state(torch.from_numpy(x0s[i]).to(dtype).cuda())
            s.step(steps)
            xr, Jr = s.moments(flux=True)
            assert torch.equal(xs[i], xr), (cand, i)
            assert torch.equal(Js[i], Jr), (cand, i)
        assert b.status() == 0
        with pytest.raises(LbmsError, match="not a Dirichlet face"):
            b.set_boundary(0, 5, [0.2, 0.3, 0.5])
        b.close()
