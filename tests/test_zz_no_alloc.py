"""lbms_mass_noalloc: the allocation-free mass entry point.

Callers that cannot call cudaMalloc (real-time loops whose device memory is
fixed at start-up, plug-ins living in a host framework's memory pool,
monitoring code reading a buffer it does not own) get species totals of a
population buffer from this entry point, which keeps its scratch in a static
device array instead of a workspace.  These tests call it through the C ABI
and check it against lbms_mass.  The file is named to be collected last, so
that a stop-at-first-failure run has run everything else.
"""

import ctypes

import numpy as np
import pytest

import synthetic as sy

torch = pytest.importorskip("torch")


def _call(lib, lattice, n, grid, dtype, pop_ptr, out):
    return lib.lbms_mass_noalloc(lattice, n, (ctypes.c_int * 3)(*grid), dtype,
                                 ctypes.c_void_p(pop_ptr), out, None)


def test_noalloc_rejects_oversized_grids_and_host_buffers_before_device_work():
    import paper_1808_06787_gb300 as p

    lib = p.load()
    out = np.zeros(3)
    # 1024^3 F32 nodes x 3 species need 96 MiB of partials: beyond the 4 MiB area
    rc = _call(lib, 2, 3, (1024, 1024, 1024), 0, 256, out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 1
    assert "scratch" in lib.lbms_last_error(None).decode()
    rc = _call(lib, 2, 3, (16, 16, 16), 0, 0, out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 1
    # a host buffer of the right size is refused before any launch
    host = np.zeros(2 * 7 * 16 * 16 * 16, dtype=np.float32)
    rc = _call(lib, 2, 3, (16, 16, 16), 0, host.ctypes.data, out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 1
    assert "device memory" in lib.lbms_last_error(None).decode()
    assert np.all(out == 0.0)


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_noalloc_matches_lbms_mass_twice(dtype):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1808_06787_gb300 as p
    from paper_1808_06787_gb300 import Solver

    lib = p.load()
    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    dims = (96, 80, 40)
    x0 = sy.two_bulb(*dims)
    s = Solver("D3Q7", D, dims, bc="noflux", dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    dt = 1 if dtype == torch.float64 else 0
    # right after set_state both entry points run the same reduction on the same
    # populations: bit-identical results
    m_init = s.mass()
    out0 = np.full(3, np.nan)
    assert _call(lib, 2, 3, dims, dt, s.populations().data_ptr(),
                 out0.ctypes.data_as(ctypes.c_void_p)) == 0
    assert np.array_equal(out0, m_init)
    s.step(25)
    torch.cuda.synchronize()
    ref = s.mass()  # existing entry point (partials in the solver's workspace)
    pop = s.populations()
    # after steps lbms_mass sums the xi its last step formed from the gathered
    # populations, this entry point the xi of the stored ones: the per-node
    # roundings differ, so the comparison uses the mass tolerance of the parity
    # tests (1e-6 relative in FP32, 1e-12 in FP64)
    tol = (1e-12 if dtype == torch.float64 else 1e-6) * np.abs(ref)
    outs = []
    for _ in range(2):  # two calls in a row share the static scratch
        out = np.full(3, np.nan)
        rc = _call(lib, 2, 3, dims, dt, pop.data_ptr(), out.ctypes.data_as(ctypes.c_void_p))
        assert rc == 0, lib.lbms_last_error(None).decode()
        assert np.all(np.abs(out - ref) <= tol), (out, ref)
        outs.append(out)
    assert np.array_equal(outs[0], outs[1])
    # device output
    dev = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    rc = _call(lib, 2, 3, dims, dt, pop.data_ptr(), ctypes.c_void_p(dev.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), outs[0])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("dims", [(1, 1, 1), (24, 20, 10), (64, 64, 18), (64, 64, 19)],
                         ids=["1node", "small", "below-77824", "at-77824"])
def test_noalloc_bit_identical_to_lbms_mass_at_every_size(dims, dtype):
    """Right after set_state both entry points reduce the same populations with
    the same block partition (64-node blocks below 2 x 152 x 256 = 77824 nodes
    on GB300's 152 SMs, 256 above), so
    the results agree bit for bit, FP64 compensated sums included."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1808_06787_gb300 as p
    from paper_1808_06787_gb300 import Solver

    lib = p.load()
    D = sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})
    x0 = sy.sin_modes(3, *dims, amp=0.1, seed=11) if dims[2] == 1 else sy.two_bulb(*dims)
    s = Solver("D3Q7", D, dims, bc="noflux", dtype=dtype)
    s.set_state(torch.from_numpy(x0).to(dtype).cuda())
    ref = s.mass()
    out = np.full(3, np.nan)
    rc = _call(lib, 2, 3, dims, 1 if dtype == torch.float64 else 0, s.populations().data_ptr(),
               out.ctypes.data_as(ctypes.c_void_p))
    assert rc == 0, lib.lbms_last_error(None).decode()
    assert np.array_equal(out, ref), (out, ref)
    s.close()
