"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point that include/lbms.h declares, sizes workspaces as
documented, and rejects invalid arguments before touching the device."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(lbms_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_1808_06787_gb300 as p

    return p.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lbms_create", "lbms_set_state", "lbms_step", "lbms_moments", "lbms_mass",
              "lbms_status", "lbms_destroy", "lbms_workspace_size", "lbms_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    import paper_1808_06787_gb300 as p

    for name in declared_functions():
        assert name in p.EXPORTED, name


@pytest.mark.parametrize("lat,q,dim", [(0, 5, 2), (1, 9, 2), (2, 7, 3), (3, 15, 3), (4, 3, 1),
                                       (5, 4, 2), (6, 6, 3)])
@pytest.mark.parametrize("n", [2, 3, 8])
@pytest.mark.parametrize("dtype,es", [(0, 4), (1, 8)])
def test_workspace_size(lib, lat, q, dim, n, dtype, es):
    import paper_1808_06787_gb300 as p

    grid = (37, 23 if dim > 1 else 1, 11 if dim == 3 else 1)
    cells = grid[0] * grid[1] * grid[2]
    size = p.lbms_workspace_size(lat, n, grid, dtype)
    pop = (n - 1) * q * cells * es
    # halo buffers of the split axis: 6 x [crossing populations][S][layer nodes]
    width = {0: 1, 1: 3, 2: 1, 3: 5, 4: 1, 5: 1, 6: 1}[lat]
    layer = {3: grid[0] * grid[1], 2: grid[0], 1: 1}[dim]
    halo = 6 * width * (n - 1) * layer * es
    assert size >= 2 * pop + n * (1 + dim) * cells * es + halo
    assert size % 256 == 0
    assert size < (2 * pop + n * (1 + dim) * cells * es + halo + 64 * 1024 + cells * n * 16 // 64
                   + 8192)


def test_workspace_size_rejects(lib):
    import paper_1808_06787_gb300 as p

    assert p.lbms_workspace_size(0, 1, (4, 4, 1), 0) == 0  # one species
    assert p.lbms_workspace_size(0, 9, (4, 4, 1), 0) == 0  # too many
    assert p.lbms_workspace_size(0, 3, (4, 4, 2), 0) == 0  # 2D lattice, nz > 1
    assert p.lbms_workspace_size(2, 3, (0, 4, 4), 0) == 0  # empty grid
    assert p.lbms_workspace_size(7, 3, (4, 4, 4), 0) == 0  # unknown lattice
    assert p.lbms_workspace_size(4, 3, (4, 2, 1), 0) == 0  # 1D lattice, ny > 1
    assert p.lbms_workspace_size(2, 3, (4, 4, 4), 2) == 0  # unknown dtype
    assert p.lbms_workspace_size(2, 3, (2048, 2048, 1024), 0) == 0  # beyond 2^31 cells


def _create(lib, *, lat=0, n=3, grid=(8, 8, 1), D=None, relax=0, bc=(0,) * 6, dtype=0,
            ws=256, wsb=1 << 30):
    h = ctypes.c_void_p()
    if D is None:
        D = np.full((n, n), 0.1)
    D = np.ascontiguousarray(D, dtype=np.float64)
    rc = lib.lbms_create(ctypes.byref(h), lat, n, (ctypes.c_int * 3)(*grid),
                         D.ctypes.data_as(ctypes.c_void_p), relax, (ctypes.c_int * 6)(*bc), dtype,
                         ctypes.c_void_p(ws), wsb, None)
    return rc, h, lib.lbms_last_error(None).decode()


def test_create_validates_before_device_work(lib):
    # each of these fails in argument checking, before any CUDA call
    rc, h, msg = _create(lib, D=np.array([[1, 0.1, -0.2], [0.1, 1, 0.1], [-0.2, 0.1, 1]]))
    assert rc == 1 and "positive" in msg and not h.value
    rc, _, msg = _create(lib, D=np.array([[1, 0.1, 0.2], [0.1, 1, 0.1], [0.3, 0.1, 1]]))
    assert rc == 1 and "symmetric" in msg
    rc, _, msg = _create(lib, D=np.array([[1, np.nan, 0.2], [np.nan, 1, 0.1], [0.2, 0.1, 1]]))
    assert rc == 1
    rc, _, msg = _create(lib, bc=(0, 1, 0, 0, 0, 0))
    assert rc == 1 and "paired" in msg
    rc, _, msg = _create(lib, bc=(4, 4, 0, 0, 0, 0))  # unknown face kind
    assert rc == 1 and "face kind" in msg
    rc, _, msg = _create(lib, bc=(3, 3, 0, 0, 0, 0))  # slab cut on x: D2Q5 is split along y
    assert rc == 1 and "split axis" in msg
    rc, _, msg = _create(lib, bc=(0, 0, 3, 0, 0, 0))  # a cut paired with a periodic face
    assert rc == 1 and "paired" in msg
    rc, _, msg = _create(lib, lat=2, grid=(4, 4, 4), bc=(1, 1, 3, 3, 1, 1))  # D3Q7 is split along z
    assert rc == 1 and "split axis" in msg
    rc, _, msg = _create(lib, bc=(2, 0, 0, 0, 0, 0))  # Dirichlet against a periodic face
    assert rc == 1 and "paired" in msg
    rc, _, msg = _create(lib, relax=3)
    assert rc == 1 and "relaxation" in msg
    rc, _, msg = _create(lib, ws=0)
    assert rc == 1 and "workspace" in msg
    rc, _, msg = _create(lib, ws=256 + 8)
    assert rc == 1 and "aligned" in msg
    rc, _, msg = _create(lib, wsb=1024)
    assert rc == 2 and "needed" in msg
    rc, _, msg = _create(lib, n=1)
    assert rc == 1
    rc, _, msg = _create(lib, lat=2, grid=(4, 4, 0))
    assert rc == 1


def test_null_handle_calls(lib):
    assert lib.lbms_step(None, 1) == 1
    assert lib.lbms_set_state(None, None) == 1
    assert lib.lbms_set_boundary(None, 0, None) == 1
    assert lib.lbms_set_reference(None, None) == 1
    assert lib.lbms_moments(None, None, None) == 1
    assert lib.lbms_mass(None, None) == 1
    assert lib.lbms_status(None, None) == 1
    assert lib.lbms_steps_done(None) == -1
    assert lib.lbms_populations(None) is None
    assert lib.lbms_set_subdomain(None, 0) == 1
    assert lib.lbms_halo_buffers(None, 0, None, None, None) == 1
    assert lib.lbms_slab_step(None, 0, 1) == 1
    lib.lbms_destroy(None)


def _header_enums():
    """NAME = value pairs of the enums and #defines of include/lbms.h."""
    text = open(os.path.join(ROOT, "include", "lbms.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, v in re.findall(r"(LBMS_\w+)\s*=\s*(\d+)", body):
            vals[name] = int(v)
    for name, v in re.findall(r"#define\s+(LBMS_\w+)\s+(0x[0-9a-fA-F]+|\d+)", text):
        vals[name] = int(v, 0)
    return vals


def test_binding_constants_match_the_header():
    """The Python binding passes the header's enum values, not its own."""
    import paper_1808_06787_gb300.lbms as b

    h = _header_enums()
    for name, v in b.LATTICES.items():
        assert h["LBMS_" + name] == v, name
    assert {"magic": h["LBMS_RELAX_MAGIC"], "srt": h["LBMS_RELAX_SRT"],
            "frozen": h["LBMS_RELAX_FROZEN"]} == b.RELAX
    assert {"periodic": h["LBMS_PERIODIC"], "noflux": h["LBMS_NOFLUX"],
            "dirichlet": h["LBMS_DIRICHLET"], "halo": h["LBMS_HALO"]} == b.FACE
    assert sorted(b.DTYPES.values()) == [h["LBMS_F32"], h["LBMS_F64"]]
    assert b.FLAG_NONFINITE == h["LBMS_FLAG_NONFINITE"]
    assert b.FLAG_RANGE == h["LBMS_FLAG_RANGE"]
    assert b.FLAG_INIT == h["LBMS_FLAG_INIT"]
    assert b.BATCH_CANDIDATES == h["LBMS_BATCH_CANDIDATES"]
    codes = {v: k[len("LBMS_"):] for k, v in h.items()
             if k in ("LBMS_EINVAL", "LBMS_ENOMEM", "LBMS_ECUDA", "LBMS_ENONFINITE", "LBMS_ERANGE",
                      "LBMS_ETIMEOUT")}
    assert codes == b.ERRORS
    assert b.LBMS_OK == h["LBMS_OK"] == 0
