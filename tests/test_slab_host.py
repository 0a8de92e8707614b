"""Host logic of the slab decomposition, without a GPU: the balanced partition
of the split axis, the face kinds of each slab, the neighbour ranks, and the
halo exchange over torch.distributed point-to-point messages, run with gloo
ranks on the CPU (world sizes 2, 3 and 4, closed and wrapping split axes).

The exchange test fills each rank's send buffers with values that name the
sender and the face, and checks that every receive buffer holds the right
neighbour's buffer: rank r's top-layer buffer (send_hi) in rank r+1's recv_lo,
its bottom-layer buffer (send_lo) in rank r-1's recv_hi, wrapping or not.
"""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")


def test_partition_is_balanced_and_covers_the_axis():
    from paper_1808_06787_gb300.slab import partition

    for extent in (1, 2, 7, 64, 255, 256):
        for parts in range(1, min(extent, 9) + 1):
            r = partition(extent, parts)
            assert len(r) == parts
            assert r[0][0] == 0 and sum(c for _, c in r) == extent
            assert all(r[i][0] + r[i][1] == r[i + 1][0] for i in range(parts - 1))
            assert max(c for _, c in r) - min(c for _, c in r) <= 1
    with pytest.raises(ValueError):
        partition(3, 4)
    with pytest.raises(ValueError):
        partition(3, 0)


def test_split_axis_is_the_lattices_last_axis():
    from paper_1808_06787_gb300.slab import split_axis

    assert [split_axis(l) for l in ("D3Q7", "D3Q15", "D3Q6")] == [2, 2, 2]
    assert [split_axis(l) for l in ("D2Q5", "D2Q9", "D2Q4")] == [1, 1, 1]
    assert split_axis("D1Q3") == 0


def test_slab_faces():
    from paper_1808_06787_gb300.slab import slab_faces

    W, P, D, H = "noflux", "periodic", "dirichlet", "halo"
    # closed split axis (z of D3Q7): the end slabs keep the grid's faces
    bc = (P, P, W, W, D, W)
    assert slab_faces("D3Q7", bc, 0, 3) == (P, P, W, W, D, H)
    assert slab_faces("D3Q7", bc, 1, 3) == (P, P, W, W, H, H)
    assert slab_faces("D3Q7", bc, 2, 3) == (P, P, W, W, H, W)
    # wrapping split axis (y of D2Q9): every slab has two cuts
    assert slab_faces("D2Q9", (W, W, P, P, P, P), 0, 2) == (W, W, H, H, P, P)
    assert slab_faces("D2Q9", (W, W, P, P, P, P), 1, 2) == (W, W, H, H, P, P)
    # one slab is the grid itself
    assert slab_faces("D2Q9", (W, W, P, P, P, P), 0, 1) == (W, W, P, P, P, P)
    # D1Q3 is split along x
    assert slab_faces("D1Q3", (W, W, P, P, P, P), 1, 3) == (H, H, P, P, P, P)
    with pytest.raises(ValueError):
        slab_faces("D3Q7", (P, P, P, P, H, H), 0, 2)


def test_neighbours():
    from paper_1808_06787_gb300.slab import neighbours

    assert neighbours(0, 3, False) == (None, 1)
    assert neighbours(1, 3, False) == (0, 2)
    assert neighbours(2, 3, False) == (1, None)
    assert neighbours(0, 3, True) == (2, 1)
    assert neighbours(2, 3, True) == (1, 0)
    assert neighbours(0, 1, True) == (None, None)
    assert neighbours(0, 2, True) == (1, 1)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, periodic, q):
    sys.path.insert(0, ROOT)
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist

    from paper_1808_06787_gb300.slab import exchange_halos, neighbours

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shape = (3, 2, 5)  # [crossing populations][S][layer nodes]
        dn, up = neighbours(rank, world, periodic)
        # sender r, face f (0 = bottom layer, 1 = top layer): value 100 r + 10 f + index
        idx = torch.arange(30, dtype=torch.float64).reshape(shape) / 100.0
        send_lo = (100.0 * rank + idx) if dn is not None else None
        send_hi = (100.0 * rank + 10.0 + idx) if up is not None else None
        recv_lo = torch.full(shape, -1.0, dtype=torch.float64) if dn is not None else None
        recv_hi = torch.full(shape, -1.0, dtype=torch.float64) if up is not None else None
        for _ in range(3):  # repeated exchanges, as every time step does
            exchange_halos(dist, rank, world, periodic, send_lo, send_hi, recv_lo, recv_hi)
        got_lo = None if recv_lo is None else recv_lo.tolist()
        got_hi = None if recv_hi is None else recv_hi.tolist()
        q.put((rank, dn, up, got_lo, got_hi, idx.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, False), (2, True), (3, False), (3, True), (4, True)])
def test_halo_exchange_routes_each_layer_to_its_neighbour(world, periodic):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, periodic, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, dn, up, got_lo, got_hi, idx in out:
        idx = torch.tensor(idx, dtype=torch.float64)
        if dn is None:
            assert got_lo is None
        else:
            # the rank below sent its top layer (face 1)
            assert torch.equal(torch.tensor(got_lo, dtype=torch.float64), 100.0 * dn + 10.0 + idx), (rank, dn)
        if up is None:
            assert got_hi is None
        else:
            # the rank above sent its bottom layer (face 0)
            assert torch.equal(torch.tensor(got_hi, dtype=torch.float64), 100.0 * up + idx), (rank, up)
    if not periodic:
        assert out[0][1] is None and out[-1][2] is None
