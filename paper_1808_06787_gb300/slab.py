"""Slab decomposition of one grid: the nearest-neighbour propagation of the
model (Eq. 3-13b) couples a node only to its neighbours, so a grid split into
slabs along one axis needs a single exchange per time step -- the populations
that cross each cut -- and the species masses of the whole grid are the sums
of the slabs' masses.

The split axis is the lattice's last axis (z for D3Q7, D3Q15, D3Q6; y for
D2Q5, D2Q9, D2Q4; x for D1Q3), so that a layer of nodes is contiguous in the
structure-of-arrays layout.  Each slab is a solver handle whose cut faces are
``"halo"`` faces (``LBMS_HALO``): every step also writes the populations that
leave through a cut into the face's send buffer, and the next step reads the
neighbour's into the face's receive buffer (``include/lbms.h``, "Slab
decomposition").  FP32 solvers key their stochastic rounding by the node's
index in the undivided grid (``set_subdomain``), so a decomposed run equals
the undivided one bit for bit.

``SlabSolver`` keeps all slabs of a grid on one GPU and exchanges through
device-to-device copies inside ``lbms_slab_step``.  ``DistSlabSolver`` holds
one slab per process (one GPU each) and exchanges with ``torch.distributed``
point-to-point messages (``exchange_halos``).  ``partition``, ``slab_faces``
and ``exchange_halos`` are plain host logic.
"""

from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from .lbms import DIMS, FACE, LbmsError, Solver, lbms_slab_step

_NAMES = {v: k for k, v in FACE.items()}


def split_axis(lattice: str) -> int:
    """Grid axis (0 = x, 1 = y, 2 = z) along which slabs are cut."""
    return DIMS[lattice] - 1


def partition(extent: int, parts: int):
    """Balanced split of ``extent`` layers into ``parts`` slabs: [(first, count)]."""
    extent, parts = int(extent), int(parts)
    if parts < 1 or parts > extent:
        raise ValueError("cannot split %d layers into %d slabs" % (extent, parts))
    base, extra = divmod(extent, parts)
    out, first = [], 0
    for i in range(parts):
        count = base + (1 if i < extra else 0)
        out.append((first, count))
        first += count
    return out


def _face_names(bc):
    if isinstance(bc, str):
        bc = (bc,) * 6
    faces = [b if isinstance(b, str) else _NAMES[int(b)] for b in bc]
    if len(faces) != 6:
        raise ValueError("bc needs 6 face kinds (x-, x+, y-, y+, z-, z+)")
    return faces


def slab_faces(lattice: str, bc, part: int, parts: int):
    """The six face kinds of slab ``part`` of ``parts``: the faces of the split
    axis that are cuts become "halo" (both faces of every slab when that axis is
    periodic and there is more than one slab; the end faces of the end slabs keep
    the grid's own kind otherwise); the other faces are the grid's."""
    faces = _face_names(bc)
    a = split_axis(lattice)
    lo, hi = 2 * a, 2 * a + 1
    if "halo" in faces:
        raise ValueError("the grid's own faces cannot be halo faces")
    if parts > 1:
        if faces[lo] == "periodic":
            faces[lo] = faces[hi] = "halo"
        else:
            if part > 0:
                faces[lo] = "halo"
            if part < parts - 1:
                faces[hi] = "halo"
    return tuple(faces)


def _field_dim(axis: int) -> int:
    """Array dimension of grid axis ``axis`` in a field [n, nz, ny, nx]."""
    return 3 - axis


def _slice(x, axis: int, first: int, count: int):
    d = _field_dim(axis)
    idx = [slice(None)] * x.ndim
    idx[d] = slice(first, first + count)
    piece = x[tuple(idx)]
    if isinstance(piece, np.ndarray):
        return np.ascontiguousarray(piece)
    return piece.contiguous()


class SlabSolver:
    """One grid as ``parts`` slabs on one GPU (halo exchange by device copies).

    Arguments as for ``Solver`` plus ``parts``.  ``boundary`` compositions of
    Dirichlet faces go to the slabs that keep those faces.  Results are those of
    the undivided ``Solver`` bit for bit."""

    def __init__(self, lattice: str, D, grid: Sequence[int], parts: int, *, bc="periodic",
                 relax: str = "magic", dtype=torch.float32, device="cuda",
                 stream: Optional[torch.cuda.Stream] = None, boundary=None, reference=None):
        g = list(grid) + [1] * (3 - len(grid))
        self.lattice = lattice
        self.grid = tuple(int(v) for v in g)
        self.axis = split_axis(lattice)
        self.ranges = partition(self.grid[self.axis], parts)
        self.dtype = dtype
        self.stream = stream if stream is not None else torch.cuda.current_stream(torch.device(device))
        self.slabs = []
        for i, (first, count) in enumerate(self.ranges):
            sg = list(self.grid)
            sg[self.axis] = count
            faces = slab_faces(lattice, bc, i, len(self.ranges))
            bnd = {f: v for f, v in (boundary or {}).items() if faces[f] == "dirichlet"}
            s = Solver(lattice, D, sg, bc=faces, relax=relax, dtype=dtype, device=device,
                       stream=self.stream, boundary=bnd, reference=reference)
            s.set_subdomain(first)
            self.slabs.append(s)
        self.n = self.slabs[0].n

    @property
    def field_shape(self):
        nx, ny, nz = self.grid
        return (self.n, nz, ny, nx)

    def set_state(self, x0) -> None:
        """Mole fractions of the whole grid, [n, nz, ny, nx] (host or device)."""
        if tuple(x0.shape) != self.field_shape:
            raise ValueError("expected a field of shape %s" % (self.field_shape,))
        self._keep = []
        for s, (first, count) in zip(self.slabs, self.ranges):
            piece = _slice(x0, self.axis, first, count)
            if isinstance(piece, torch.Tensor):
                piece = piece.to(self.dtype)
            s.set_state(piece)
            self._keep.append(piece)

    def step(self, n: int) -> None:
        lbms_slab_step([s._h for s in self.slabs], int(n))

    def moments(self, flux: bool = False):
        outs = [s.moments(flux=flux) for s in self.slabs]
        d = _field_dim(self.axis)
        if not flux:
            return torch.cat(outs, dim=d)
        return torch.cat([o[0] for o in outs], dim=d), torch.cat([o[1] for o in outs], dim=d + 1)

    def gradient(self) -> torch.Tensor:
        return torch.cat([s.gradient() for s in self.slabs], dim=_field_dim(self.axis) + 1)

    def mass(self) -> np.ndarray:
        return np.sum([s.mass() for s in self.slabs], axis=0)

    def status(self) -> int:
        fl = 0
        for s in self.slabs:
            fl |= s.status()
        return fl

    @property
    def steps_done(self) -> int:
        return self.slabs[0].steps_done

    def close(self) -> None:
        for s in self.slabs:
            s.close()


def neighbours(rank: int, world: int, periodic: bool):
    """(rank below, rank above) of a slab in split-axis order, None at a closed end."""
    up = rank + 1 if rank + 1 < world else (0 if periodic and world > 1 else None)
    dn = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else None)
    return dn, up


def exchange_halos(dist, rank: int, world: int, periodic: bool, send_lo, send_hi, recv_lo, recv_hi,
                   group=None) -> None:
    """One halo exchange of a slab decomposition with one slab per rank: the
    populations of this rank's top layer that cross upward (``send_hi``) go to
    the rank above, into its ``recv_lo``; those of the bottom layer that cross
    downward (``send_lo``) go to the rank below, into its ``recv_hi``.  Every
    rank posts its upward traffic before its downward traffic, so that with two
    ranks on a wrapping axis -- both messages between the same pair -- they are
    matched in order.  Buffers of a face that is not a cut may be None."""
    dn, up = neighbours(rank, world, periodic)
    ops = []
    if up is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, up, group))
    if dn is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, dn, group))
    if dn is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, dn, group))
    if up is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, up, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


class DistSlabSolver:
    """One slab of a grid per process (one GPU each), ``torch.distributed`` ranks
    in split-axis order; halo exchange by point-to-point messages (NCCL between
    GPUs).  Each step is one exchange followed by one step of the local slab;
    the species masses of the whole grid come from one all-reduce of n doubles."""

    def __init__(self, lattice: str, D, grid: Sequence[int], dist, *, bc="periodic",
                 relax: str = "magic", dtype=torch.float32, device="cuda",
                 stream: Optional[torch.cuda.Stream] = None, boundary=None, reference=None):
        g = list(grid) + [1] * (3 - len(grid))
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.grid = tuple(int(v) for v in g)
        self.axis = split_axis(lattice)
        self.ranges = partition(self.grid[self.axis], self.world)
        first, count = self.ranges[self.rank]
        self.first, self.count = first, count
        faces = slab_faces(lattice, bc, self.rank, self.world)
        self.periodic = _face_names(bc)[2 * self.axis] == "periodic"
        sg = list(self.grid)
        sg[self.axis] = count
        bnd = {f: v for f, v in (boundary or {}).items() if faces[f] == "dirichlet"}
        self.solver = Solver(lattice, D, sg, bc=faces, relax=relax, dtype=dtype, device=device,
                             stream=stream, boundary=bnd, reference=reference)
        self.solver.set_subdomain(first)
        self.lo_face, self.hi_face = 2 * self.axis, 2 * self.axis + 1
        self.cut = (faces[self.lo_face] == "halo", faces[self.hi_face] == "halo")

    def set_state(self, x_local) -> None:
        """This rank's share of the initial mole fractions ([n, ...] of its slab)."""
        self.solver.set_state(x_local)

    def _exchange(self) -> None:
        s = self.solver
        send_lo = recv_lo = send_hi = recv_hi = None
        if self.cut[0]:
            send_lo, recv_lo = s.halo_buffers(self.lo_face)
        if self.cut[1]:
            send_hi, recv_hi = s.halo_buffers(self.hi_face)
        with torch.cuda.stream(s.stream):
            exchange_halos(self.dist, self.rank, self.world, self.periodic, send_lo, send_hi, recv_lo,
                           recv_hi)

    def step(self, n: int) -> None:
        for _ in range(int(n)):
            if self.world > 1:
                self._exchange()
            self.solver.step(1)

    def moments(self, flux: bool = False):
        return self.solver.moments(flux=flux)

    def mass(self) -> np.ndarray:
        m = torch.from_numpy(self.solver.mass()).to(self.solver.device)
        self.dist.all_reduce(m)
        return m.cpu().numpy()

    def status(self) -> int:
        return self.solver.status()

    def close(self) -> None:
        self.solver.close()
