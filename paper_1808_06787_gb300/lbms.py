"""Thin Python binding of the C ABI in ``include/lbms.h``.

Every function of the C library is bound under its own name (``lbms_create``,
``lbms_set_state``, ``lbms_step``, ``lbms_moments``, ``lbms_mass``,
``lbms_status``, ``lbms_steps_done``, ``lbms_last_error``, ``lbms_destroy``,
``lbms_workspace_size``); this module only marshals arguments.  All arithmetic
runs in the CUDA kernels of ``liblbms.so``.  PyTorch provides the device
memory (the workspace and field tensors) and the CUDA stream.

``Solver`` wraps one handle with its workspace tensor.
"""

from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

LATTICES = {"D2Q5": 0, "D2Q9": 1, "D3Q7": 2, "D3Q15": 3, "D1Q3": 4, "D2Q4": 5, "D3Q6": 6}
DIMS = {"D2Q5": 2, "D2Q9": 2, "D3Q7": 3, "D3Q15": 3, "D1Q3": 1, "D2Q4": 2, "D3Q6": 3}
Q_OF = {"D2Q5": 5, "D2Q9": 9, "D3Q7": 7, "D3Q15": 15, "D1Q3": 3, "D2Q4": 4, "D3Q6": 6}
RELAX = {"magic": 0, "srt": 1, "frozen": 2}
FACE = {"periodic": 0, "noflux": 1, "dirichlet": 2, "halo": 3}
DTYPES = {torch.float32: 0, torch.float64: 1}

LBMS_OK = 0
FLAG_NONFINITE = 0x1
FLAG_RANGE = 0x2
FLAG_INIT = 0x4
ERRORS = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ERANGE", 6: "ETIMEOUT"}

EXPORTED = (
    "lbms_workspace_size", "lbms_create", "lbms_set_state", "lbms_set_boundary",
    "lbms_set_reference", "lbms_step",
    "lbms_moments", "lbms_gradient",
    "lbms_mass", "lbms_mass_noalloc", "lbms_status", "lbms_steps_done", "lbms_populations",
    "lbms_last_error",
    "lbms_destroy",
    "lbms_batch_workspace_size", "lbms_batch_create", "lbms_batch_set_state", "lbms_batch_step",
    "lbms_batch_moments", "lbms_batch_mass", "lbms_batch_status", "lbms_batch_set_boundary",
    "lbms_batch_set_schedule",
    "lbms_batch_get_schedule", "lbms_batch_launches_per_step", "lbms_batch_tune",
    "lbms_batch_steps_done",
    "lbms_batch_last_error", "lbms_batch_destroy",
    "lbms_get_state", "lbms_set_state_raw", "lbms_recompute", "lbms_adjoint_scratch_size",
    "lbms_adjoint_seed",
    "lbms_adjoint_step", "lbms_adjoint_steps", "lbms_adjoint_initial", "lbms_adjoint_reduce",
    "lbms_set_subdomain", "lbms_halo_buffers", "lbms_slab_step",
)
BATCH_CANDIDATES = 14

_lock = threading.Lock()
_lib = None


class LbmsError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load ``liblbms.so`` (building it first if it is missing).  Raises if the
    CUDA library cannot be loaded: there is no fallback path."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise LbmsError("liblbms.so is not built; run paper_1808_06787_gb300.build.build()")
            _build.build()
        # the CUDA runtime torch loaded is reused by soname
        torch.cuda.is_available()
        L = ctypes.CDLL(path)
        P, I, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        L.lbms_workspace_size.argtypes = [I, I, P, I]
        L.lbms_workspace_size.restype = SZ
        L.lbms_create.argtypes = [P, I, I, P, P, I, P, I, P, SZ, P]
        L.lbms_create.restype = I
        L.lbms_set_state.argtypes = [P, P]
        L.lbms_set_state.restype = I
        L.lbms_set_boundary.argtypes = [P, I, P]
        L.lbms_set_boundary.restype = I
        L.lbms_set_reference.argtypes = [P, P]
        L.lbms_set_reference.restype = I
        L.lbms_step.argtypes = [P, ctypes.c_long]
        L.lbms_step.restype = I
        L.lbms_moments.argtypes = [P, P, P]
        L.lbms_moments.restype = I
        L.lbms_gradient.argtypes = [P, P]
        L.lbms_gradient.restype = I
        L.lbms_mass.argtypes = [P, P]
        L.lbms_mass.restype = I
        L.lbms_mass_noalloc.argtypes = [I, I, P, I, P, P, P]
        L.lbms_mass_noalloc.restype = I
        L.lbms_status.argtypes = [P, P]
        L.lbms_status.restype = I
        L.lbms_steps_done.argtypes = [P]
        L.lbms_steps_done.restype = ctypes.c_long
        L.lbms_populations.argtypes = [P]
        L.lbms_populations.restype = P
        L.lbms_last_error.argtypes = [P]
        L.lbms_last_error.restype = ctypes.c_char_p
        L.lbms_destroy.argtypes = [P]
        L.lbms_destroy.restype = None
        L.lbms_get_state.argtypes = [P, P]
        L.lbms_get_state.restype = I
        L.lbms_set_state_raw.argtypes = [P, P, ctypes.c_long]
        L.lbms_set_state_raw.restype = I
        L.lbms_recompute.argtypes = [P, P, ctypes.c_long, I, P]
        L.lbms_recompute.restype = I
        L.lbms_adjoint_scratch_size.argtypes = [P]
        L.lbms_adjoint_scratch_size.restype = SZ
        L.lbms_adjoint_seed.argtypes = [P, P, P]
        L.lbms_adjoint_seed.restype = I
        L.lbms_adjoint_step.argtypes = [P, P, P, P, P]
        L.lbms_adjoint_step.restype = I
        L.lbms_adjoint_steps.argtypes = [P, P, P, I, P, P, P]
        L.lbms_adjoint_steps.restype = I
        L.lbms_adjoint_initial.argtypes = [P, P, P]
        L.lbms_adjoint_initial.restype = I
        L.lbms_adjoint_reduce.argtypes = [P, P, P]
        L.lbms_adjoint_reduce.restype = I
        L.lbms_set_subdomain.argtypes = [P, ctypes.c_long]
        L.lbms_set_subdomain.restype = I
        L.lbms_halo_buffers.argtypes = [P, I, P, P, P]
        L.lbms_halo_buffers.restype = I
        L.lbms_slab_step.argtypes = [P, I, ctypes.c_long]
        L.lbms_slab_step.restype = I
        L.lbms_batch_workspace_size.argtypes = [I, I, I, P, I]
        L.lbms_batch_workspace_size.restype = SZ
        L.lbms_batch_create.argtypes = [P, I, I, I, P, P, I, P, I, P, SZ, P]
        L.lbms_batch_create.restype = I
        L.lbms_batch_set_state.argtypes = [P, P, P]
        L.lbms_batch_set_state.restype = I
        L.lbms_batch_step.argtypes = [P, ctypes.c_long]
        L.lbms_batch_step.restype = I
        L.lbms_batch_moments.argtypes = [P, P, P, P]
        L.lbms_batch_moments.restype = I
        L.lbms_batch_mass.argtypes = [P, P]
        L.lbms_batch_mass.restype = I
        L.lbms_batch_status.argtypes = [P, P]
        L.lbms_batch_status.restype = I
        L.lbms_batch_set_boundary.argtypes = [P, I, I, P]
        L.lbms_batch_set_boundary.restype = I
        L.lbms_batch_set_schedule.argtypes = [P, I]
        L.lbms_batch_set_schedule.restype = I
        L.lbms_batch_get_schedule.argtypes = [P]
        L.lbms_batch_get_schedule.restype = I
        L.lbms_batch_launches_per_step.argtypes = [P]
        L.lbms_batch_launches_per_step.restype = I
        L.lbms_batch_tune.argtypes = [P, I, P, P]
        L.lbms_batch_tune.restype = I
        L.lbms_batch_steps_done.argtypes = [P]
        L.lbms_batch_steps_done.restype = ctypes.c_long
        L.lbms_batch_last_error.argtypes = [P]
        L.lbms_batch_last_error.restype = ctypes.c_char_p
        L.lbms_batch_destroy.argtypes = [P]
        L.lbms_batch_destroy.restype = None
        _lib = L
        return L


def _grid(grid) -> ctypes.Array:
    g = list(grid) + [1] * (3 - len(grid))
    return (ctypes.c_int * 3)(*[int(v) for v in g])


def _faces(bc) -> ctypes.Array:
    if isinstance(bc, str):
        bc = (bc,) * 6
    vals = [FACE[b] if isinstance(b, str) else int(b) for b in bc]
    if len(vals) != 6:
        raise ValueError("bc needs 6 face kinds (x-, x+, y-, y+, z-, z+)")
    return (ctypes.c_int * 6)(*vals)


# --- the C entry points under their own names ------------------------------

def lbms_workspace_size(lattice: int, n_species: int, grid, dtype: int) -> int:
    return int(load().lbms_workspace_size(lattice, n_species, _grid(grid), dtype))


def lbms_create(lattice: int, n_species: int, grid, D, relax: int, bc, dtype: int,
                workspace_ptr: int, workspace_bytes: int, stream_ptr: int) -> ctypes.c_void_p:
    L = load()
    h = ctypes.c_void_p()
    Dm = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    rc = L.lbms_create(ctypes.byref(h), lattice, n_species, _grid(grid),
                       Dm.ctypes.data_as(ctypes.c_void_p), relax, _faces(bc), dtype,
                       ctypes.c_void_p(workspace_ptr), workspace_bytes, ctypes.c_void_p(stream_ptr))
    if rc != LBMS_OK:
        raise LbmsError("lbms_create: %s (%s)" % (ERRORS.get(rc, rc), L.lbms_last_error(None).decode()))
    return h


def _check(h, rc: int, what: str) -> None:
    if rc != LBMS_OK:
        raise LbmsError("%s: %s (%s)" % (what, ERRORS.get(rc, rc), load().lbms_last_error(h).decode()))


def lbms_set_state(h, x0_ptr: int) -> None:
    _check(h, load().lbms_set_state(h, ctypes.c_void_p(x0_ptr)), "lbms_set_state")


def lbms_set_boundary(h, face: int, xi_b) -> None:
    v = np.ascontiguousarray(np.asarray(xi_b, dtype=np.float64).reshape(-1))
    _check(h, load().lbms_set_boundary(h, int(face), v.ctypes.data_as(ctypes.c_void_p)),
           "lbms_set_boundary")


def lbms_set_reference(h, xi_ref) -> None:
    v = np.ascontiguousarray(np.asarray(xi_ref, dtype=np.float64).reshape(-1))
    _check(h, load().lbms_set_reference(h, v.ctypes.data_as(ctypes.c_void_p)), "lbms_set_reference")


def lbms_step(h, n_steps: int) -> None:
    _check(h, load().lbms_step(h, int(n_steps)), "lbms_step")


def lbms_moments(h, x_ptr: int, J_ptr: Optional[int]) -> None:
    _check(h, load().lbms_moments(h, ctypes.c_void_p(x_ptr),
                                  ctypes.c_void_p(J_ptr) if J_ptr else None), "lbms_moments")


def lbms_gradient(h, g_ptr: int) -> None:
    _check(h, load().lbms_gradient(h, ctypes.c_void_p(g_ptr)), "lbms_gradient")


def lbms_mass(h, n_species: int) -> np.ndarray:
    out = np.zeros(n_species, dtype=np.float64)
    _check(h, load().lbms_mass(h, out.ctypes.data_as(ctypes.c_void_p)), "lbms_mass")
    return out


def lbms_mass_noalloc(lattice: int, n_species: int, grid, dtype: int, populations_ptr: int,
                      mass_out_ptr: int, stream_ptr: int) -> None:
    """Species totals of a population buffer without a handle or any device
    allocation (for callers that cannot allocate; see include/lbms.h)."""
    L = load()
    rc = L.lbms_mass_noalloc(lattice, n_species, _grid(grid), dtype, ctypes.c_void_p(populations_ptr),
                             ctypes.c_void_p(mass_out_ptr), ctypes.c_void_p(stream_ptr))
    if rc != LBMS_OK:
        raise LbmsError("lbms_mass_noalloc: %s (%s)" % (ERRORS.get(rc, rc), L.lbms_last_error(None).decode()))


def lbms_status(h) -> int:
    fl = ctypes.c_uint32()
    _check(h, load().lbms_status(h, ctypes.byref(fl)), "lbms_status")
    return int(fl.value)


def lbms_steps_done(h) -> int:
    return int(load().lbms_steps_done(h))


def lbms_last_error(h) -> str:
    return load().lbms_last_error(h).decode()


def lbms_destroy(h) -> None:
    load().lbms_destroy(h)


def lbms_set_subdomain(h, first_layer: int) -> None:
    _check(h, load().lbms_set_subdomain(h, int(first_layer)), "lbms_set_subdomain")


def lbms_halo_buffers(h, face: int):
    """(send address, receive address, bytes) of a cut face of a slab."""
    send, recv, nbytes = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_size_t()
    _check(h, load().lbms_halo_buffers(h, int(face), ctypes.byref(send), ctypes.byref(recv),
                                       ctypes.byref(nbytes)), "lbms_halo_buffers")
    return int(send.value), int(recv.value), int(nbytes.value)


def lbms_slab_step(handles, n_steps: int) -> None:
    arr = (ctypes.c_void_p * len(handles))(*[h.value for h in handles])
    rc = load().lbms_slab_step(arr, len(handles), int(n_steps))
    if rc != LBMS_OK:
        first = handles[0] if handles else None
        raise LbmsError("lbms_slab_step: %s (%s)" % (ERRORS.get(rc, rc), load().lbms_last_error(first).decode()))


# --- convenience wrapper ---------------------------------------------------

class Solver:
    """One solver handle and the torch-owned workspace it runs in.

    ``lattice``: "D2Q5" | "D2Q9" | "D3Q7"; ``D``: n x n binary diffusivities in
    lattice units; ``grid``: (nx, ny[, nz]); ``bc``: one kind for all faces or six
    kinds (x-, x+, y-, y+, z-, z+), each "periodic", "noflux" or "dirichlet";
    ``boundary``: {face index: composition of all n species} for the Dirichlet
    faces (see ``set_boundary``); ``relax``: "magic" (Eq. 3-16), "srt", or
    "frozen" (relaxation matrices at the fixed composition ``reference``, a
    linear test mode);
    ``dtype``: torch.float32 or torch.float64.  Work is ordered on ``stream``
    (default: the current torch stream of ``device``).
    """

    def __init__(self, lattice: str, D, grid: Sequence[int], *, bc="periodic",
                 relax: str = "magic", dtype=torch.float32, device="cuda",
                 stream: Optional[torch.cuda.Stream] = None, boundary=None, reference=None):
        if not torch.cuda.is_available():
            raise LbmsError("the lbms solver needs a CUDA device")
        self.lattice = lattice
        self.D = np.asarray(D, dtype=np.float64)
        self.n = int(self.D.shape[0])
        g = list(grid) + [1] * (3 - len(grid))
        self.grid = tuple(int(v) for v in g)
        self.dim = DIMS[lattice]
        self.dtype = dtype
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        lat, dt = LATTICES[lattice], DTYPES[dtype]
        nbytes = lbms_workspace_size(lat, self.n, self.grid, dt)
        if nbytes == 0:
            raise LbmsError("invalid lattice/species/grid/dtype combination")
        # workspace: raw bytes owned by torch, 256-byte aligned by the caching allocator
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = lbms_create(lat, self.n, self.grid, self.D, RELAX[relax], bc, dt,
                              self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)
        for face, xi_b in (boundary or {}).items():
            self.set_boundary(face, xi_b)
        if reference is not None:
            self.set_reference(reference)

    def set_reference(self, xi_ref) -> None:
        """Reference composition (all n species) of a "frozen" solver."""
        lbms_set_reference(self._h, xi_ref)

    def set_boundary(self, face: int, xi_b) -> None:
        """Composition (all n species) held on Dirichlet face ``face`` (0..5 as in
        ``bc``); applies to the steps issued after this call."""
        lbms_set_boundary(self._h, face, xi_b)

    def set_subdomain(self, first_layer: int) -> None:
        """Index of this slab's first layer along the split axis in the undivided
        grid (slab decomposition; see ``slab.py``)."""
        lbms_set_subdomain(self._h, first_layer)

    def halo_buffers(self, face: int):
        """(send, receive) views of cut face ``face`` (0..5 as in ``bc``): tensors
        [halo width, n - 1, layer nodes] in the workspace.  The receive buffer is
        the one the next step reads (it alternates with the population buffers)."""
        send, recv, nbytes = lbms_halo_buffers(self._h, face)
        base = self.workspace.data_ptr()
        es = 8 if self.dtype == torch.float64 else 4
        plane = {3: self.grid[0] * self.grid[1], 2: self.grid[0], 1: 1}[self.dim]
        width = nbytes // (es * (self.n - 1) * plane)

        def view(addr):
            raw = self.workspace[addr - base: addr - base + nbytes]
            return raw.view(self.dtype).view(width, self.n - 1, plane)

        return view(send), view(recv)

    @property
    def field_shape(self):
        nx, ny, nz = self.grid
        return (self.n, nz, ny, nx)

    @property
    def flux_shape(self):
        nx, ny, nz = self.grid
        return (self.n, self.dim, nz, ny, nx)

    def _field(self, t: torch.Tensor, shape) -> torch.Tensor:
        if tuple(t.shape) != tuple(shape) or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError("expected a contiguous %s tensor of shape %s" % (self.dtype, shape))
        return t

    def set_state(self, x0) -> None:
        if isinstance(x0, np.ndarray):
            x0 = torch.from_numpy(np.ascontiguousarray(x0)).to(self.dtype)
        x0 = self._field(x0, self.field_shape)
        lbms_set_state(self._h, x0.data_ptr())
        self._keep = x0  # host sources must live until the copies ran
        if not x0.is_cuda:
            self.stream.synchronize()

    def step(self, n: int) -> None:
        lbms_step(self._h, n)

    def moments(self, x_out: Optional[torch.Tensor] = None, J_out: Optional[torch.Tensor] = None,
                flux: bool = False):
        if x_out is None:
            x_out = torch.empty(self.field_shape, dtype=self.dtype, device=self.device)
        self._field(x_out, self.field_shape)
        if flux and J_out is None:
            J_out = torch.empty(self.flux_shape, dtype=self.dtype, device=x_out.device)
        if J_out is not None:
            self._field(J_out, self.flux_shape)
        lbms_moments(self._h, x_out.data_ptr(), J_out.data_ptr() if J_out is not None else None)
        return (x_out, J_out) if J_out is not None else x_out

    def gradient(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Local mole-fraction gradients of Eq. xix, [n, dim, nz, ny, nx]."""
        if out is None:
            out = torch.empty(self.flux_shape, dtype=self.dtype, device=self.device)
        self._field(out, self.flux_shape)
        lbms_gradient(self._h, out.data_ptr())
        return out

    def mass(self) -> np.ndarray:
        return lbms_mass(self._h, self.n)

    @property
    def state_shape(self):
        nx, ny, nz = self.grid
        return (self.n - 1, Q_OF[self.lattice], nx * ny * nz)

    def get_state(self, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Copy of the post-collision populations [n - 1, Q, cells] (a checkpoint)."""
        if out is None:
            out = torch.empty(self.state_shape, dtype=self.dtype, device=self.device)
        _check(self._h, load().lbms_get_state(self._h, ctypes.c_void_p(out.data_ptr())), "lbms_get_state")
        return out

    def set_state_raw(self, f: torch.Tensor, step: int) -> None:
        """Load a checkpoint taken after ``step`` steps."""
        f = self._field(f, self.state_shape)
        _check(self._h, load().lbms_set_state_raw(self._h, ctypes.c_void_p(f.data_ptr()), int(step)),
               "lbms_set_state_raw")
        self._keep = f

    def recompute(self, f_in: torch.Tensor, step: int, count: int, out: torch.Tensor) -> None:
        """Forward steps step+1 .. step+count from f_in into out[0 .. count-1]
        (bit-identical to ``step``); the handle's state is left unchanged."""
        if out.dtype != self.dtype or out.numel() < count * int(np.prod(self.state_shape)):
            raise ValueError("out must hold count states of the solver's dtype")
        _check(self._h, load().lbms_recompute(self._h, ctypes.c_void_p(f_in.data_ptr()), int(step),
                                              int(count), ctypes.c_void_p(out.data_ptr())),
               "lbms_recompute")

    def adjoint_state(self) -> torch.Tensor:
        """An adjoint-state buffer: FP64 [n-1, Q, cells] for FP64 solvers, and
        [n-1, Q, cells, 2] float pairs (hi, lo) for FP32 solvers."""
        if self.dtype == torch.float64:
            return torch.empty(self.state_shape, dtype=torch.float64, device=self.device)
        return torch.empty(self.state_shape + (2,), dtype=torch.float32, device=self.device)

    @staticmethod
    def adjoint_value(lam: torch.Tensor) -> torch.Tensor:
        """The adjoint state as FP64 values (sums the float pairs)."""
        if lam.dtype == torch.float64:
            return lam
        return lam[..., 0].double() + lam[..., 1].double()

    def adjoint_scratch(self) -> torch.Tensor:
        nbytes = int(load().lbms_adjoint_scratch_size(self._h))
        if nbytes == 0:
            raise LbmsError("the adjoint supports up to 5 species and not the frozen mode")
        return torch.zeros(nbytes // 8, dtype=torch.float64, device=self.device)

    def adjoint_seed(self, grad_x: torch.Tensor, lam: torch.Tensor) -> None:
        grad_x = self._field(grad_x.contiguous(), self.field_shape)
        _check(self._h, load().lbms_adjoint_seed(self._h, ctypes.c_void_p(grad_x.data_ptr()),
                                                 ctypes.c_void_p(lam.data_ptr())), "lbms_adjoint_seed")

    def adjoint_step(self, f_prev: torch.Tensor, lam_in: torch.Tensor, lam_out: torch.Tensor,
                     gacc: torch.Tensor) -> None:
        _check(self._h, load().lbms_adjoint_step(self._h, ctypes.c_void_p(f_prev.data_ptr()),
                                                 ctypes.c_void_p(lam_in.data_ptr()),
                                                 ctypes.c_void_p(lam_out.data_ptr()),
                                                 ctypes.c_void_p(gacc.data_ptr())), "lbms_adjoint_step")

    def adjoint_steps(self, f_first: torch.Tensor, f_rest: Optional[torch.Tensor], count: int,
                      lam_a: torch.Tensor, lam_b: torch.Tensor, gacc: torch.Tensor) -> None:
        """``count`` adjoint steps of a segment in one call (lbms_adjoint_steps):
        forward states f_first = f+(t0) and f_rest[j] = f+(t0 + 1 + j); lambda
        starts in lam_a and ends in lam_a (even count) or lam_b (odd count)."""
        rest = ctypes.c_void_p(f_rest.data_ptr()) if f_rest is not None else None
        _check(self._h, load().lbms_adjoint_steps(self._h, ctypes.c_void_p(f_first.data_ptr()), rest,
                                                  int(count), ctypes.c_void_p(lam_a.data_ptr()),
                                                  ctypes.c_void_p(lam_b.data_ptr()),
                                                  ctypes.c_void_p(gacc.data_ptr())), "lbms_adjoint_steps")

    def adjoint_initial(self, lam0: torch.Tensor) -> torch.Tensor:
        out = torch.empty(self.field_shape, dtype=self.dtype, device=self.device)
        _check(self._h, load().lbms_adjoint_initial(self._h, ctypes.c_void_p(lam0.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr())), "lbms_adjoint_initial")
        return out

    def adjoint_reduce(self, gacc: torch.Tensor) -> np.ndarray:
        out = np.zeros(self.n * (self.n - 1) // 2, dtype=np.float64)
        _check(self._h, load().lbms_adjoint_reduce(self._h, ctypes.c_void_p(gacc.data_ptr()),
                                                   out.ctypes.data_as(ctypes.c_void_p)), "lbms_adjoint_reduce")
        return out

    def populations(self) -> torch.Tensor:
        """View of the current population buffer, shape [n - 1, Q, cells]."""
        q = Q_OF[self.lattice]
        es = 8 if self.dtype == torch.float64 else 4
        nx, ny, nz = self.grid
        cells = nx * ny * nz
        nbytes = (self.n - 1) * q * cells * es
        off = int(load().lbms_populations(self._h)) - self.workspace.data_ptr()
        return self.workspace[off:off + nbytes].view(self.dtype).view(self.n - 1, q, cells)

    def status(self) -> int:
        return lbms_status(self._h)

    @property
    def steps_done(self) -> int:
        return lbms_steps_done(self._h)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lbms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- batched solves --------------------------------------------------------

def _bcheck(b, rc: int, what: str) -> None:
    if rc != LBMS_OK:
        raise LbmsError("%s: %s (%s)" % (what, ERRORS.get(rc, rc),
                                         load().lbms_batch_last_error(b).decode()))


def lbms_batch_workspace_size(lattice: int, n_species: int, grids, dtype: int) -> int:
    g = np.ascontiguousarray(np.asarray(grids, dtype=np.int32).reshape(-1, 3))
    return int(load().lbms_batch_workspace_size(lattice, n_species, g.shape[0],
                                                g.ctypes.data_as(ctypes.c_void_p), dtype))


class BatchSolver:
    """Many independent solves of one lattice / species count / dtype.

    ``grids``: list of (nx, ny[, nz]); ``Ds``: list (or array) of n x n
    diffusivity matrices; ``bcs``: None (all periodic) or a list of 6-tuples of
    face kinds ("periodic", "noflux", "dirichlet"); ``boundary``:
    {(instance, face): composition of all n species} for the Dirichlet faces.  Fields are exchanged as lists of [n, nz, ny, nx] tensors or as
    one packed 1-D tensor (instance after instance).
    """

    def __init__(self, lattice: str, Ds, grids, *, bcs=None, relax: str = "magic",
                 dtype=torch.float32, device="cuda", stream: Optional[torch.cuda.Stream] = None,
                 boundary=None):
        if not torch.cuda.is_available():
            raise LbmsError("the lbms solver needs a CUDA device")
        L = load()
        self.lattice = lattice
        self.dim = DIMS[lattice]
        self.dtype = dtype
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.grids = [tuple(int(v) for v in (list(g) + [1] * (3 - len(g)))) for g in grids]
        self.count = len(self.grids)
        D = np.ascontiguousarray(np.asarray(Ds, dtype=np.float64).reshape(self.count, -1))
        self.n = int(round(D.shape[1] ** 0.5))
        self.cells = [g[0] * g[1] * g[2] for g in self.grids]
        self.offsets = np.zeros(self.count + 1, dtype=np.int64)
        self.offsets[1:] = np.cumsum([self.n * c for c in self.cells])
        g = np.ascontiguousarray(np.asarray(self.grids, dtype=np.int32))
        self._g = g
        dt = DTYPES[dtype]
        nbytes = int(L.lbms_batch_workspace_size(LATTICES[lattice], self.n, self.count,
                                                 g.ctypes.data_as(ctypes.c_void_p), dt))
        if nbytes == 0:
            raise LbmsError("invalid batch (lattice/species/grids/dtype)")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        bc = None
        if bcs is not None:
            bc = np.ascontiguousarray(np.array(
                [[FACE[v] if isinstance(v, str) else int(v) for v in (b if not isinstance(b, str) else (b,) * 6)]
                 for b in bcs], dtype=np.int32))
        self._h = ctypes.c_void_p()
        rc = L.lbms_batch_create(ctypes.byref(self._h), LATTICES[lattice], self.n, self.count,
                                 g.ctypes.data_as(ctypes.c_void_p), D.ctypes.data_as(ctypes.c_void_p),
                                 RELAX[relax], bc.ctypes.data_as(ctypes.c_void_p) if bc is not None else None,
                                 dt, ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                 ctypes.c_void_p(self.stream.cuda_stream))
        if rc != LBMS_OK:
            self._h = None
            raise LbmsError("lbms_batch_create: %s (%s)" % (ERRORS.get(rc, rc),
                                                            L.lbms_batch_last_error(None).decode()))
        for (inst, face), xi_b in (boundary or {}).items():
            self.set_boundary(inst, face, xi_b)

    def set_boundary(self, instance: int, face: int, xi_b) -> None:
        """Composition (all n species) held on Dirichlet face ``face`` of instance
        ``instance`` (lbms_batch_set_boundary)."""
        v = np.ascontiguousarray(np.asarray(xi_b, dtype=np.float64).reshape(-1))
        _bcheck(self._h, load().lbms_batch_set_boundary(self._h, int(instance), int(face),
                                                        v.ctypes.data_as(ctypes.c_void_p)),
                "lbms_batch_set_boundary")

    def pack(self, fields) -> torch.Tensor:
        """Concatenate per-instance [n, nz, ny, nx] arrays into one flat tensor."""
        parts = [torch.as_tensor(np.ascontiguousarray(f) if isinstance(f, np.ndarray) else f)
                 .reshape(-1).to(self.dtype) for f in fields]
        return torch.cat(parts)

    def unpack(self, flat: torch.Tensor, per=1, flux: bool = False):
        """Per-instance views of a packed field: mole fractions [n, nz, ny, nx], or
        with ``flux`` (or ``per`` > 1) fluxes [n, dim, nz, ny, nx] (``per`` = dim)."""
        flux = flux or per > 1
        per = self.dim if flux else per
        out = []
        for i, (nx, ny, nz) in enumerate(self.grids):
            a, b = int(self.offsets[i]) * per, int(self.offsets[i + 1]) * per
            shape = (self.n, self.dim, nz, ny, nx) if flux else (self.n, nz, ny, nx)
            out.append(flat[a:b].view(shape))
        return out

    def set_state(self, x0) -> None:
        flat = x0 if isinstance(x0, torch.Tensor) and x0.dim() == 1 else self.pack(x0)
        if flat.numel() != int(self.offsets[-1]) or flat.dtype != self.dtype:
            raise ValueError("packed field has the wrong size or dtype")
        flat = flat.contiguous()
        _bcheck(self._h, load().lbms_batch_set_state(self._h, ctypes.c_void_p(flat.data_ptr()), None),
                "lbms_batch_set_state")
        self._keep = flat

    def step(self, n: int) -> None:
        _bcheck(self._h, load().lbms_batch_step(self._h, int(n)), "lbms_batch_step")

    def moments(self, flux: bool = False, out_device=None):
        dev = self.device if out_device is None else torch.device(out_device)
        pin = dev.type == "cpu"  # host outputs pinned: the moments kernel writes them in place
        x = torch.empty(int(self.offsets[-1]), dtype=self.dtype, device=dev, pin_memory=pin)
        J = (torch.empty(int(self.offsets[-1]) * self.dim, dtype=self.dtype, device=dev, pin_memory=pin)
             if flux else None)
        _bcheck(self._h, load().lbms_batch_moments(self._h, ctypes.c_void_p(x.data_ptr()),
                                                   ctypes.c_void_p(J.data_ptr()) if J is not None else None,
                                                   None), "lbms_batch_moments")
        return (x, J) if flux else x

    def mass(self) -> np.ndarray:
        out = np.zeros(self.count * self.n, dtype=np.float64)
        _bcheck(self._h, load().lbms_batch_mass(self._h, out.ctypes.data_as(ctypes.c_void_p)), "lbms_batch_mass")
        return out.reshape(self.count, self.n)

    def status(self) -> int:
        fl = ctypes.c_uint32()
        _bcheck(self._h, load().lbms_batch_status(self._h, ctypes.byref(fl)), "lbms_batch_status")
        return int(fl.value)

    def set_schedule(self, candidate: int) -> None:
        _bcheck(self._h, load().lbms_batch_set_schedule(self._h, int(candidate)), "lbms_batch_set_schedule")

    @property
    def schedule(self) -> int:
        return int(load().lbms_batch_get_schedule(self._h))

    def launches_per_step(self) -> int:
        """Step-kernel launches per step under the current schedule."""
        return int(load().lbms_batch_launches_per_step(self._h))

    def tune(self, trial_steps: int = 32):
        """Time every step candidate (schedule x kernel shape) and keep the fastest
        (advances the state: call before set_state).  Returns (chosen, ms_per_step
        of each candidate; -1 for the candidates this batch cannot run)."""
        times = np.zeros(BATCH_CANDIDATES, dtype=np.float64)
        chosen = ctypes.c_int()
        _bcheck(self._h, load().lbms_batch_tune(self._h, int(trial_steps), times.ctypes.data_as(ctypes.c_void_p),
                                                ctypes.byref(chosen)), "lbms_batch_tune")
        return int(chosen.value), times

    @property
    def steps_done(self) -> int:
        return int(load().lbms_batch_steps_done(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().lbms_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
