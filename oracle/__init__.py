"""FP64 CPU oracle of the Maxwell-Stefan MRT lattice Boltzmann model (arXiv:1808.06787).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package, and this package never imports the product.

The arithmetic lives in ``ms_mrt_oracle.c`` (plain C, FP64, written literally
from the paper's equations; see its header for the equation-by-equation map).
This module only compiles it with gcc into ``oracle/_build/`` and marshals
NumPy arrays through ctypes.

Every function is pinned by ``tests/test_oracle_pins.py`` against closed forms,
exact discrete predictions and numbers printed in the paper.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_mrt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libmsoracle.so")
_lock = threading.Lock()
_lib = None

LATTICES = {"D2Q5": 0, "D2Q9": 1, "D3Q7": 2, "D3Q15": 3, "D1Q3": 4, "D2Q4": 5, "D3Q6": 6}
RELAX = {"magic": 0, "srt": 1, "frozen": 2}
BC = {"periodic": 0, "noflux": 1, "dirichlet": 2}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
            "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            I = ctypes.c_int
            L.orc_lattice_info.argtypes = [I, P, P, P, P, P, P]
            L.orc_moment_basis.argtypes = [I, P, P, P]
            L.orc_B.argtypes = [I, P, P, P]
            L.orc_Dtilde.argtypes = [I, P, P, P]
            L.orc_lambdas.argtypes = [I, I, P, P, I, P, P]
            L.orc_collide_node.argtypes = [I, I, P, I, P, P]
            L.orc_run.argtypes = [I, I, I, I, I, P, I, P, P, P, ctypes.c_long, P, P, P]
            L.orc_run_snap.argtypes = [I, I, I, I, I, P, I, P, P, P, ctypes.c_long, P, P, P,
                                       I, P, P]
            L.orc_set_reference.argtypes = [I, P]
            L.orc_set_threads.argtypes = [I]
            L.orc_get_threads.restype = I
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def lattice_info(lattice: str):
    """(Q, dim, c[Q,3], w[Q], opp[Q], c_s^2) in the paper's velocity order."""
    c = np.zeros((15, 3), dtype=np.int32)
    w = np.zeros(15)
    opp = np.zeros(15, dtype=np.int32)
    Q = ctypes.c_int()
    dim = ctypes.c_int()
    cs2 = ctypes.c_double()
    rc = lib().orc_lattice_info(LATTICES[lattice], ctypes.byref(Q), ctypes.byref(dim),
                                _p(c), _p(w), _p(opp), ctypes.byref(cs2))
    assert rc == 0
    q = Q.value
    return q, dim.value, c[:q].copy(), w[:q].copy(), opp[:q].copy(), cs2.value


def moment_basis(lattice: str):
    """(M, M^{-1}, group) with group 0 = conserved, 1 = odd order, 2 = even order."""
    q = lattice_info(lattice)[0]
    M = np.zeros((q, q))
    Mi = np.zeros((q, q))
    g = np.zeros(q, dtype=np.int32)
    assert lib().orc_moment_basis(LATTICES[lattice], _p(M), _p(Mi), _p(g)) == 0
    return M, Mi, g


def B_matrix(xi, D) -> np.ndarray:
    """B of Eq. 2-10 from all n mole fractions and the n x n diffusivities."""
    xi = _f64(xi)
    D = _f64(D)
    n = xi.size
    out = np.zeros((n - 1, n - 1))
    assert lib().orc_B(n, _p(xi), _p(D), _p(out)) == 0
    return out


def Dtilde(xi, D) -> np.ndarray:
    """Generalised Fick matrix D~ = B^{-1} (Eq. 2-11)."""
    xi = _f64(xi)
    D = _f64(D)
    n = xi.size
    out = np.zeros((n - 1, n - 1))
    assert lib().orc_Dtilde(n, _p(xi), _p(D), _p(out)) == 0
    return out


def lambdas(lattice: str, xi, D, relax: str = "magic"):
    """(Lambda_1, Lambda_2) at one node: Eq. 3-26 and Eq. 3-16."""
    xi = _f64(xi)
    D = _f64(D)
    n = xi.size
    L1 = np.zeros((n - 1, n - 1))
    L2 = np.zeros((n - 1, n - 1))
    assert lib().orc_lambdas(LATTICES[lattice], n, _p(xi), _p(D), RELAX[relax],
                             _p(L1), _p(L2)) == 0
    return L1, L2


def collide_node(lattice: str, D, fs, relax: str = "magic") -> np.ndarray:
    """Post-collision populations of one node; fs[s, k] in the paper's velocity order."""
    D = _f64(D)
    fs = _f64(fs)
    n = D.shape[0]
    out = np.zeros_like(fs)
    assert lib().orc_collide_node(LATTICES[lattice], n, _p(D), RELAX[relax], _p(fs), _p(out)) == 0
    return out


def run(lattice: str, D, x0, steps: int, *, bc=("periodic",) * 6, relax: str = "magic",
        flux: bool = False, snapshots=None, xb=None, grad: bool = False, xi_ref=None):
    """Run the scheme from f = f_eq(x0) for ``steps`` steps.

    ``x0`` is [n, nz, ny, nx] (all n species).  ``bc`` names the six faces
    (x-low, x-high, y-low, y-high, z-low, z-high) "periodic", "noflux" or
    "dirichlet"; ``xb`` is [6, n], the composition held on each Dirichlet face
    (rows of other faces are ignored).  Returns ``x`` of the same shape at
    t = steps; ``relax="frozen"`` evaluates the relaxation matrices (and the
    flux's D~) at the fixed composition ``xi_ref`` (n values), which makes the
    scheme linear.  With ``flux=True`` also ``J`` of shape [n, dim, nz, ny, nx]; with
    ``grad=True`` also the local gradients of Eq. xix, same shape; with
    ``snapshots`` (ascending step counts <= steps) also the mole-fraction fields
    at those steps, shape [len(snapshots), n, nz, ny, nx].
    """
    D = _f64(D)
    x0 = _f64(x0)
    n, nz, ny, nx = x0.shape
    q, dim = lattice_info(lattice)[:2]
    bcs = np.asarray([BC[b] if isinstance(b, str) else int(b) for b in bc], dtype=np.int32)
    if relax == "frozen":
        ref = _f64(np.asarray(xi_ref, dtype=np.float64).reshape(-1))
        if ref.size != n or lib().orc_set_reference(n, _p(ref)) != 0:
            raise ValueError("relax='frozen' needs xi_ref with n mole fractions")
    if xb is not None:
        xb = _f64(np.nan_to_num(np.asarray(xb, dtype=np.float64)).reshape(6, n))
    xo = np.zeros_like(x0)
    Jo = np.zeros((n, dim, nz, ny, nx)) if flux else None
    Go = np.zeros((n, dim, nz, ny, nx)) if grad else None
    if snapshots is not None:
        snap = np.ascontiguousarray(np.asarray(snapshots, dtype=np.int64))
        if snap.size and (np.any(np.diff(snap) <= 0) or snap[0] < 0 or snap[-1] > steps):
            raise ValueError("snapshots must be ascending step counts within [0, steps]")
        so = np.zeros((snap.size,) + x0.shape)
        rc = lib().orc_run_snap(LATTICES[lattice], n, nx, ny, nz, _p(D), RELAX[relax], _p(bcs),
                                None if xb is None else _p(xb), _p(x0), int(steps), _p(xo), _p(Jo) if flux else None,
                                _p(Go) if grad else None, int(snap.size), _p(snap), _p(so))
    else:
        so = None
        rc = lib().orc_run(LATTICES[lattice], n, nx, ny, nz, _p(D), RELAX[relax], _p(bcs),
                           None if xb is None else _p(xb), _p(x0), int(steps), _p(xo), _p(Jo) if flux else None,
                           _p(Go) if grad else None)
    if rc != 0:
        raise RuntimeError("oracle run failed with code %d" % rc)
    out = [xo]
    if flux:
        out.append(Jo)
    if grad:
        out.append(Go)
    if snapshots is not None:
        out.append(so)
    return out[0] if len(out) == 1 else tuple(out)
