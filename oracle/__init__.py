"""FP64 CPU oracle for the spectral-element pressure-Poisson path.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or calls anything here, and this package never imports the
library: the two share no code.  Inputs (mesh vertices, right-hand sides) come
to both from ``paper_2405_05640_gb300.inputs``, which holds no arithmetic of
the method.

The numerics live in ``sem_oracle.c`` (plain loops, FP64, single thread),
compiled here with gcc on first use.  Each wrapper names the definition it
follows; the paper (Karp et al., arXiv 2405.05640, section 3.1 "Neko") gives
the method in prose and refers the formulas to Deville, Fischer & Mund (2002).

Functions with no independent pin: none -- every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` (closed forms, invariants,
brute-force dense assembly and spectral convergence).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sem_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_LIBDIR, "libsem_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, EMESH, ENAN, ENOTCONV = 0, -1, -3, -5, -6

_D = ctypes.POINTER(ctypes.c_double)
_L = ctypes.POINTER(ctypes.c_long)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_ubyte)


def build() -> str:
    """Compile sem_oracle.c into oracle/_lib/libsem_oracle.so (gcc, -O2, no
    fast-math so that FP64 semantics are IEEE)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.or_legendre.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D]
            lib.or_gll.argtypes = [ctypes.c_int, _D, _D]
            lib.or_gll.restype = ctypes.c_int
            lib.or_deriv.argtypes = [ctypes.c_int, _D, _D]
            lib.or_geometry.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D, _D, _D, _D, _D]
            lib.or_geometry.restype = ctypes.c_int
            lib.or_box_numbering.argtypes = [ctypes.c_int, _I, _I, _L]
            lib.or_box_numbering.restype = ctypes.c_long
            lib.or_box_mask.argtypes = [ctypes.c_int, _I, _I, ctypes.c_int, _U8]
            lib.or_dssum.argtypes = [ctypes.c_long, _L, ctypes.c_long, _D, _D]
            lib.or_apply_mask.argtypes = [ctypes.c_long, _U8, _D]
            lib.or_ax_local.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D, _D]
            lib.or_helmholtz_local.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D,
                                               ctypes.c_double, ctypes.c_double, _D, _D]
            lib.or_jacobi_diag_local.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D]
            lib.or_glsc3.argtypes = [ctypes.c_long, _D, _D, _D]
            lib.or_glsc3.restype = ctypes.c_double
            lib.or_pcg.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D, ctypes.c_double,
                                   ctypes.c_double, _L, ctypes.c_long, _U8, _D, _D, _D, _D,
                                   ctypes.c_double, ctypes.c_int, _I, _D, _D]
            lib.or_pcg.restype = ctypes.c_int
            lib.or_inverse_jacobian.argtypes = [ctypes.c_int, ctypes.c_long, _D, _D, _D, _D]
            lib.or_inverse_jacobian.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, ptr):
    return a.ctypes.data_as(ptr)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def legendre(N: int, x: float) -> tuple[float, float]:
    """P_N(x) and P_N'(x) by the three-term recurrence."""
    P, dP = ctypes.c_double(), ctypes.c_double()
    _load().or_legendre(N, float(x), ctypes.byref(P), ctypes.byref(dP))
    return P.value, dP.value


def gll(N: int) -> tuple[np.ndarray, np.ndarray]:
    """GLL nodes xi (ascending, xi_0 = -1) and quadrature weights rho."""
    xi, rho = np.zeros(N + 1), np.zeros(N + 1)
    if _load().or_gll(N, _p(xi, _D), _p(rho, _D)) != OK:
        raise ValueError(f"invalid order N={N}")
    return xi, rho


def deriv(N: int, xi: np.ndarray | None = None) -> np.ndarray:
    """D[i, j] = l_j'(xi_i) for the GLL Lagrange basis."""
    if xi is None:
        xi = gll(N)[0]
    D = np.zeros((N + 1, N + 1))
    _load().or_deriv(N, _p(_f64(xi), _D), _p(D, _D))
    return D


def geometry(N: int, verts: np.ndarray):
    """(xyz[3,E,npt], G[E,6,npt], B[E,npt], status) for trilinear hexahedra;
    status is -3 when det J <= 0 somewhere."""
    verts = _f64(verts).reshape(-1, 8, 3)
    E = verts.shape[0]
    npt = (N + 1) ** 3
    xi, rho = gll(N)
    D = deriv(N, xi)
    xyz = np.zeros((3, E, npt))
    G = np.zeros((E, 6, npt))
    B = np.zeros((E, npt))
    st = _load().or_geometry(N, E, _p(verts, _D), _p(xi, _D), _p(rho, _D), _p(D, _D),
                             _p(xyz, _D), _p(G, _D), _p(B, _D))
    return xyz, G, B, st


def inverse_jacobian(N: int, verts: np.ndarray) -> np.ndarray:
    """RX[e, 3a+m, p] = dr_a/dx_m at the GLL points (trilinear hexahedra)."""
    verts = _f64(verts).reshape(-1, 8, 3)
    E = verts.shape[0]
    xi, _ = gll(N)
    D = deriv(N, xi)
    RX = np.zeros((E, 9, (N + 1) ** 3))
    st = _load().or_inverse_jacobian(N, E, _p(verts, _D), _p(xi, _D), _p(D, _D), _p(RX, _D))
    if st != OK:
        raise ValueError("det J <= 0")
    return RX


def box_numbering(N: int, nel, periodic) -> tuple[np.ndarray, int]:
    nel_a = np.asarray(nel, dtype=np.int32)
    per = np.asarray(periodic, dtype=np.int32)
    nloc = int(np.prod(nel_a.astype(np.int64))) * (N + 1) ** 3
    gid = np.zeros(nloc, dtype=np.int64)
    nglob = _load().or_box_numbering(N, _p(nel_a, _I), _p(per, _I), _p(gid, _L))
    return gid, int(nglob)


def box_mask(N: int, nel, periodic, faces: int) -> np.ndarray:
    nel_a = np.asarray(nel, dtype=np.int32)
    per = np.asarray(periodic, dtype=np.int32)
    nloc = int(np.prod(nel_a.astype(np.int64))) * (N + 1) ** 3
    mask = np.zeros(nloc, dtype=np.uint8)
    _load().or_box_mask(N, _p(nel_a, _I), _p(per, _I), int(faces), _p(mask, _U8))
    return mask


def dssum(u: np.ndarray, gid: np.ndarray, nglob: int) -> np.ndarray:
    """Q Q^T u (returns a new array)."""
    out = _f64(u).copy().reshape(-1)
    tmp = np.zeros(nglob)
    _load().or_dssum(out.size, _p(gid, _L), nglob, _p(out, _D), _p(tmp, _D))
    return out.reshape(np.shape(u))


def apply_mask(u: np.ndarray, mask: np.ndarray) -> np.ndarray:
    out = _f64(u).copy().reshape(-1)
    _load().or_apply_mask(out.size, _p(mask, _U8), _p(out, _D))
    return out.reshape(np.shape(u))


def ax_local(N: int, D: np.ndarray, G: np.ndarray, u: np.ndarray) -> np.ndarray:
    u = _f64(u)
    G = _f64(G)
    E = G.shape[0]
    w = np.zeros_like(u)
    _load().or_ax_local(N, E, _p(_f64(D), _D), _p(G, _D), _p(u, _D), _p(w, _D))
    return w


def helmholtz_local(N, D, G, B, h1, h2, u):
    u = _f64(u)
    G = _f64(G)
    w = np.zeros_like(u)
    _load().or_helmholtz_local(N, G.shape[0], _p(_f64(D), _D), _p(G, _D), _p(_f64(B), _D),
                               float(h1), float(h2), _p(u, _D), _p(w, _D))
    return w


def jacobi_diag_local(N, D, G):
    G = _f64(G)
    E = G.shape[0]
    d = np.zeros((E, (N + 1) ** 3))
    _load().or_jacobi_diag_local(N, E, _p(_f64(D), _D), _p(G, _D), _p(d, _D))
    return d


def glsc3(a, b, minv) -> float:
    a, b, minv = _f64(a).reshape(-1), _f64(b).reshape(-1), _f64(minv).reshape(-1)
    return _load().or_glsc3(a.size, _p(a, _D), _p(b, _D), _p(minv, _D))


class Mesh:
    """Everything the oracle derives from a box topology plus vertex array:
    GLL data, geometric factors, numbering, mask, multiplicity and the
    assembled Jacobi preconditioner."""

    def __init__(self, N: int, nel, periodic, dirichlet_faces: int, verts: np.ndarray):
        self.N = int(N)
        self.nel = tuple(int(a) for a in nel)
        self.periodic = tuple(int(bool(a)) for a in periodic)
        self.faces = int(dirichlet_faces)
        self.E = int(np.prod(self.nel))
        self.npt = (self.N + 1) ** 3
        self.nloc = self.E * self.npt
        self.xi, self.rho = gll(self.N)
        self.D = deriv(self.N, self.xi)
        self.xyz, self.G, self.B, self.status = geometry(self.N, verts)
        if self.status != OK:
            raise ValueError("mesh has det J <= 0")
        self.gid, self.nglob = box_numbering(self.N, self.nel, self.periodic)
        self.mask = box_mask(self.N, self.nel, self.periodic, self.faces)
        self.mult = dssum(np.ones(self.nloc), self.gid, self.nglob)
        self.minv = 1.0 / self.mult
        self.h1, self.h2 = 1.0, 0.0
        self._set_diag()

    def _set_diag(self):
        d = self.h1 * jacobi_diag_local(self.N, self.D, self.G).reshape(-1)
        if self.h2 != 0.0:
            d = d + self.h2 * self.B.reshape(-1)
        d = dssum(d, self.gid, self.nglob)
        self.diag = d
        self.dinv = np.where(self.mask.astype(bool), 0.0, 1.0 / d)

    def set_helmholtz(self, h1: float, h2: float):
        """Switch the operator to h1*A + h2*B (Poisson: h1=1, h2=0)."""
        self.h1, self.h2 = float(h1), float(h2)
        self._set_diag()

    def ax_local(self, u):
        return ax_local(self.N, self.D, self.G, np.reshape(u, (self.E, self.npt))).reshape(-1)

    def dssum(self, u):
        return dssum(np.reshape(u, -1), self.gid, self.nglob)

    def apply_mask(self, u):
        return apply_mask(np.reshape(u, -1), self.mask)

    def apply(self, u):
        """Assembled operator M Q Q^T (h1 A_L + h2 B) u."""
        if self.h2 == 0.0:
            w = self.h1 * self.ax_local(u)
        else:
            w = helmholtz_local(self.N, self.D, self.G, self.B, self.h1, self.h2,
                                np.reshape(u, (self.E, self.npt))).reshape(-1)
        return self.apply_mask(self.dssum(w))

    def glsc3(self, a, b):
        return glsc3(a, b, self.minv)

    def scatter(self, u_glob):
        """Q u_glob: copy each global value to all of its local copies."""
        return np.asarray(u_glob, dtype=np.float64)[self.gid]

    def pcg(self, b, x0=None, tol=1e-10, max_iter=10000):
        """Jacobi-PCG; returns (x, iters, rel_res, status)."""
        b = _f64(b).reshape(-1)
        x = np.zeros(self.nloc) if x0 is None else _f64(x0).reshape(-1).copy()
        work = np.zeros(4 * self.nloc + self.nglob)
        it, rr = ctypes.c_int(), ctypes.c_double()
        st = _load().or_pcg(self.N, self.E, _p(self.D, _D), _p(self.G, _D), _p(self.B, _D),
                            self.h1, self.h2, _p(self.gid, _L), self.nglob, _p(self.mask, _U8),
                            _p(self.minv, _D), _p(self.dinv, _D), _p(b, _D), _p(x, _D),
                            float(tol), int(max_iter), ctypes.byref(it), ctypes.byref(rr),
                            _p(work, _D))
        return x, it.value, rr.value, st
