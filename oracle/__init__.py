"""Plain FP64 CPU oracle for the even-odd Wilson-Dirac hot path (BSMBench,
Sec. II-A field content, Sec. II-B Dirac operator and CG).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.  The arithmetic
lives in oracle.c; this module only marshals numpy arrays through ctypes.

Array conventions (canonical layout, complex128):
  links    U[site, mu, a, b]        (N x N fundamental, or d x d representation)
  spinors  psi[site, spin, colour]  shape (V, 4, d)
with site = ((t*X + x)*Y + y)*Z + z and dims = (T, X, Y, Z).
"""
import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

FUND, ADJ, SYM, ASYM = 0, 1, 2, 3
EVEN, ODD, FULL = 0, 1, 2
DHAT, DHAT_DAG, DHAT_DAG_DHAT = 0, 1, 2


class _Lat(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("N", ctypes.c_int), ("rep", ctypes.c_int),
                ("m0", ctypes.c_double), ("phase", ctypes.c_double * 4)]


@dataclass
class Lattice:
    dims: tuple          # (T, X, Y, Z)
    N: int
    rep: int = FUND
    m0: float = 0.1
    phase: tuple = field(default=(0.0, 0.0, 0.0, 0.0))

    @property
    def V(self):
        return int(np.prod(self.dims))

    @property
    def d(self):
        return rep_dim(self.N, self.rep)

    def c(self):
        return _Lat((ctypes.c_int * 4)(*self.dims), self.N, self.rep, self.m0,
                    (ctypes.c_double * 4)(*self.phase))


_lib = None


def _load(path):
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    LP = ctypes.POINTER(_Lat)
    L.orc_rep_dim.argtypes = [ctypes.c_int, ctypes.c_int]
    L.orc_gamma.argtypes = [ctypes.c_int, P]
    L.orc_rep_matrix.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
    L.orc_links_to_rep.argtypes = [LP, P, P]
    L.orc_hop.argtypes = [LP, P, P, P, ctypes.c_int, ctypes.c_int]
    L.orc_dirac.argtypes = [LP, P, P, P, ctypes.c_int]
    L.orc_dhat.argtypes = [LP, P, P, P, ctypes.c_int]
    L.orc_cg.argtypes = [LP, P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                         ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.orc_dense_dirac.argtypes = [LP, P, P]
    L.orc_lu_solve.argtypes = [ctypes.c_int, P, P]
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def use_library(path):
    """Route the wrappers below through another build of oracle.c (used by
    the mutation tests, which plant mistakes in a copy of the source).
    Returns the previous handle for restore_library()."""
    global _lib
    prev = lib()
    _lib = _load(path)
    return prev


def restore_library(handle):
    global _lib
    _lib = handle


def _c(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def rep_dim(N, rep):
    return lib().orc_rep_dim(N, rep)


def gamma(mu):
    g = np.zeros((4, 4), np.complex128)
    lib().orc_gamma(mu, g.ctypes.data_as(ctypes.c_void_p))
    return g


def rep_matrix(N, rep, U):
    d = rep_dim(N, rep)
    U, pu = _c(U)
    R = np.zeros((d, d), np.complex128)
    if lib().orc_rep_matrix(N, rep, pu, R.ctypes.data_as(ctypes.c_void_p)):
        raise ValueError("unsupported representation")
    return R


def links_to_rep(lat, U):
    U, pu = _c(U)
    R = np.zeros((lat.V, 4, lat.d, lat.d), np.complex128)
    lc = lat.c()
    if lib().orc_links_to_rep(ctypes.byref(lc), pu, R.ctypes.data_as(ctypes.c_void_p)):
        raise ValueError("unsupported representation")
    return R


def hop(lat, R, psi, out_parity=FULL, dagger=False):
    R, pr = _c(R)
    psi, pp = _c(psi)
    out = np.zeros_like(psi)
    lc = lat.c()
    lib().orc_hop(ctypes.byref(lc), pr, pp, out.ctypes.data_as(ctypes.c_void_p),
                  out_parity, int(dagger))
    return out


def dirac(lat, R, psi, dagger=False):
    R, pr = _c(R)
    psi, pp = _c(psi)
    out = np.zeros_like(psi)
    lc = lat.c()
    lib().orc_dirac(ctypes.byref(lc), pr, pp, out.ctypes.data_as(ctypes.c_void_p), int(dagger))
    return out


def dhat(lat, R, psi, op=DHAT):
    R, pr = _c(R)
    psi, pp = _c(psi)
    out = np.zeros_like(psi)
    lc = lat.c()
    lib().orc_dhat(ctypes.byref(lc), pr, pp, out.ctypes.data_as(ctypes.c_void_p), op)
    return out


def cg(lat, R, b, eo=True, tol=1e-10, max_iter=10000, x0=None):
    """Returns (x, iterations, iterated relative residual); iterations = -1
    when max_iter was reached."""
    R, pr = _c(R)
    b, pb = _c(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128, copy=True)
    res = ctypes.c_double(0.0)
    lc = lat.c()
    it = lib().orc_cg(ctypes.byref(lc), pr, pb, x.ctypes.data_as(ctypes.c_void_p), int(eo),
                      tol, max_iter, int(x0 is not None), ctypes.byref(res))
    return x, it, res.value


def dense_dirac(lat, R):
    R, pr = _c(R)
    n = lat.V * 4 * lat.d
    M = np.zeros((n, n), np.complex128)
    lc = lat.c()
    lib().orc_dense_dirac(ctypes.byref(lc), pr, M.ctypes.data_as(ctypes.c_void_p))
    return M


def lu_solve(A, b):
    A = np.array(A, dtype=np.complex128, copy=True, order="C")
    x = np.array(b, dtype=np.complex128, copy=True)
    if lib().orc_lu_solve(A.shape[0], A.ctypes.data_as(ctypes.c_void_p),
                          x.ctypes.data_as(ctypes.c_void_p)):
        raise ZeroDivisionError("singular matrix")
    return x


def parity_mask(dims):
    """Boolean (V,) array, True on odd sites."""
    T, X, Y, Z = dims
    t, x, y, z = np.meshgrid(np.arange(T), np.arange(X), np.arange(Y), np.arange(Z), indexing="ij")
    return ((t + x + y + z) % 2 == 1).reshape(-1)
