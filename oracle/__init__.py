"""HODLR2D CPU oracle (FP64): Python bindings over ``oracle.c``.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs are the only callers.
The CUDA library never imports, links or executes anything here, and this
package shares no code with it.

What each function follows in the paper (arXiv 2204.05536):
  entry / direct_matvec / direct_rows -- kernels of Sec. 3, Eq. 1byr, Eq. ker;
                                         the explicit product of Sec. 5.1
  Oracle(...)                         -- InitializeHODLR2D, Alg. 1
  Oracle.matvec                       -- MatVec, Alg. 2
  aca                                 -- the ACA step of Alg. 1
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

KINDS = {"imq": 0, "mq": 1, "log": 2, "inv_r": 3, "phi1": 4, "phi2": 5}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so with gcc (plain C11,
    no FMA contraction, single thread)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    fresh = (os.path.exists(_LIB)
             and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if fresh and not force:
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("a", C.c_double), ("diag_mode", C.c_int),
                ("diag_value", C.c_double)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        K = C.POINTER(_Kernel)
        i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
        sig = {
            "orc_entry": (dbl, [K, _dp, i64, i64]),
            "orc_direct_matvec": (None, [i64, _dp, K, _dp, _dp, C.c_int]),
            "orc_direct_rows": (None, [i64, _dp, K, _dp, C.c_int, i64, _lp, _dp]),
            "orc_build": (C.c_int, [i64, _dp, K, C.c_int, dbl, C.c_void_p, C.c_int,
                                    C.c_int, C.POINTER(C.c_void_p)]),
            "orc_free": (None, [C.c_void_p]),
            "orc_matvec": (None, [C.c_void_p, _dp, _dp, C.c_int]),
            "orc_matvec_far_levels": (None, [C.c_void_p, _dp, _dp, C.c_int, C.c_int, C.c_int]),
            "orc_info": (None, [C.c_void_p, C.POINTER(C.c_int), _dp, C.POINTER(i64),
                                C.POINTER(i64)]),
            "orc_box_counts": (None, [C.c_void_p, C.c_int, _lp]),
            "orc_box_points": (i64, [C.c_void_p, C.c_int, i64, _lp]),
            "orc_paper_index": (i64, [C.c_int, i32, i32]),
            "orc_paper_coords": (None, [C.c_int, i64, C.POINTER(i32), C.POINTER(i32)]),
            "orc_edge_list": (C.c_int, [C.c_void_p, C.c_int, i64, _lp, C.c_int]),
            "orc_interaction_list": (C.c_int, [C.c_void_p, C.c_int, i64, _lp, C.c_int]),
            "orc_level_counts": (None, [C.c_void_p, C.c_int, _lp]),
            "orc_coverage": (None, [C.c_void_p, _ip]),
            "orc_pair_info": (None, [C.c_void_p, i64, _ip, C.POINTER(i64), C.POINTER(i64)]),
            "orc_pair_factors": (None, [C.c_void_p, i64, _dp, _dp]),
            "orc_export_factors": (None, [C.c_void_p, _ip, _lp, C.c_void_p]),
            "orc_aca": (C.c_int, [K, _dp, i64, _lp, i64, _lp, dbl, _dp, _dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def kernel(kind: str, a: float = 0.0, diag: float | None = None) -> _Kernel:
    """Kernel descriptor.  diag=None keeps phi(0) (0 for log / 1/r)."""
    return _Kernel(KINDS[kind], float(a), 0 if diag is None else 1,
                   0.0 if diag is None else float(diag))


def _pts(points) -> np.ndarray:
    p = np.ascontiguousarray(points, dtype=np.float64)
    if p.ndim != 2 or p.shape[1] != 2:
        raise ValueError("points must be N x 2")
    return p


def _cols(x, n) -> tuple[np.ndarray, int]:
    """x as n x nrhs column-major (Fortran) data, returned flat."""
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    if x.shape[0] != n:
        raise ValueError("x has %d rows, expected %d" % (x.shape[0], n))
    return np.ascontiguousarray(x.T).reshape(-1), x.shape[1]


def _uncols(flat, n, nrhs, squeeze):
    y = flat.reshape(nrhs, n).T.copy()
    return y[:, 0] if squeeze else y


def entry(points, k: _Kernel, i: int, j: int) -> float:
    return _load().orc_entry(C.byref(k), _pts(points), int(i), int(j))


def dense_matrix(points, k: _Kernel) -> np.ndarray:
    """The full matrix A (for tiny N only)."""
    p = _pts(points)
    n = p.shape[0]
    lib = _load()
    A = np.empty((n, n))
    for i in range(n):
        for j in range(n):
            A[i, j] = lib.orc_entry(C.byref(k), p, i, j)
    return A


def direct_matvec(points, k: _Kernel, x) -> np.ndarray:
    p = _pts(points)
    n = p.shape[0]
    xf, nrhs = _cols(x, n)
    y = np.empty(n * nrhs)
    _load().orc_direct_matvec(n, p, C.byref(k), xf, y, nrhs)
    return _uncols(y, n, nrhs, np.asarray(x).ndim == 1)


def direct_rows(points, k: _Kernel, x, rows) -> np.ndarray:
    p = _pts(points)
    n = p.shape[0]
    xf, nrhs = _cols(x, n)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty(len(rows) * nrhs)
    _load().orc_direct_rows(n, p, C.byref(k), xf, nrhs, len(rows), rows, y)
    return _uncols(y, len(rows), nrhs, np.asarray(x).ndim == 1)


def aca(points, k: _Kernel, I, J, eps: float):
    """ACA of A(I, J); returns (U, V) with A(I,J) ~ U V^T."""
    p = _pts(points)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    kmax = min(len(I), len(J))
    U = np.zeros(len(I) * max(kmax, 1))
    V = np.zeros(len(J) * max(kmax, 1))
    r = _load().orc_aca(C.byref(k), p, len(I), I, len(J), J, float(eps), U, V)
    if r < 0:
        raise MemoryError("orc_aca failed")
    U = U[: len(I) * r].reshape(r, len(I)).T
    V = V[: len(J) * r].reshape(r, len(J)).T
    return U, V


def paper_index(level: int, ix: int, iy: int) -> int:
    return int(_load().orc_paper_index(level, ix, iy))


def paper_coords(level: int, b: int) -> tuple[int, int]:
    ix, iy = C.c_int32(), C.c_int32()
    _load().orc_paper_coords(level, b, C.byref(ix), C.byref(iy))
    return ix.value, iy.value


class Oracle:
    """InitializeHODLR2D (Alg. 1) on the CPU, then MatVec (Alg. 2)."""

    def __init__(self, points, k: _Kernel, leaf_size: int, eps: float, root=None,
                 levels: int = -1, compress: bool = True):
        lib = _load()
        self._lib = lib
        self.points = _pts(points)
        self.n = self.points.shape[0]
        self.kernel = k
        h = C.c_void_p()
        rootarr = None
        rootp = None
        if root is not None:
            rootarr = (C.c_double * 3)(*[float(v) for v in root])
            rootp = C.cast(rootarr, C.c_void_p)
        rc = lib.orc_build(self.n, self.points, C.byref(k), int(leaf_size), float(eps),
                           rootp, int(levels), int(bool(compress)), C.byref(h))
        if rc != 0:
            raise RuntimeError("orc_build failed with code %d" % rc)
        self._h = h
        kap = C.c_int()
        r3 = np.zeros(3)
        npairs, nvals = C.c_int64(), C.c_int64()
        lib.orc_info(h, C.byref(kap), r3, C.byref(npairs), C.byref(nvals))
        self.kappa = kap.value
        self.root = tuple(r3)
        self.npairs = npairs.value
        self.nvalues = nvals.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.orc_free(h)
            self._h = None

    def matvec(self, x) -> np.ndarray:
        xf, nrhs = _cols(x, self.n)
        y = np.empty(self.n * nrhs)
        self._lib.orc_matvec(self._h, xf, y, nrhs)
        return _uncols(y, self.n, nrhs, np.asarray(x).ndim == 1)

    def matvec_far_levels(self, x, l0: int, l1: int) -> np.ndarray:
        xf, nrhs = _cols(x, self.n)
        y = np.zeros(self.n * nrhs)
        self._lib.orc_matvec_far_levels(self._h, xf, y, nrhs, int(l0), int(l1))
        return _uncols(y, self.n, nrhs, np.asarray(x).ndim == 1)

    def box_counts(self, level: int) -> np.ndarray:
        out = np.zeros(4 ** level, dtype=np.int64)
        self._lib.orc_box_counts(self._h, level, out)
        return out

    def box_points(self, level: int, b: int) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        c = self._lib.orc_box_points(self._h, level, b, out)
        return out[:c].copy()

    def edge_list(self, level: int, b: int) -> list[int]:
        out = np.zeros(8, dtype=np.int64)
        c = self._lib.orc_edge_list(self._h, level, b, out, 8)
        return [int(v) for v in out[:c]]

    def interaction_list(self, level: int, b: int) -> list[int]:
        out = np.zeros(32, dtype=np.int64)
        c = self._lib.orc_interaction_list(self._h, level, b, out, 32)
        return [int(v) for v in out[:c]]

    def level_counts(self, level: int) -> dict:
        out = np.zeros(4, dtype=np.int64)
        self._lib.orc_level_counts(self._h, level, out)
        return {"self": int(out[0]), "edge": int(out[1]), "vertex": int(out[2]),
                "far": int(out[3])}

    def coverage(self) -> np.ndarray:
        mark = np.zeros(self.n * self.n, dtype=np.int32)
        self._lib.orc_coverage(self._h, mark)
        return mark.reshape(self.n, self.n)

    def pair(self, p: int):
        """Stored pair p: (info dict, U, V) with rows in ascending point index."""
        info = np.zeros(6, dtype=np.int32)
        nx, ny = C.c_int64(), C.c_int64()
        self._lib.orc_pair_info(self._h, p, info, C.byref(nx), C.byref(ny))
        k = int(info[5])
        U = np.zeros(max(nx.value * k, 1))
        V = np.zeros(max(ny.value * k, 1))
        self._lib.orc_pair_factors(self._h, p, U, V)
        U = U[: nx.value * k].reshape(k, nx.value).T
        V = V[: ny.value * k].reshape(k, ny.value).T
        d = {"level": int(info[0]), "x": (int(info[1]), int(info[2])),
             "y": (int(info[3]), int(info[4])), "rank": k, "nx": nx.value, "ny": ny.value}
        return d, U, V

    def pairs(self):
        for p in range(self.npairs):
            yield self.pair(p)

    def export_factors(self):
        """All stored pairs in the flat layout the CUDA library's import call
        reads: info (npairs x 6 int32: level, ixX, iyX, ixY, iyY, rank),
        offsets (npairs+1 int64) and values (for each pair U then V, each
        column-major, rows in ascending original point index)."""
        info = np.zeros((max(self.npairs, 1), 6), dtype=np.int32)
        offs = np.zeros(self.npairs + 1, dtype=np.int64)
        self._lib.orc_export_factors(self._h, info, offs, None)
        vals = np.zeros(max(int(offs[-1]), 1))
        self._lib.orc_export_factors(self._h, info, offs, C.c_void_p(vals.ctypes.data))
        return info[: self.npairs], offs, vals[: int(offs[-1])]
