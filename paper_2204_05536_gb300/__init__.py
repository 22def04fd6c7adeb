"""GB300 (sm_103a) HODLR2D: quadtree, admissibility lists, batched ACA and
the O(p N log N) matrix-vector product of "HODLR2D: A new class of
hierarchical matrices" (arXiv 2204.05536), behind the C ABI of
``include/hodlr2d.h``.

This module marshals arguments only; every step runs in the CUDA library.
Device buffers are torch CUDA tensors (float64); host arrays may be numpy.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import KINDS, MODES, HodlrError, check, load

__all__ = ["HODLR2D", "RankModel", "Batch", "autotune_leaf", "kernel", "load", "HodlrError",
           "KINDS", "MODES"]


def kernel(kind: str, a: float = 0.0, diag: float | None = None) -> _lib.Kernel:
    """Kernel descriptor: kind in KINDS; diag=None keeps phi(0) (0 for log, 1/r)."""
    return _lib.Kernel(KINDS[kind], float(a), 0 if diag is None else 1,
                       0.0 if diag is None else float(diag))


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keepalive) of a contiguous float64 torch tensor or numpy array."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float64:
            raise TypeError("expected a float64 tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return C.c_void_p(x.data_ptr()), x
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 array")
    return C.c_void_p(a.ctypes.data), a


def _colmajor(x, n):
    """x (n,) or (n, nrhs) -> column-major buffer of the same kind, nrhs."""
    if _is_torch(x):
        if x.dim() == 1:
            return x.contiguous(), 1
        if x.shape[0] != n:
            raise ValueError("x must have n rows")
        return x.t().contiguous(), x.shape[1]
    a = np.asarray(x, dtype=np.float64)
    if a.ndim == 1:
        return np.ascontiguousarray(a), 1
    if a.shape[0] != n:
        raise ValueError("x must have n rows")
    return np.ascontiguousarray(a.T), a.shape[1]


class HODLR2D:
    """A built HODLR2D matrix on the current CUDA device (hodlr2d_build_ex)."""

    def __init__(self, points, k: _lib.Kernel, leaf_size: int, eps: float, root=None,
                 levels: int = -1, compress: bool = True, max_rank: int = 256,
                 mode: str = "f64", stream=None, rank_model=None):
        lib = load()
        self._lib = lib
        opts = _lib.Opts()
        lib.hodlr2d_default_opts(C.byref(opts))
        if root is not None:
            for i in range(3):
                opts.root[i] = float(root[i])
        opts.levels = int(levels)
        opts.compress = int(bool(compress))
        opts.max_rank = int(max_rank)
        opts.mode = MODES[mode]
        opts.rank_model = None if rank_model is None else rank_model.handle.value
        if _is_torch(points):
            pts = points.contiguous()
        else:
            pts = np.ascontiguousarray(points, dtype=np.float64)
        if pts.shape[-1] != 2 or len(pts.shape) != 2:
            raise ValueError("points must be N x 2")
        self.n = int(pts.shape[0])
        p, keep = _ptr(pts)
        h = C.c_void_p()
        check(lib.hodlr2d_build_ex(p, self.n, k, int(leaf_size), float(eps), C.byref(opts),
                                   C.byref(h)), "hodlr2d_build_ex")
        self._h = h
        self.kernel = k
        if stream is not None:
            self.set_stream(stream)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hodlr2d_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- products -----------------------------------------------------------
    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (default)."""
        s = 0 if stream is None else getattr(stream, "cuda_stream", stream)
        check(self._lib.hodlr2d_set_stream(self._h, C.c_void_p(int(s))), "hodlr2d_set_stream")

    def prepare(self, mode: str):
        check(self._lib.hodlr2d_prepare(self._h, MODES[mode]), "hodlr2d_prepare")

    def check(self):
        """hodlr2d_check: synchronise; raise if a bounded device wait gave up."""
        check(self._lib.hodlr2d_check(self._h), "hodlr2d_check")

    def release(self, mode: str):
        """Free one mode's factor copy (hodlr2d_release)."""
        check(self._lib.hodlr2d_release(self._h, MODES[mode]), "hodlr2d_release")

    def matvec(self, x, mode: str = "f64", out=None):
        """y = K_hat x for x of shape (n,) or (n, nrhs).  torch CUDA tensors stay
        on the device (asynchronous on the handle's stream); numpy arrays go
        through host staging."""
        xc, nrhs = _colmajor(x, self.n)
        if out is None:
            if _is_torch(xc):
                import torch
                yc = torch.empty_like(xc)
            else:
                yc = np.empty_like(xc)
        else:
            yc = out
        px, kx = _ptr(xc)
        py, ky = _ptr(yc)
        check(self._lib.hodlr2d_matvec_ex(self._h, px, py, nrhs, MODES[mode]),
              "hodlr2d_matvec_ex")
        if out is not None:
            return out
        if nrhs == 1 and (x.dim() == 1 if _is_torch(x) else np.ndim(x) == 1):
            return yc
        return yc.t() if _is_torch(yc) else yc.T

    def gmres(self, b, x0=None, tol: float = 1e-8, restart: int = 50, maxit: int | None = None,
              inner_mode: str = "f64", raise_on_noconv: bool = False):
        """Restarted GMRES for A x = b; returns (x, iters, relres, code)."""
        if _is_torch(b):
            import torch
            x = torch.zeros_like(b) if x0 is None else x0.clone()
        else:
            x = np.zeros_like(np.asarray(b, dtype=np.float64)) if x0 is None else np.array(
                x0, dtype=np.float64)
        if maxit is None:
            maxit = int(min(10 * self.n, 100000))
        pb, kb = _ptr(b)
        px, kx = _ptr(x)
        it = C.c_int()
        rr = C.c_double()
        rc = self._lib.hodlr2d_gmres_ex(self._h, pb, px, float(tol), int(restart), int(maxit),
                                        MODES[inner_mode], C.byref(it), C.byref(rr))
        if rc not in (_lib.OK, _lib.ERR_NOCONV) or (raise_on_noconv and rc != _lib.OK):
            check(rc, "hodlr2d_gmres_ex")
        return x, it.value, rr.value, rc

    # -- introspection --------------------------------------------------------
    def stats(self) -> dict:
        s = _lib.Stats()
        check(self._lib.hodlr2d_get_stats(self._h, C.byref(s)), "hodlr2d_get_stats")
        k = s.kappa
        return {
            "n": s.n, "kappa": k, "root": tuple(s.root), "npairs": s.npairs,
            "pairs_per_level": list(s.pairs_per_level)[: k + 1],
            "values_per_level": list(s.values_per_level)[: k + 1],
            "max_rank_per_level": list(s.max_rank_per_level)[: k + 1],
            "max_rank": s.max_rank, "far_values": s.far_values,
            "near_entries": s.near_entries, "unconverged": s.unconverged,
            "compression_ratio": s.compression_ratio, "build_ms": list(s.build_ms),
            "bytes_per_matvec": dict(zip(MODES, list(s.bytes_per_matvec))),
            "aca_fallbacks": s.aca_fallbacks, "aca_workspace_values": s.aca_workspace_values,
        }

    def pair_features(self):
        """(features npairs x 8 float32, log2(rank + 1) npairs float32) of the
        stored pairs, in pairs() order: training data of the rank predictor."""
        n = C.c_int64()
        check(self._lib.hodlr2d_pair_features(self._h, C.byref(n), None, None),
              "hodlr2d_pair_features")
        f = np.zeros((max(n.value, 1), 8), dtype=np.float32)
        r = np.zeros(max(n.value, 1), dtype=np.float32)
        check(self._lib.hodlr2d_pair_features(self._h, C.byref(n), C.c_void_p(f.ctypes.data),
                                              C.c_void_p(r.ctypes.data)), "hodlr2d_pair_features")
        return f[: n.value], r[: n.value]

    def profile(self, enable: bool):
        check(self._lib.hodlr2d_profile(self._h, int(bool(enable))), "hodlr2d_profile")

    def get_profile(self) -> dict:
        """Per phase: summed device ms, launches, algorithmic bytes and flops."""
        ms = np.zeros(_lib.NPHASE)
        nl = np.zeros(_lib.NPHASE, dtype=np.int64)
        by = np.zeros(_lib.NPHASE, dtype=np.int64)
        check(self._lib.hodlr2d_get_profile(self._h, C.c_void_p(ms.ctypes.data),
                                            C.c_void_p(nl.ctypes.data),
                                            C.c_void_p(by.ctypes.data)), "hodlr2d_get_profile")
        fl = np.zeros(_lib.NPHASE, dtype=np.int64)
        check(self._lib.hodlr2d_get_profile_flops(self._h, C.c_void_p(fl.ctypes.data)),
              "hodlr2d_get_profile_flops")
        return {name: {"ms": float(ms[i]), "launches": int(nl[i]), "bytes": int(by[i]),
                       "flops": int(fl[i])}
                for i, name in enumerate(_lib.PHASES)}

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        check(self._lib.hodlr2d_get_perm(self._h, C.c_void_p(out.ctypes.data)), "hodlr2d_get_perm")
        return out

    def pairs(self) -> np.ndarray:
        """(npairs, 6) int32: level, ixX, iyX, ixY, iyY, rank."""
        n = C.c_int64()
        check(self._lib.hodlr2d_get_pairs(self._h, C.byref(n), None), "hodlr2d_get_pairs")
        info = np.zeros((max(n.value, 1), 6), dtype=np.int32)
        check(self._lib.hodlr2d_get_pairs(self._h, C.byref(n), C.c_void_p(info.ctypes.data)),
              "hodlr2d_get_pairs")
        return info[: n.value]

    def import_factors(self, info, offsets, values):
        info = np.ascontiguousarray(info, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        values = np.ascontiguousarray(values, dtype=np.float64)
        check(self._lib.hodlr2d_import_factors(
            self._h, int(info.shape[0]), C.c_void_p(info.ctypes.data),
            C.c_void_p(offsets.ctypes.data), C.c_void_p(values.ctypes.data)),
            "hodlr2d_import_factors")

    def export_factors(self):
        npairs, nvals = C.c_int64(), C.c_int64()
        check(self._lib.hodlr2d_export_factors(self._h, C.byref(npairs), C.byref(nvals), None,
                                               None, None), "hodlr2d_export_factors")
        info = np.zeros((max(npairs.value, 1), 6), dtype=np.int32)
        offs = np.zeros(npairs.value + 1, dtype=np.int64)
        vals = np.zeros(max(nvals.value, 1))
        check(self._lib.hodlr2d_export_factors(
            self._h, C.byref(npairs), C.byref(nvals), C.c_void_p(info.ctypes.data),
            C.c_void_p(offs.ctypes.data), C.c_void_p(vals.ctypes.data)), "hodlr2d_export_factors")
        return info[: npairs.value], offs, vals[: nvals.value]


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, C.c_void_p(a.ctypes.data)


class RankModel:
    """Rank predictor network (hodlr2d_rank_model_*), trained on the GPU."""

    def __init__(self, hidden: int = 64, params=None):
        self._lib = load()
        h = C.c_void_p()
        keep = None
        ptr = None
        if params is not None:
            keep, ptr = _f32(params)
        check(self._lib.hodlr2d_rank_model_create(int(hidden), ptr, C.byref(h)),
              "hodlr2d_rank_model_create")
        self._h = h
        self.hidden = hidden

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hodlr2d_rank_model_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        n = C.c_int64()
        check(self._lib.hodlr2d_rank_model_params(self._h, None, C.byref(n)), "params")
        out = np.zeros(n.value, dtype=np.float32)
        check(self._lib.hodlr2d_rank_model_params(self._h, C.c_void_p(out.ctypes.data),
                                                  C.byref(n)), "params")
        return out

    def loss_grad(self, feats, targets):
        f, fp = _f32(feats)
        t, tp = _f32(targets)
        n = C.c_int64()
        self._lib.hodlr2d_rank_model_params(self._h, None, C.byref(n))
        g = np.zeros(n.value, dtype=np.float32)
        loss = C.c_float()
        check(self._lib.hodlr2d_rank_model_loss_grad(self._h, fp, tp, len(t), C.byref(loss),
                                                     C.c_void_p(g.ctypes.data)), "loss_grad")
        return loss.value, g

    def train(self, feats, targets, batch: int = 4096, epochs: int = 10, lr: float = 1e-3):
        f, fp = _f32(feats)
        t, tp = _f32(targets)
        loss = C.c_float()
        check(self._lib.hodlr2d_rank_model_train(self._h, fp, tp, len(t), int(batch),
                                                 int(epochs), float(lr), C.byref(loss)), "train")
        return loss.value

    def predict(self, feats) -> np.ndarray:
        f, fp = _f32(feats)
        out = np.zeros(len(f), dtype=np.float32)
        check(self._lib.hodlr2d_rank_model_predict(self._h, fp, len(f),
                                                   C.c_void_p(out.ctypes.data)), "predict")
        return out


BATCH_FORMS = {"auto": 0, "graph": 1, "persistent": 2}


class Batch:
    """Independent HODLR2D matrices multiplied as one unit (hodlr2d_batch_*):
    one CUDA graph launch, or one persistent cooperative kernel over all sets
    (form "auto", "graph" or "persistent").  Keeps the handles alive."""

    def __init__(self, matrices, stream=None, form: str = "auto"):
        self._lib = load()
        self.mats = list(matrices)
        arr = (C.c_void_p * len(self.mats))(*[m.handle.value for m in self.mats])
        h = C.c_void_p()
        check(self._lib.hodlr2d_batch_create(arr, len(self.mats), C.byref(h)),
              "hodlr2d_batch_create")
        self._h = h
        if stream is not None:
            s = getattr(stream, "cuda_stream", stream)
            check(self._lib.hodlr2d_batch_set_stream(self._h, C.c_void_p(int(s))),
                  "hodlr2d_batch_set_stream")
        self.set_form(form)

    def set_form(self, form: str):
        check(self._lib.hodlr2d_batch_set_form(self._h, BATCH_FORMS[form]),
              "hodlr2d_batch_set_form")

    def set_wait_limit(self, polls: int):
        """Polls of a grid-barrier wait (persistent form) before it gives up."""
        check(self._lib.hodlr2d_batch_set_wait_limit(self._h, int(polls)),
              "hodlr2d_batch_set_wait_limit")

    def check(self):
        """hodlr2d_batch_check: synchronise; raise if a barrier wait gave up."""
        check(self._lib.hodlr2d_batch_check(self._h), "hodlr2d_batch_check")

    @property
    def last_form(self):
        f = self._lib.hodlr2d_batch_last_form(self._h)
        return {1: "graph", 2: "persistent"}.get(f)

    @property
    def persistent_recorded(self):
        """True if the persistent launch is replayed from a CUDA graph, False if
        it is launched directly, None before the first persistent product."""
        r = self._lib.hodlr2d_batch_persistent_recorded(self._h)
        return None if r < 0 else bool(r)

    def _args(self, xs, ys):
        n = len(self.mats)
        xa = (C.c_void_p * n)(*[x.data_ptr() for x in xs])
        ya = (C.c_void_p * n)(*[y.data_ptr() for y in ys])
        nr = (C.c_int * n)(*[1 if x.dim() == 1 else x.shape[0] for x in xs])
        return xa, ya, nr

    def matvec(self, xs, ys, mode: str = "f64"):
        """xs[i], ys[i]: float64 CUDA tensors holding n_i x nrhs_i column-major
        data (shape (nrhs_i, n_i) contiguous, or (n_i,))."""
        xa, ya, nr = self._args(xs, ys)
        check(self._lib.hodlr2d_batch_matvec(self._h, xa, ya, nr, MODES[mode]),
              "hodlr2d_batch_matvec")

    def set_shapes(self, pair_rows: int, warp_rows: int):
        """Persistent form: levels of boxes <= pair_rows points run as pairs
        (one per warp up to warp_rows points), coarser ones in two passes."""
        check(self._lib.hodlr2d_batch_set_shapes(self._h, int(pair_rows), int(warp_rows)),
              "hodlr2d_batch_set_shapes")

    def shapes(self):
        a, b = C.c_int(), C.c_int()
        check(self._lib.hodlr2d_batch_get_shapes(self._h, C.byref(a), C.byref(b)),
              "hodlr2d_batch_get_shapes")
        return a.value, b.value

    def autotune(self, xs, ys, mode: str = "f32", reps: int = 3):
        """hodlr2d_batch_autotune: time the persistent form's shape candidates
        on these inputs, keep the fastest; returns ((pair_rows, warp_rows),
        ms per product)."""
        xa, ya, nr = self._args(xs, ys)
        ms = C.c_double()
        check(self._lib.hodlr2d_batch_autotune(self._h, xa, ya, nr, MODES[mode], int(reps),
                                               C.byref(ms)), "hodlr2d_batch_autotune")
        return self.shapes(), ms.value

    def set_blocks_per_sm(self, blocks: int):
        """Resident blocks per SM of the persistent kernel (2, 3 or 4)."""
        check(self._lib.hodlr2d_batch_set_blocks_per_sm(self._h, int(blocks)),
              "hodlr2d_batch_set_blocks_per_sm")

    def set_placement(self, place: int):
        """Persistent form: bit 0 runs the near field beside the expansions,
        bit 1 the one-warp pairs beside the chunk sums."""
        check(self._lib.hodlr2d_batch_set_placement(self._h, int(place)),
              "hodlr2d_batch_set_placement")

    def tune_table(self):
        """[(pair_rows, warp_rows, blocks per SM, placement, ms per product)]
        of the last autotune."""
        cnt = C.c_int(0)
        check(self._lib.hodlr2d_batch_tune_table(self._h, C.byref(cnt), None, None, None, None,
                                                 None), "hodlr2d_batch_tune_table")
        n = cnt.value
        arr = [(C.c_int * n)() for _ in range(4)]
        ms = (C.c_double * n)()
        check(self._lib.hodlr2d_batch_tune_table(self._h, C.byref(cnt), *arr, ms),
              "hodlr2d_batch_tune_table")
        return [(arr[0][i], arr[1][i], arr[2][i], arr[3][i], ms[i]) for i in range(n)]

    def phase_ms(self):
        """Milliseconds of the five phases of the last persistent product."""
        out = (C.c_double * 5)()
        check(self._lib.hodlr2d_batch_phase_ms(self._h, out), "hodlr2d_batch_phase_ms")
        return list(out)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.hodlr2d_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_leaf(points, k, eps, candidates=(32, 64, 128), nrhs: int = 1, mode: str = "f64",
                  reps: int = 5, root=None):
    """Leaf size (N_max of Alg. 1) with the fastest product for this point set:
    builds the matrix for every candidate, times reps products with CUDA
    events, and returns (best leaf, {leaf: ms})."""
    import torch
    times = {}
    n = len(points)
    x = torch.ones((nrhs, n), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for leaf in candidates:
        g = HODLR2D(points, k, leaf, eps, root=root)
        if mode != "f64":
            g.prepare(mode)
        g.set_stream(torch.cuda.current_stream())
        g.matvec(x.t() if nrhs > 1 else x[0], mode=mode)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.matvec(x.t() if nrhs > 1 else x[0], mode=mode)
        e1.record()
        torch.cuda.synchronize()
        times[leaf] = e0.elapsed_time(e1) / reps
        g.close()
    best = min(times, key=times.get)
    return best, times
