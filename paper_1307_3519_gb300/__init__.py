"""GB300 (sm_103a) Kruskal-Wallis SNP x trait scan: Python binding of libkrux.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/krux.h``); this module only marshals torch tensors into raw pointers
and back.  There is no CPU fallback: if the library is missing the import
fails.  Function names follow the C ABI (``krux_rank``, ``krux_scan``,
``krux_scan_plain``, ``krux_permute``, ``krux_scan_grouped``); the ``Krux``
class wraps them with allocation of outputs, and ``Krux.krux_scan_host`` is the
end-to-end call from host arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkrux.so")

KRUX_OK, KRUX_EINVAL, KRUX_ENOMEM, KRUX_ECUDA, KRUX_EOVERFLOW, KRUX_ETIMEOUT, KRUX_EUNSUPPORTED = range(7)
KRUX_FLAG_MULTIALLELIC = 1  # genotype codes 0..4
STATUS_NAMES = ["KRUX_OK", "KRUX_EINVAL", "KRUX_ENOMEM", "KRUX_ECUDA", "KRUX_EOVERFLOW",
                "KRUX_ETIMEOUT", "KRUX_EUNSUPPORTED"]

# Every entry point declared in include/krux.h.
EXPORTS = ["krux_create", "krux_destroy", "krux_status_string", "krux_last_error", "krux_rank",
           "krux_rankset_free", "krux_rankset_export", "krux_scan", "krux_scan_host", "krux_scan_plain",
           "krux_permute", "krux_scan_grouped", "krux_make_perms", "krux_set_profiling",
           "krux_get_profile", "krux_set_wait_limit", "krux_set_tuning", "krux_scan_noalloc", "krux_debug_plan",
           "krux_autotune", "krux_graph_scan", "krux_graph_permute", "krux_graph_grouped",
           "krux_graph_launch", "krux_graph_wait", "krux_graph_last_error", "krux_graph_destroy",
           "krux_scan_cis", "krux_scan_parametric", "krux_debug_tail"]


class KruxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("pthresh", ctypes.c_double), ("hit_capacity", ctypes.c_int64),
                ("snp_begin", ctypes.c_int64), ("snp_end", ctypes.c_int64),
                ("dense_H", ctypes.c_void_p), ("dense_p", ctypes.c_void_p),
                ("recheck_margin", ctypes.c_double), ("flags", ctypes.c_int32),
                ("reserved_", ctypes.c_int32)]


class Profile(ctypes.Structure):
    _fields_ = [("ms_rank", ctypes.c_float), ("ms_pack", ctypes.c_float),
                ("ms_scan", ctypes.c_float), ("ms_finalize", ctypes.c_float),
                ("ms_gemm", ctypes.c_float), ("launches", ctypes.c_int32),
                ("scan_grid", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("scan_form", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class Cohort(ctypes.Structure):
    _fields_ = [("rs", ctypes.c_void_p), ("geno", ctypes.c_void_p), ("S", ctypes.c_int64),
                ("ldg", ctypes.c_int64), ("hits", ctypes.c_void_p), ("hit_H", ctypes.c_void_p),
                ("hit_p", ctypes.c_void_p), ("hit_capacity", ctypes.c_int64),
                ("n_hits", ctypes.c_int64)]


_lib = None


def load_library(path=LIB_PATH):
    """Loads libkrux.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libkrux.so not built at {path}; run paper_1307_3519_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "krux_create": ([ctypes.POINTER(P), I], I),
        "krux_destroy": ([P], None),
        "krux_status_string": ([I], ctypes.c_char_p),
        "krux_last_error": ([P], ctypes.c_char_p),
        "krux_rank": ([P, P, I, I, I64, ctypes.POINTER(P), P], I),
        "krux_rankset_free": ([P, P], None),
        "krux_rankset_export": ([P, P, P, P, P, P], I),
        "krux_scan": ([P, P, P, I64, I64, ctypes.POINTER(Opts), P, P, P, ctypes.POINTER(I64), P], I),
        "krux_scan_plain": ([P, P, P, I64, I64, ctypes.POINTER(Opts), P, P, P, ctypes.POINTER(I64), P], I),
        "krux_scan_host": ([P, P, I, I, I64, P, I64, I64, ctypes.POINTER(Opts), P, P, P,
                            ctypes.POINTER(I64), P], I),
        "krux_permute": ([P, P, P, I64, I64, P, I, ctypes.POINTER(Opts), P, P, P, P,
                          ctypes.POINTER(I64), P, I, D, P], I),
        "krux_scan_grouped": ([P, ctypes.POINTER(Cohort), I, ctypes.POINTER(Opts), P], I),
        "krux_make_perms": ([ctypes.c_uint64, I, I, P], I),
        "krux_set_profiling": ([P, I], I),
        "krux_get_profile": ([P, ctypes.POINTER(Profile)], I),
        "krux_set_wait_limit": ([P, ctypes.c_longlong], I),
        "krux_set_tuning": ([P, I, I, I, I], I),
        "krux_debug_plan": ([I, I, I, I, I, I, P], I),
        "krux_scan_noalloc": ([P, I, I, I64, P, I64, I64, D, P, P, P, I64, ctypes.POINTER(I64), P], I),
        "krux_autotune": ([P, P, P, I64, I64, D, P, P], I),
        "krux_scan_parametric": ([P, P, I, I, I64, P, I64, I64, I, ctypes.POINTER(Opts), P, P, P,
                                  ctypes.POINTER(I64), P], I),
        "krux_debug_tail": ([I, D, D, D], D),
        "krux_scan_cis": ([P, P, P, I64, I64, P, P, I64, ctypes.POINTER(Opts), P, P, P,
                           ctypes.POINTER(I64), P], I),
        "krux_graph_scan": ([P, P, P, I64, I64, ctypes.POINTER(Opts), P, P, P, ctypes.POINTER(P)], I),
        "krux_graph_permute": ([P, P, P, I64, I64, P, I, ctypes.POINTER(Opts), P, P, P, P, P, I, D,
                                ctypes.POINTER(P)], I),
        "krux_graph_grouped": ([P, ctypes.POINTER(Cohort), I, ctypes.POINTER(Opts), ctypes.POINTER(P)], I),
        "krux_graph_launch": ([P, P], I),
        "krux_graph_wait": ([P, ctypes.POINTER(I64), I], I),
        "krux_graph_last_error": ([P], ctypes.c_char_p),
        "krux_graph_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _ld(t):
    """Row stride (elements) of a 2-D tensor as a leading dimension: a one-row
    matrix may carry any stride for its single row (numpy gives 0 to an inserted
    axis), so its leading dimension is its row length."""
    return t.stride(0) if t.shape[0] > 1 else t.shape[1]


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def krux_scan_noalloc(expr, geno, pthresh, hits, hit_H, hit_p, stream=None):
    """Scan without any device allocation by the library (see include/krux.h):
    expr cuda float32 [T, N], geno cuda int8 [S, N], outputs preallocated by the
    caller (hits int32 [cap, 4], hit_H / hit_p float64 [cap]).  Returns
    (status, exact hit count)."""
    import torch
    for name, t, dt in (("expr", expr, torch.float32), ("geno", geno, torch.int8),
                        ("hits", hits, torch.int32), ("hit_H", hit_H, torch.float64),
                        ("hit_p", hit_p, torch.float64)):
        if t.dtype != dt or not t.is_cuda:
            raise ValueError(f"krux_scan_noalloc: {name} must be a CUDA {dt} tensor")
    if expr.dim() != 2 or geno.dim() != 2 or expr.stride(1) != 1 or geno.stride(1) != 1:
        raise ValueError("krux_scan_noalloc: expr and geno must be 2-D with contiguous rows")
    if hits.dim() != 2 or hits.shape[1] != 4 or not hits.is_contiguous():
        raise ValueError("krux_scan_noalloc: hits must be a contiguous int32 [capacity, 4] tensor")
    if hit_H.numel() < hits.shape[0] or hit_p.numel() < hits.shape[0] or \
            not hit_H.is_contiguous() or not hit_p.is_contiguous():
        raise ValueError("krux_scan_noalloc: hit_H and hit_p need hits.shape[0] contiguous entries")
    if len({expr.device, geno.device, hits.device, hit_H.device, hit_p.device}) != 1:
        raise ValueError("krux_scan_noalloc: all tensors must be on one device")
    n = ctypes.c_int64()
    st = load_library().krux_scan_noalloc(
        ctypes.c_void_p(expr.data_ptr()), expr.shape[0], expr.shape[1], _ld(expr),
        ctypes.c_void_p(geno.data_ptr()), geno.shape[0], _ld(geno), float(pthresh),
        ctypes.c_void_p(hits.data_ptr()), ctypes.c_void_p(hit_H.data_ptr()),
        ctypes.c_void_p(hit_p.data_ptr()), hits.shape[0], ctypes.byref(n), _stream(stream))
    return st, n.value


def krux_debug_plan(N, with_nan=False, layout=-1, nc=0, nA=0, ka=0):
    """(status, dict) of the pipeline shape a scan of N samples would use."""
    out = np.zeros(7, dtype=np.int32)
    st = load_library().krux_debug_plan(N, int(with_nan), layout, nc, nA, ka,
                                        out.ctypes.data_as(ctypes.c_void_p))
    keys = ["ka", "nA", "b_region", "nc", "nkb", "b_stride", "smem"]
    return st, dict(zip(keys, out.tolist()))


def krux_make_perms(seed, P, N):
    """Host int32 [P, N] permutations (Fisher-Yates driven by SplitMix64)."""
    out = np.empty((P, N), dtype=np.int32)
    st = load_library().krux_make_perms(seed, P, N, out.ctypes.data_as(ctypes.c_void_p))
    if st != KRUX_OK:
        raise KruxError(st, "krux_make_perms")
    return out


class RankSet:
    """A rank set owned by its context (centred ranks, tie sums, K on device)."""

    def __init__(self, ctx, handle, T, N):
        self.ctx, self.handle, self.T, self.N = ctx, handle, T, N

    def free(self):
        if self.handle:
            load_library().krux_rankset_free(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            if self.ctx.handle:
                self.free()
        except Exception:
            pass


class Krux:
    """A library context on one CUDA device."""

    def __init__(self, device=0):
        import torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        torch.cuda.init()
        h = ctypes.c_void_p()
        st = self.lib.krux_create(ctypes.byref(h), device)
        if st != KRUX_OK:
            raise KruxError(st, "krux_create failed (device must be sm_103)")
        self.handle = h

    def close(self):
        if self.handle:
            self.lib.krux_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st not in (KRUX_OK, KRUX_EOVERFLOW):
            msg = self.lib.krux_last_error(self.handle)
            raise KruxError(st, f"{what}: {msg.decode() if msg else ''}")
        return st

    # ---- thin wrappers --------------------------------------------------------
    def set_profiling(self, on=True):
        self._check(self.lib.krux_set_profiling(self.handle, 1 if on else 0), "set_profiling")

    def profile(self):
        p = Profile()
        self._check(self.lib.krux_get_profile(self.handle, ctypes.byref(p)), "get_profile")
        return {f: getattr(p, f) for f, _ in Profile._fields_}

    def set_tuning(self, layout=-1, nc=0, nA=0, ka=0):
        """Tile shape: layout (0: 64-sample atoms, 1: 16-sample atoms, -1 auto), nc
        resident SNP chunks, nA rank-tile stages, ka samples per rank stage (0 =
        whole K); nc = nA = 0 = automatic."""
        self._check(self.lib.krux_set_tuning(self.handle, layout, nc, nA, ka), "set_tuning")

    def set_wait_limit(self, cycles):
        self._check(self.lib.krux_set_wait_limit(self.handle, int(cycles)), "set_wait_limit")

    def krux_rank(self, expr, stream=None):
        """expr: cuda float32 [T, N] (row stride may exceed N). Returns a RankSet."""
        import torch
        assert expr.is_cuda and expr.dtype == torch.float32 and expr.dim() == 2 and expr.stride(1) == 1
        T, N = expr.shape
        h = ctypes.c_void_p()
        st = self.lib.krux_rank(self.handle, _ptr(expr), T, N, _ld(expr), ctypes.byref(h),
                                _stream(stream))
        self._check(st, "krux_rank")
        return RankSet(self, h, T, N)

    def export(self, rs, stream=None):
        """(centred int16 [T,N], tie int64 [T], K int32 [T]) as cuda tensors."""
        import torch
        c = torch.empty((rs.T, rs.N), dtype=torch.int16, device=self.device)
        tie = torch.empty(rs.T, dtype=torch.int64, device=self.device)
        K = torch.empty(rs.T, dtype=torch.int32, device=self.device)
        self._check(self.lib.krux_rankset_export(self.handle, rs.handle, _ptr(c), _ptr(tie), _ptr(K),
                                                 _stream(stream)), "krux_rankset_export")
        return c, tie, K

    def _opts(self, pthresh, capacity, snp_begin=0, snp_end=0, dense=None, margin=0.0, flags=0):
        o = Opts()
        o.pthresh = pthresh
        o.hit_capacity = capacity
        o.snp_begin = snp_begin
        o.snp_end = snp_end
        o.dense_H = dense[0].data_ptr() if dense is not None else None
        o.dense_p = dense[1].data_ptr() if dense is not None else None
        o.recheck_margin = margin
        o.flags = flags
        return o

    def _scan(self, fn, rs, geno, pthresh, capacity, snp_begin, snp_end, dense, margin, stream,
              flags=0):
        import torch
        assert geno.is_cuda and geno.dtype == torch.int8 and geno.dim() == 2 and geno.stride(1) == 1
        S = geno.shape[0]
        e = snp_end if snp_end > 0 else S
        hits = torch.empty((max(capacity, 1), 4), dtype=torch.int32, device=self.device)
        H = torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device)
        P = torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device)
        dn = None
        if dense:
            dn = (torch.empty((rs.T, e - snp_begin), dtype=torch.float64, device=self.device),
                  torch.empty((rs.T, e - snp_begin), dtype=torch.float64, device=self.device))
        o = self._opts(pthresh, capacity, snp_begin, snp_end, dn, margin, flags)
        n = ctypes.c_int64()
        st = fn(self.handle, rs.handle, _ptr(geno), S, _ld(geno), ctypes.byref(o), _ptr(hits),
                _ptr(H), _ptr(P), ctypes.byref(n), _stream(stream))
        st = self._check(st, fn.__name__)
        k = min(n.value, capacity)
        out = dict(n_hits=n.value, overflow=st == KRUX_EOVERFLOW, hits=hits[:k], H=H[:k], p=P[:k])
        if dn is not None:
            out["dense_H"], out["dense_p"] = dn
        return out

    def krux_scan(self, rs, geno, pthresh, capacity, snp_begin=0, snp_end=0, dense=False,
                  margin=0.0, stream=None, multiallelic=False):
        """Fused scan.  Returns dict(n_hits, overflow, hits int32 [k,4] (trait, snp,
        d0, d1), H, p float64 [k], and dense_H / dense_p [T, S] if dense).
        multiallelic: genotype codes 0..4 (KRUX_FLAG_MULTIALLELIC)."""
        return self._scan(self.lib.krux_scan, rs, geno, pthresh, capacity, snp_begin, snp_end,
                          dense, margin, stream, KRUX_FLAG_MULTIALLELIC if multiallelic else 0)

    def krux_scan_cis(self, rs, geno, snp_pos, trait_pos, window, pthresh, capacity, stream=None,
                      multiallelic=False):
        """cis scan: only pairs with |snp_pos - trait_pos| <= window (int64 device
        coordinates, nondecreasing).  Returns the result dict of krux_scan."""
        hits, H, P = self._outputs(capacity)
        o = self._opts(pthresh, capacity, flags=KRUX_FLAG_MULTIALLELIC if multiallelic else 0)
        n = ctypes.c_int64()
        st = self.lib.krux_scan_cis(self.handle, rs.handle, _ptr(geno), geno.shape[0], _ld(geno),
                                    _ptr(snp_pos), _ptr(trait_pos), int(window), ctypes.byref(o),
                                    _ptr(hits), _ptr(H), _ptr(P), ctypes.byref(n), _stream(stream))
        st = self._check(st, "krux_scan_cis")
        k = min(n.value, capacity)
        return dict(n_hits=n.value, overflow=st == KRUX_EOVERFLOW, hits=hits[:k], H=H[:k], p=P[:k])

    def krux_scan_parametric(self, expr, geno, model, pthresh, capacity, stream=None):
        """Parametric comparison statistics (model 'anova' or 'linear') on the same
        tiles; returns dict(n_hits, overflow, hits (d0 = d1 = 0), stat, p)."""
        import torch
        assert expr.is_cuda and expr.dtype == torch.float32 and expr.stride(1) == 1
        m = {"anova": 0, "linear": 1}[model]
        hits, H, P = self._outputs(capacity)
        o = self._opts(pthresh, capacity)
        n = ctypes.c_int64()
        st = self.lib.krux_scan_parametric(self.handle, _ptr(expr), expr.shape[0], expr.shape[1],
                                           _ld(expr), _ptr(geno), geno.shape[0], _ld(geno),
                                           m, ctypes.byref(o), _ptr(hits), _ptr(H), _ptr(P),
                                           ctypes.byref(n), _stream(stream))
        st = self._check(st, "krux_scan_parametric")
        k = min(n.value, capacity)
        return dict(n_hits=n.value, overflow=st == KRUX_EOVERFLOW, hits=hits[:k], stat=H[:k], p=P[:k])

    def krux_scan_plain(self, rs, geno, pthresh, capacity, snp_begin=0, snp_end=0, dense=False,
                        margin=0.0, stream=None):
        """Plain two-pass form (library GEMM, then a separate epilogue)."""
        return self._scan(self.lib.krux_scan_plain, rs, geno, pthresh, capacity, snp_begin,
                          snp_end, dense, margin, stream)

    def krux_permute(self, rs, geno, perms, pthresh, capacity, fdr_bins=0, fdr_bin_width=0.1,
                     stream=None):
        """Permutation null: returns dict(minp float64 [P, T], the unpermuted hits and,
        with fdr_bins > 0, fdr_hist int64 [1 + P, fdr_bins] (row 0 the real data's
        hits, row q the pairs of permutation q with p' < P_c, binned by
        -log10 p in steps of fdr_bin_width from -log10 P_c))."""
        import torch
        S = geno.shape[0]
        P_ = perms.shape[0]
        hist = (torch.empty((1 + P_, fdr_bins), dtype=torch.int64, device=self.device)
                if fdr_bins > 0 else None)
        minp = torch.empty((P_, rs.T), dtype=torch.float64, device=self.device)
        hits = torch.empty((max(capacity, 1), 4), dtype=torch.int32, device=self.device)
        H = torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device)
        Pv = torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device)
        o = self._opts(pthresh, capacity)
        n = ctypes.c_int64()
        st = self.lib.krux_permute(self.handle, rs.handle, _ptr(geno), S, _ld(geno), _ptr(perms),
                                   P_, ctypes.byref(o), _ptr(minp), _ptr(hits), _ptr(H), _ptr(Pv),
                                   ctypes.byref(n), _ptr(hist), fdr_bins, float(fdr_bin_width),
                                   _stream(stream))
        st = self._check(st, "krux_permute")
        k = min(n.value, capacity)
        return dict(minp=minp, n_hits=n.value, overflow=st == KRUX_EOVERFLOW, hits=hits[:k],
                    H=H[:k], p=Pv[:k], fdr_hist=hist)

    def krux_scan_grouped(self, cohorts, pthresh, stream=None, multiallelic=False):
        """cohorts: list of dict(rs, geno, capacity).  Returns a list of result dicts."""
        import torch
        arr = (Cohort * len(cohorts))()
        keep = []
        for i, c in enumerate(cohorts):
            cap = c["capacity"]
            hits = torch.empty((max(cap, 1), 4), dtype=torch.int32, device=self.device)
            H = torch.empty(max(cap, 1), dtype=torch.float64, device=self.device)
            P = torch.empty(max(cap, 1), dtype=torch.float64, device=self.device)
            keep.append((hits, H, P))
            g = c["geno"]
            arr[i].rs = c["rs"].handle
            arr[i].geno = g.data_ptr()
            arr[i].S = g.shape[0]
            arr[i].ldg = _ld(g)
            arr[i].hits = hits.data_ptr()
            arr[i].hit_H = H.data_ptr()
            arr[i].hit_p = P.data_ptr()
            arr[i].hit_capacity = cap
        o = self._opts(pthresh, 0, flags=KRUX_FLAG_MULTIALLELIC if multiallelic else 0)
        st = self.lib.krux_scan_grouped(self.handle, arr, len(cohorts), ctypes.byref(o), _stream(stream))
        self._check(st, "krux_scan_grouped")
        out = []
        for i, c in enumerate(cohorts):
            k = min(arr[i].n_hits, c["capacity"])
            hits, H, P = keep[i]
            out.append(dict(n_hits=arr[i].n_hits, overflow=arr[i].n_hits > c["capacity"],
                            hits=hits[:k], H=H[:k], p=P[:k]))
        return out

    # ---- autotuner and CUDA graphs ---------------------------------------------
    def autotune(self, rs, geno, pthresh, stream=None):
        """Times every launch shape on a sample of geno and keeps the fastest for
        this rank set's width.  Returns (layout, nc, nA, ka) of the winner."""
        shape = (ctypes.c_int32 * 4)()
        st = self.lib.krux_autotune(self.handle, rs.handle, _ptr(geno), geno.shape[0], _ld(geno),
                                    float(pthresh), _stream(stream), shape)
        self._check(st, "krux_autotune")
        return tuple(shape)

    def _outputs(self, capacity):
        import torch
        return (torch.empty((max(capacity, 1), 4), dtype=torch.int32, device=self.device),
                torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device),
                torch.empty(max(capacity, 1), dtype=torch.float64, device=self.device))

    def graph_scan(self, rs, geno, pthresh, capacity, dense=False, multiallelic=False):
        """krux_scan captured as a CUDA graph; returns a Graph (launch / wait)."""
        import torch
        hits, H, P = self._outputs(capacity)
        dn = None
        if dense:
            dn = (torch.empty((rs.T, geno.shape[0]), dtype=torch.float64, device=self.device),
                  torch.empty((rs.T, geno.shape[0]), dtype=torch.float64, device=self.device))
        o = self._opts(pthresh, capacity, dense=dn,
                       flags=KRUX_FLAG_MULTIALLELIC if multiallelic else 0)
        h = ctypes.c_void_p()
        st = self.lib.krux_graph_scan(self.handle, rs.handle, _ptr(geno), geno.shape[0], _ld(geno),
                                      ctypes.byref(o), _ptr(hits), _ptr(H), _ptr(P), ctypes.byref(h))
        self._check(st, "krux_graph_scan")
        g = Graph(self, h, [(hits, H, P, capacity)], keep=(geno, rs))
        if dn is not None:
            g.dense = dn
        return g

    def graph_permute(self, rs, geno, perms, pthresh, capacity, fdr_bins=0, fdr_bin_width=0.1):
        """krux_permute captured as a CUDA graph (minp, fdr_hist and the hits are
        rewritten by every replay)."""
        import torch
        hits, H, P = self._outputs(capacity)
        P_ = perms.shape[0]
        minp = torch.empty((P_, rs.T), dtype=torch.float64, device=self.device)
        hist = (torch.empty((1 + P_, fdr_bins), dtype=torch.int64, device=self.device)
                if fdr_bins > 0 else None)
        o = self._opts(pthresh, capacity)
        h = ctypes.c_void_p()
        st = self.lib.krux_graph_permute(self.handle, rs.handle, _ptr(geno), geno.shape[0],
                                         _ld(geno), _ptr(perms), P_, ctypes.byref(o), _ptr(minp),
                                         _ptr(hits), _ptr(H), _ptr(P), _ptr(hist), fdr_bins,
                                         float(fdr_bin_width), ctypes.byref(h))
        self._check(st, "krux_graph_permute")
        g = Graph(self, h, [(hits, H, P, capacity)], keep=(geno, perms, rs))
        g.minp, g.fdr_hist = minp, hist
        return g

    def graph_grouped(self, cohorts, pthresh, multiallelic=False):
        """krux_scan_grouped captured as a CUDA graph; cohorts as for krux_scan_grouped."""
        arr = (Cohort * len(cohorts))()
        outs = []
        for i, c in enumerate(cohorts):
            hits, H, P = self._outputs(c["capacity"])
            outs.append((hits, H, P, c["capacity"]))
            g = c["geno"]
            arr[i].rs = c["rs"].handle
            arr[i].geno = g.data_ptr()
            arr[i].S = g.shape[0]
            arr[i].ldg = _ld(g)
            arr[i].hits = hits.data_ptr()
            arr[i].hit_H = H.data_ptr()
            arr[i].hit_p = P.data_ptr()
            arr[i].hit_capacity = c["capacity"]
        o = self._opts(pthresh, 0, flags=KRUX_FLAG_MULTIALLELIC if multiallelic else 0)
        h = ctypes.c_void_p()
        st = self.lib.krux_graph_grouped(self.handle, arr, len(cohorts), ctypes.byref(o), ctypes.byref(h))
        self._check(st, "krux_graph_grouped")
        return Graph(self, h, outs, keep=tuple(cohorts))

    # ---- end to end from host arrays -------------------------------------------
    def krux_scan_host(self, expr, geno, pthresh, capacity, out=None, stream=None):
        """End-to-end scan through the C ABI on host memory (krux_scan_host): the
        library copies expr (float32 [T, N]) and geno (int8 [S, N]) to the device,
        ranks, scans and copies the hit list back.  expr / geno: numpy arrays or
        CPU torch tensors (page-locked ones copy at the link's rate).  out: optional
        preallocated host torch tensors (hits int32 [cap, 4], H, p float64 [cap]),
        reused across calls.  Returns dict(n_hits, overflow, hits, H, p) with numpy
        views of the first min(n_hits, capacity) records and d2h_bytes."""
        import torch
        e = torch.as_tensor(expr)
        g = torch.as_tensor(geno)
        assert e.device.type == "cpu" and e.dtype == torch.float32 and e.dim() == 2 and e.stride(1) == 1
        assert g.device.type == "cpu" and g.dtype == torch.int8 and g.dim() == 2 and g.stride(1) == 1
        assert g.shape[1] == e.shape[1] or g.shape[0] == 0
        cap = max(int(capacity), 0)
        if out is None:
            out = (torch.empty((max(cap, 1), 4), dtype=torch.int32),
                   torch.empty(max(cap, 1), dtype=torch.float64),
                   torch.empty(max(cap, 1), dtype=torch.float64))
        hits, H, P = out
        assert hits.shape[0] >= cap and H.shape[0] >= cap and P.shape[0] >= cap
        o = self._opts(pthresh, cap)
        n = ctypes.c_int64()
        st = self.lib.krux_scan_host(self.handle, ctypes.c_void_p(e.data_ptr()), e.shape[0], e.shape[1],
                                     _ld(e), ctypes.c_void_p(g.data_ptr()), g.shape[0],
                                     _ld(g), ctypes.byref(o),
                                     ctypes.c_void_p(hits.data_ptr()), ctypes.c_void_p(H.data_ptr()),
                                     ctypes.c_void_p(P.data_ptr()), ctypes.byref(n), _stream(stream))
        st = self._check(st, "krux_scan_host")
        k = min(n.value, cap)
        return dict(n_hits=n.value, overflow=st == KRUX_EOVERFLOW, hits=hits[:k].numpy(),
                    H=H[:k].numpy(), p=P[:k].numpy(), d2h_bytes=k * (16 + 8 + 8))

    scan_host = krux_scan_host


class Graph:
    """A captured scan (krux_graph_*): launch() enqueues a replay, wait() returns
    one result dict per hit list (as krux_scan's).  Keeps the tensors it reads
    and writes alive."""

    def __init__(self, ctx, handle, outs, keep=()):
        self.ctx, self.handle, self.outs, self.keep = ctx, handle, outs, keep
        self.lib = ctx.lib

    def launch(self, stream=None):
        st = self.lib.krux_graph_launch(self.handle, _stream(stream))
        if st != KRUX_OK:
            raise KruxError(st, "krux_graph_launch: " + (self.lib.krux_graph_last_error(self.handle) or b"").decode())

    def wait(self):
        n = (ctypes.c_int64 * len(self.outs))()
        st = self.lib.krux_graph_wait(self.handle, n, len(self.outs))
        if st not in (KRUX_OK, KRUX_EOVERFLOW):
            raise KruxError(st, "krux_graph_wait: " + (self.lib.krux_graph_last_error(self.handle) or b"").decode())
        res = []
        for (hits, H, P, cap), cnt in zip(self.outs, n):
            k = min(cnt, cap)
            res.append(dict(n_hits=cnt, overflow=cnt > cap, hits=hits[:k], H=H[:k], p=P[:k]))
        return res

    def close(self):
        if self.handle:
            self.lib.krux_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def krux_debug_tail(kind, x, d1, d2=0.0):
    """The parametric finalisation's FP64 tails on the host (kind 0: F upper tail,
    1: two-sided t tail, 2: regularised incomplete beta I_x(d1, d2))."""
    return float(load_library().krux_debug_tail(int(kind), float(x), float(d1), float(d2)))
