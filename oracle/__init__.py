"""FP64 CPU oracle for the Kruskal-Wallis SNP x trait scan (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import this package.  The product path (the CUDA library and
its binding) never imports it.  The arithmetic lives in ``krux_oracle.c``
(plain C, FP64, one pair at a time from the definition: sort, average ranks,
group rank sums, Eq. 2, tie correction, chi-square tail); this module compiles
it with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "krux_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libkrux_oracle.so")
_lib = None


class _Pair(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("H_alt", ctypes.c_double),
                ("p", ctypes.c_double), ("tie", ctypes.c_double),
                ("rank2", ctypes.c_int64 * 5), ("d", ctypes.c_int64 * 5),
                ("n", ctypes.c_int32 * 5), ("K", ctypes.c_int32),
                ("df", ctypes.c_int32), ("hit", ctypes.c_int32)]


def build(force=False):
    """Compile krux_oracle.c into _build/libkrux_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_pair.argtypes = [P, P, ctypes.c_int, ctypes.c_double, ctypes.POINTER(_Pair)]
        lib.oracle_pair.restype = ctypes.c_int
        lib.oracle_pair_l.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.POINTER(_Pair)]
        lib.oracle_pair_l.restype = ctypes.c_int
        lib.oracle_chi2_upper.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.oracle_chi2_upper.restype = ctypes.c_double
        lib.oracle_scan_l.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      P, ctypes.c_int64, P, ctypes.c_int64, P,
                                      ctypes.c_double, P, P, P, P, P, P, P, P]
        lib.oracle_scan_l.restype = ctypes.c_int
        lib.oracle_rank_row.argtypes = [P, ctypes.c_int, P, ctypes.POINTER(ctypes.c_double)]
        lib.oracle_rank_row.restype = ctypes.c_int32
        lib.oracle_scan.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int,
                                    P, ctypes.c_int64, P, ctypes.c_int64, P,
                                    ctypes.c_double, P, P, P, P, P, P, P, P]
        lib.oracle_scan.restype = ctypes.c_int
        lib.oracle_perm_minp.argtypes = [P, ctypes.c_int64, P, ctypes.c_int64, ctypes.c_int,
                                         P, ctypes.c_int64, P, ctypes.c_int64, P,
                                         ctypes.c_int, P]
        lib.oracle_perm_minp.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def num_threads():
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def kw_pair(x, g, pthresh=0.05, max_code=2):
    """Kruskal-Wallis test of one trait against one marker with codes
    0..max_code (max_code <= 4; -1 = missing).  Returns a dict with H, H_alt, p,
    df, K, tie, n (max_code+1), rank2 (max_code+1) = 2*rank sums, d
    (max_code+1) = centred sums 2*S_i - N_i*(K+1), hit."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    g = np.ascontiguousarray(g, dtype=np.int8)
    assert x.shape == g.shape and x.ndim == 1
    r = _Pair()
    rc = _load().oracle_pair_l(_ptr(x), _ptr(g), x.size, int(max_code), float(pthresh),
                               ctypes.byref(r))
    if rc != 0:
        raise ValueError(f"genotype code outside {{-1, 0..{max_code}}}")
    k = max_code + 1
    return dict(H=r.H, H_alt=r.H_alt, p=r.p, df=r.df, K=r.K, tie=r.tie,
                n=list(r.n)[:k], rank2=list(r.rank2)[:k], d=list(r.d)[:k], hit=bool(r.hit))


def chi2_upper(H, df):
    """Upper tail of the chi-square law with df degrees of freedom at H."""
    return float(_load().oracle_chi2_upper(float(H), int(df)))


def rank_row(x):
    """(2*average rank int64 array, 0 at NaN; tie sum; K) of one row."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    r2 = np.empty(x.size, dtype=np.int64)
    tie = ctypes.c_double()
    K = _load().oracle_rank_row(_ptr(x), x.size, _ptr(r2), ctypes.byref(tie))
    return r2, tie.value, int(K)


def scan(expr, geno, pthresh, traits=None, snps=None, perm=None, max_code=2):
    """Dense per-pair results over traits x snps (defaults: all); genotype codes
    0..max_code.  Returns a dict of arrays shaped (len(traits), len(snps)): H, p,
    df, K, hit, H_alt, and d / n shaped (..., max_code + 1)."""
    expr = np.ascontiguousarray(expr, dtype=np.float32)
    geno = np.ascontiguousarray(geno, dtype=np.int8)
    T, N = expr.shape
    S, N2 = geno.shape
    assert N == N2
    traits = np.arange(T, dtype=np.int64) if traits is None else np.ascontiguousarray(traits, dtype=np.int64)
    snps = np.arange(S, dtype=np.int64) if snps is None else np.ascontiguousarray(snps, dtype=np.int64)
    nt, ns = traits.size, snps.size
    ng = max_code + 1
    out = dict(H=np.empty((nt, ns)), p=np.empty((nt, ns)),
               df=np.empty((nt, ns), np.int32), d=np.empty((nt, ns, ng), np.int64),
               n=np.empty((nt, ns, ng), np.int32), K=np.empty((nt, ns), np.int32),
               hit=np.empty((nt, ns), np.uint8), H_alt=np.empty((nt, ns)))
    pp = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    rc = _load().oracle_scan_l(_ptr(expr), N, _ptr(geno), N, N, int(max_code), _ptr(traits), nt,
                               _ptr(snps), ns, _ptr(pp), float(pthresh),
                               _ptr(out["H"]), _ptr(out["p"]), _ptr(out["df"]),
                               _ptr(out["d"]), _ptr(out["n"]), _ptr(out["K"]),
                               _ptr(out["hit"]), _ptr(out["H_alt"]))
    if rc != 0:
        raise ValueError(f"genotype code outside {{-1, 0..{max_code}}}")
    out["hit"] = out["hit"].astype(bool)
    return out


def hits(expr, geno, pthresh, traits=None, snps=None):
    """Sorted hit list (trait, snp) (global indices) with p < pthresh, and the
    dense result dict it came from."""
    r = scan(expr, geno, pthresh, traits, snps)
    T, S = expr.shape[0], geno.shape[0]
    traits = np.arange(T) if traits is None else np.asarray(traits)
    snps = np.arange(S) if snps is None else np.asarray(snps)
    a, b = np.nonzero(r["hit"])
    pairs = np.stack([traits[a], snps[b]], axis=1).astype(np.int64)
    order = np.lexsort((pairs[:, 0], pairs[:, 1]))
    return pairs[order], r


def perm_minp(expr, geno, perms, traits=None, snps=None):
    """P x len(traits) minimum p over the selected SNPs, expression columns
    permuted by each row of ``perms``."""
    expr = np.ascontiguousarray(expr, dtype=np.float32)
    geno = np.ascontiguousarray(geno, dtype=np.int8)
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    T, N = expr.shape
    S = geno.shape[0]
    traits = np.arange(T, dtype=np.int64) if traits is None else np.ascontiguousarray(traits, dtype=np.int64)
    snps = np.arange(S, dtype=np.int64) if snps is None else np.ascontiguousarray(snps, dtype=np.int64)
    P = perms.shape[0]
    out = np.empty((P, traits.size))
    rc = _load().oracle_perm_minp(_ptr(expr), N, _ptr(geno), N, N, _ptr(traits), traits.size,
                                  _ptr(snps), snps.size, _ptr(perms), P, _ptr(out))
    if rc != 0:
        raise ValueError("genotype code outside {-1,0,1,2}")
    return out


def fdr_from_pvalues(p_real, p_perm, pthresh, thresholds):
    """Empirical FDR (section "P-value calculation and empirical FDR correction"):
    for each threshold P <= P_c, the mean over the randomised data sets of the
    number of pairs with P' <= P, divided by the number of real pairs with P' <= P.
    Only pairs with p < P_c take part (the permuted scans use the same P_c).
    p_real: 1-D p-values of the real data; p_perm: list of 1-D arrays, one per
    permutation.  Returns (n_real [len(thresholds)], perm_counts [P, len], fdr),
    fdr NaN where n_real is 0."""
    thr = np.asarray(thresholds, dtype=np.float64)

    def count(pv):
        pv = np.asarray(pv, dtype=np.float64).ravel()
        pv = pv[pv < pthresh]
        return np.array([int(np.count_nonzero(pv <= P)) for P in thr], dtype=np.int64)

    n_real = count(p_real)
    perm_counts = np.stack([count(q) for q in p_perm]) if len(p_perm) else np.zeros((0, thr.size), np.int64)
    mean = perm_counts.mean(axis=0) if len(p_perm) else np.full(thr.size, np.nan)
    fdr = np.array([mean[i] / n_real[i] if n_real[i] > 0 else np.nan for i in range(thr.size)])
    return n_real, perm_counts, fdr


def fdr(expr, geno, perms, pthresh, thresholds, snps=None):
    """Empirical FDR of the scan at each threshold: the real scan and one scan
    per permutation row of ``perms`` (expression columns permuted), all traits."""
    p_real = scan(expr, geno, pthresh, snps=snps)["p"]
    p_perm = [scan(expr, geno, pthresh, snps=snps, perm=perms[q])["p"] for q in range(len(perms))]
    return fdr_from_pvalues(p_real, p_perm, pthresh, thresholds)


def scan_cis(expr, geno, pthresh, snp_pos, trait_pos, window):
    """cis scan (the paper's cis-eQTL analysis: marker-trait pairs within a fixed
    distance): the full scan with every pair outside |snp_pos - trait_pos| <=
    window marked as not a hit.  Returns the dense result dict of ``scan``."""
    r = scan(expr, geno, pthresh)
    d = np.abs(np.asarray(trait_pos, dtype=np.int64)[:, None] - np.asarray(snp_pos, dtype=np.int64)[None, :])
    r["in_window"] = d <= window
    r["hit"] = r["hit"] & r["in_window"]
    return r


def parametric_pair(x, g, model):
    """Parametric statistics of one trait against one biallelic marker (the
    paper's comparison: matrix-eQTL's ANOVA and linear models), FP64 from the
    definitions over the samples with a genotype (codes 0,1,2).
    model 'anova': one-way ANOVA over the non-empty genotype groups,
      F = (SS_between / (g - 1)) / (SS_within / (K - g)), p = upper F(g-1, K-g) tail;
    model 'linear': least-squares regression of x on the dosage (the code),
      t = r sqrt((K - 2) / (1 - r^2)), p = two-sided Student t(K - 2) tail.
    Returns (stat, p); degenerate pairs (one group, constant dosage or x) give
    (0, 1).  The tails are scipy.stats' (a library step)."""
    import scipy.stats as sst
    x = np.asarray(x, dtype=np.float64)
    g = np.asarray(g)
    use = g >= 0
    x, g = x[use], g[use].astype(np.float64)
    K = x.size
    if model == "anova":
        levels = [c for c in (0, 1, 2) if np.any(g == c)]
        k = len(levels)
        if k < 2 or K <= k:
            return 0.0, 1.0
        m = x.mean()
        ssb = sum(np.sum(g == c) * (x[g == c].mean() - m) ** 2 for c in levels)
        ssw = sum(np.sum((x[g == c] - x[g == c].mean()) ** 2) for c in levels)
        if ssw == 0.0:
            return (np.inf, 0.0) if ssb > 0 else (0.0, 1.0)
        F = (ssb / (k - 1)) / (ssw / (K - k))
        return float(F), float(sst.f.sf(F, k - 1, K - k))
    if model == "linear":
        if K < 3:
            return 0.0, 1.0
        dg, dx = g - g.mean(), x - x.mean()
        sgg, sxx, sxg = np.sum(dg * dg), np.sum(dx * dx), np.sum(dx * dg)
        if sgg == 0.0 or sxx == 0.0:
            return 0.0, 1.0
        r = sxg / np.sqrt(sgg * sxx)
        if abs(r) >= 1.0:
            return (np.inf if r > 0 else -np.inf), 0.0
        t = r * np.sqrt((K - 2) / (1.0 - r * r))
        return float(t), float(2.0 * sst.t.sf(abs(t), K - 2))
    raise ValueError("model must be 'anova' or 'linear'")


def parametric_scan(expr, geno, pthresh, model, traits=None, snps=None):
    """parametric_pair over traits x snps: dict of (nt, ns) arrays stat, p, hit."""
    expr = np.asarray(expr)
    geno = np.asarray(geno)
    traits = np.arange(expr.shape[0]) if traits is None else np.asarray(traits)
    snps = np.arange(geno.shape[0]) if snps is None else np.asarray(snps)
    stat = np.empty((traits.size, snps.size))
    p = np.empty((traits.size, snps.size))
    for a, t in enumerate(traits):
        for b, s in enumerate(snps):
            stat[a, b], p[a, b] = parametric_pair(expr[t], geno[s], model)
    return dict(stat=stat, p=p, hit=p < pthresh)
