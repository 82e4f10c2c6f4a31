"""Seeded synthetic inputs for the Kruskal-Wallis SNP x trait scan.

This module only draws random data: genotype matrices (SNPs x samples, int8
codes 0/1/2, -1 = missing), expression matrices (traits x samples, float32,
NaN = missing) and sample permutations.  It holds none of the statistic's
arithmetic, so both the FP64 oracle and the CUDA path can take their inputs
from here without sharing any computation.

The paper's data sets (yeast segregants, STAGE human blood: 19,610 traits x
530,222 SNPs x 102 samples, MAF > 5 %, no missing values, HWE; section
"Validation data") are not available, so these generators stand in for their
shapes and distributions.  Every generator takes a ``numpy.random.Generator``
(or a seed) and draws in a fixed, documented order.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "hwe_genotypes", "ld_block_genotypes", "expression_rounded_normal",
    "expression_lognormal", "plant_shifts", "add_missing_genotypes",
    "add_missing_expression", "splitmix64_stream", "make_perms", "config",
    "CONFIG_SHAPES", "COHORT_NS",
]

# Full shapes of the five workloads (N samples, T traits, S SNPs).
CONFIG_SHAPES = {
    1: dict(N=60, T=500, S=2_000),
    2: dict(N=102, T=20_000, S=500_000),
    3: dict(N=102, T=5_000, S=100_000),
    4: dict(N=102, T=20_000, S=200_000, P=16),
    5: dict(N=None, T=15_000, S=300_000),
}
COHORT_NS = (48, 75, 102, 150, 200, 300, 400, 500)


def _rng(seed_or_rng):
    if isinstance(seed_or_rng, np.random.Generator):
        return seed_or_rng
    return np.random.default_rng(seed_or_rng)


def _hwe_draw(rng, q, shape_rows, N):
    """Genotype codes under Hardy-Weinberg: P(0,1,2) = ((1-q)^2, 2q(1-q), q^2),
    q = per-row minor allele frequency."""
    u = rng.random((shape_rows, N), dtype=np.float32)
    q = q.astype(np.float32)[:, None]
    p0 = (1.0 - q) ** 2
    p01 = 1.0 - q * q
    return ((u >= p0).astype(np.int8) + (u >= p01).astype(np.int8))


def hwe_genotypes(rng, S, N, maf_lo=0.05, maf_hi=0.5):
    """Independent SNPs, per-SNP MAF ~ U[maf_lo, maf_hi]. Returns (geno int8 SxN, maf)."""
    rng = _rng(rng)
    maf = rng.uniform(maf_lo, maf_hi, size=S)
    geno = np.empty((S, N), dtype=np.int8)
    step = 65536
    for s0 in range(0, S, step):
        s1 = min(S, s0 + step)
        geno[s0:s1] = _hwe_draw(rng, maf[s0:s1], s1 - s0, N)
    return geno, maf


def ld_block_genotypes(rng, S, N, maf_lo=0.01, maf_hi=0.5, block=1000, redraw=0.02):
    """SNPs in linkage-disequilibrium blocks: each block of ``block`` SNPs is a
    founder SNP (HWE, MAF ~ U[maf_lo, maf_hi]) plus copies in which each entry
    is redrawn from the founder's HWE law with probability ``redraw``.

    Returns (geno int8 SxN, founders int8 BxN, block_of_snp int32 S)."""
    rng = _rng(rng)
    nb = (S + block - 1) // block
    maf = rng.uniform(maf_lo, maf_hi, size=nb)
    founders = _hwe_draw(rng, maf, nb, N)
    geno = np.empty((S, N), dtype=np.int8)
    blk = np.repeat(np.arange(nb, dtype=np.int32), block)[:S]
    bstep = 64
    for b0 in range(0, nb, bstep):
        b1 = min(nb, b0 + bstep)
        s0, s1 = b0 * block, min(S, b1 * block)
        rows = blk[s0:s1]
        g = founders[rows].copy()
        fresh = _hwe_draw(rng, maf[rows], s1 - s0, N)
        m = rng.random((s1 - s0, N), dtype=np.float32) < redraw
        g[m] = fresh[m]
        geno[s0:s1] = g
    return geno, founders, blk


def expression_rounded_normal(rng, T, N, decimals=2):
    """fp32 N(0,1) rounded to ``decimals`` decimals (many exact ties)."""
    rng = _rng(rng)
    return np.round(rng.standard_normal((T, N)), decimals).astype(np.float32)


def expression_lognormal(rng, T, N, outlier_frac=0.01, outlier_factor=10.0, log_shift=None):
    """fp32 exp(N(0,1) + log_shift), then a fraction ``outlier_frac`` of entries
    multiplied by ``outlier_factor``."""
    rng = _rng(rng)
    z = rng.standard_normal((T, N))
    if log_shift is not None:
        z = z + log_shift
    x = np.exp(z)
    if outlier_frac > 0:
        m = rng.random((T, N)) < outlier_frac
        x[m] *= outlier_factor
    return x.astype(np.float32)


def plant_shifts(rng, T, N, founders, n_causal=5, shift=1.0):
    """Planted associations: each trait gets ``n_causal`` causal LD blocks; for
    each, samples in one (non-empty, uniformly chosen) genotype group of the
    block's founder get +``shift`` on the log scale.

    Returns (log_shift float64 TxN, causal_blocks int32 T x n_causal)."""
    rng = _rng(rng)
    nb = founders.shape[0]
    n_causal = min(n_causal, nb)
    causal = np.empty((T, n_causal), dtype=np.int32)
    log_shift = np.zeros((T, N))
    for t in range(T):
        blocks = rng.choice(nb, size=n_causal, replace=False)
        causal[t] = blocks
        for b in blocks:
            f = founders[b]
            present = [g for g in (0, 1, 2) if np.any(f == g)]
            g = present[rng.integers(len(present))]
            log_shift[t, f == g] += shift
    return log_shift, causal


def add_missing_genotypes(rng, geno, snp_frac=0.10, n_patterns=200, per_pattern=2):
    """Mark ``per_pattern`` samples as missing (-1) in a fraction ``snp_frac`` of
    SNPs; each affected SNP takes one of ``n_patterns`` random sample sets.
    Modifies ``geno`` in place; returns (pattern_of_snp int32 S, -1 = complete;
    patterns int32 n_patterns x per_pattern)."""
    rng = _rng(rng)
    S, N = geno.shape
    patterns = np.stack([np.sort(rng.choice(N, size=per_pattern, replace=False))
                         for _ in range(n_patterns)]).astype(np.int32)
    affected = np.sort(rng.choice(S, size=int(round(snp_frac * S)), replace=False))
    which = rng.integers(0, n_patterns, size=affected.size).astype(np.int32)
    pat = np.full(S, -1, dtype=np.int32)
    pat[affected] = which
    for s, w in zip(affected, which):
        geno[s, patterns[w]] = -1
    return pat, patterns


def add_missing_expression(rng, expr, frac=0.01):
    """Replace a fraction ``frac`` of entries (i.i.d.) by NaN, in place."""
    rng = _rng(rng)
    m = rng.random(expr.shape) < frac
    expr[m] = np.nan
    return m


_MASK64 = (1 << 64) - 1


def splitmix64_stream(state, count):
    """``count`` outputs of SplitMix64 (Steele, Lea & Flood 2014) from ``state``."""
    out = []
    s = state & _MASK64
    for _ in range(count):
        s = (s + 0x9E3779B97F4A7C15) & _MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


def make_perms(seed, P, N):
    """P sample permutations of 0..N-1 (int32 P x N).  Permutation p is a
    Fisher-Yates shuffle of the identity driven by SplitMix64 started at state
    ``seed + p``: for i = N-1 down to 1, j = next() mod (i+1), swap(i, j)."""
    out = np.empty((P, N), dtype=np.int32)
    for p in range(P):
        perm = list(range(N))
        draws = splitmix64_stream(seed + p, max(N - 1, 0))
        for n, i in enumerate(range(N - 1, 0, -1)):
            j = draws[n] % (i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        out[p] = perm
    return out


def config(c, T=None, S=None, N=None, seed=None):
    """Inputs for workload ``c`` (1..5), optionally at reduced T/S (same
    distributions).  Seed defaults to 1307 + c.  Returns a dict with ``expr``
    (TxN float32), ``geno`` (SxN int8), ``pthresh`` and config-specific extras.

    Draw order: genotypes, then expression, then planting / missing values /
    permutations, each from the same Generator."""
    seed = 1307 + c if seed is None else seed
    rng = np.random.default_rng(seed)
    shp = dict(CONFIG_SHAPES[c])
    T = shp["T"] if T is None else T
    S = shp["S"] if S is None else S
    if c == 1:
        N = shp["N"] if N is None else N
        geno, _ = hwe_genotypes(rng, S, N, 0.05, 0.5)
        expr = expression_rounded_normal(rng, T, N)
        return dict(expr=expr, geno=geno, pthresh=1e-3, N=N, T=T, S=S)
    if c in (2, 4):
        N = shp["N"] if N is None else N
        geno, founders, blk = ld_block_genotypes(rng, S, N, 0.01, 0.5)
        log_shift, causal = plant_shifts(rng, T, N, founders)
        expr = expression_lognormal(rng, T, N, log_shift=log_shift)
        d = dict(expr=expr, geno=geno, pthresh=1e-5, N=N, T=T, S=S,
                 causal_blocks=causal, block_of_snp=blk)
        if c == 4:
            d["P"] = shp["P"]
            d["perms"] = make_perms(1307, shp["P"], N)
        return d
    if c == 3:
        N = shp["N"] if N is None else N
        geno, _, _ = ld_block_genotypes(rng, S, N, 0.05, 0.5)
        expr = expression_lognormal(rng, T, N)
        pat, patterns = add_missing_genotypes(rng, geno)
        add_missing_expression(rng, expr, 0.01)
        return dict(expr=expr, geno=geno, pthresh=1e-4, N=N, T=T, S=S,
                    pattern_of_snp=pat, patterns=patterns)
    if c == 5:
        cohorts = []
        for n_c in COHORT_NS:
            g, _ = hwe_genotypes(rng, S, n_c, 0.05, 0.5)
            e = expression_lognormal(rng, T, n_c)
            cohorts.append(dict(expr=e, geno=g, N=n_c))
        return dict(cohorts=cohorts, pthresh=1e-5, T=T, S=S)
    raise ValueError(f"unknown workload {c}")


def genome_positions(rng, S, T, n_chrom=22, chrom_len=150_000_000):
    """Synthetic map for cis scans: SNP rows spread in order over ``n_chrom``
    chromosomes of ``chrom_len`` bases (sorted uniform positions), and one gene
    position per trait (uniform over the genome, sorted).  Coordinates are global:
    chromosome * 2^40 + base position, int64, nondecreasing.  Returns
    (snp_pos [S], trait_pos [T])."""
    rng = _rng(rng)
    per = np.full(n_chrom, S // n_chrom, dtype=np.int64)
    per[: S % n_chrom] += 1
    snp = np.concatenate([(np.int64(c) << 40) + np.sort(rng.integers(0, chrom_len, size=int(k)))
                          for c, k in enumerate(per)]).astype(np.int64)
    chrom = np.sort(rng.integers(0, n_chrom, size=T)).astype(np.int64)
    gene = (chrom << 40) + rng.integers(0, chrom_len, size=T)
    order = np.lexsort((gene & ((1 << 40) - 1), chrom))
    return snp, gene[order].astype(np.int64)


def multiallelic_genotypes(rng, S, N, max_code=4, alpha=1.5):
    """Markers with a varying number of alleles (section "Input data": values
    0..l, also varying between markers): marker m uses codes 0..k_m with k_m
    uniform in 1..max_code and code frequencies ~ Dirichlet(alpha); int8 S x N."""
    rng = _rng(rng)
    k = rng.integers(1, max_code + 1, size=S)
    geno = np.empty((S, N), dtype=np.int8)
    for m in range(S):
        f = rng.dirichlet(np.full(k[m] + 1, alpha))
        geno[m] = rng.choice(k[m] + 1, size=N, p=f).astype(np.int8)
    return geno
