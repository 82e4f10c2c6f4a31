"""Pins for the FP64 oracle: each test ties the oracle to something other than
itself -- hand-worked exact examples, library routines (scipy's Kruskal-Wallis,
Mann-Whitney, chi-square and incomplete-gamma functions), invariants of the
statistic and exhaustive permutation distributions at N <= 8."""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sps
import scipy.stats as st

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kw_worked_examples.txt")


def _load_golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            vals, codes, frac, df, d = line.rstrip("\n").split("\t")
            x = np.array([float(v) for v in vals.split(",")], dtype=np.float32)
            g = np.array([int(c) for c in codes.split(",")], dtype=np.int8)
            rows.append((x, g, Fraction(frac), int(df), [int(v) for v in d.split(",")]))
    return rows


def _mp_tail(H, df):
    """Upper chi-square tail at an exact rational H, 40 digits (mpmath's
    regularised upper incomplete gamma)."""
    import mpmath as mp
    mp.mp.dps = 40
    h = mp.mpf(H.numerator) / H.denominator
    if df == 0 or h == 0:
        return 1.0
    return float(mp.gammainc(mp.mpf(df) / 2, h / 2, mp.inf, regularized=True))


@pytest.mark.parametrize("case", range(8))
def test_worked_examples(oracle_mod, case):
    x, g, H, df, d = _load_golden()[case]
    r = oracle_mod.kw_pair(x, g)
    assert r["df"] == df
    assert r["d"] == d
    assert sum(r["d"]) == 0
    assert r["H"] == pytest.approx(float(H), rel=1e-12, abs=1e-12)
    assert r["p"] == pytest.approx(_mp_tail(H, df), rel=1e-12)


def _random_case(rng, n, tie_decimals=None, missing=False):
    x = rng.standard_normal(n).astype(np.float32)
    if tie_decimals is not None:
        x = np.round(x, tie_decimals).astype(np.float32)
    g = rng.integers(0, 3, n).astype(np.int8)
    if missing:
        x[rng.random(n) < 0.1] = np.nan
        g[rng.random(n) < 0.1] = -1
    return x, g


@pytest.mark.parametrize("seed", range(40))
def test_against_scipy_kruskal(oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(5, 130))
    x, g = _random_case(rng, n, tie_decimals=[None, 1, 0][seed % 3], missing=seed % 2 == 1)
    r = oracle_mod.kw_pair(x, g)
    use = (g >= 0) & ~np.isnan(x)
    groups = [x[use & (g == i)].astype(np.float64) for i in range(3)]
    groups = [a for a in groups if a.size]
    assert r["df"] == len(groups) - 1
    if len(groups) < 2 or np.unique(x[use]).size < 2:
        assert r["H"] == 0 and r["p"] == 1
        return
    s = st.kruskal(*groups)
    assert r["H"] == pytest.approx(s.statistic, rel=1e-9, abs=1e-12)
    assert r["p"] == pytest.approx(s.pvalue, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("seed", range(20))
def test_two_groups_equal_mann_whitney(oracle_mod, seed):
    """With two groups, the Kruskal-Wallis chi-square(1) tail equals the
    two-sided normal tail of the tie-corrected Mann-Whitney z."""
    rng = np.random.default_rng(2000 + seed)
    n = int(rng.integers(6, 90))
    x = np.round(rng.standard_normal(n), seed % 3).astype(np.float32)
    g = (rng.random(n) < 0.4).astype(np.int8) * 2  # groups 0 and 2 only
    if g.min() == g.max():
        g[0] = 2 - g[0]
    r = oracle_mod.kw_pair(x, g)
    a, b = x[g == 0].astype(np.float64), x[g == 2].astype(np.float64)
    mw = st.mannwhitneyu(a, b, use_continuity=False, method="asymptotic")
    assert r["df"] == 1
    assert r["p"] == pytest.approx(mw.pvalue, rel=1e-9, abs=1e-15)


@pytest.mark.parametrize("H", [1e-6, 0.3, 2.0, 7.5, 19.2, 35.0, 60.0, 120.0, 600.0])
def test_closed_form_tails_vs_library(oracle_mod, H):
    """The closed forms used for df=1 (erfc) and df=2 (exp) against scipy's
    chi-square law and the regularised upper incomplete gamma Q(df/2, H/2)."""
    for df in (1, 2):
        ref1 = st.chi2.sf(H, df)
        ref2 = sps.gammaincc(df / 2.0, H / 2.0)
        closed = math.erfc(math.sqrt(H / 2)) if df == 1 else math.exp(-H / 2)
        assert closed == pytest.approx(ref1, rel=1e-12)
        assert closed == pytest.approx(ref2, rel=1e-12)


@pytest.mark.parametrize("seed", range(30))
def test_oracle_tail_matches_chi2(oracle_mod, seed):
    rng = np.random.default_rng(3000 + seed)
    n = int(rng.integers(8, 120))
    x, g = _random_case(rng, n, tie_decimals=seed % 2 or None)
    r = oracle_mod.kw_pair(x, g)
    if r["df"] == 0 or r["H"] == 0:
        return
    assert r["p"] == pytest.approx(st.chi2.sf(r["H"], r["df"]), rel=1e-11, abs=1e-300)
    assert r["p"] == pytest.approx(sps.gammaincc(r["df"] / 2, r["H"] / 2), rel=1e-11, abs=1e-300)


@pytest.mark.parametrize("seed", range(30))
def test_two_textbook_forms_agree(oracle_mod, seed):
    rng = np.random.default_rng(4000 + seed)
    n = int(rng.integers(4, 200))
    x, g = _random_case(rng, n, tie_decimals=[None, 1, 0][seed % 3], missing=seed % 2 == 0)
    r = oracle_mod.kw_pair(x, g)
    if r["df"] == 0 or r["H"] == 0:
        return
    assert r["H"] == pytest.approx(r["H_alt"], rel=1e-10, abs=1e-11)


@pytest.mark.parametrize("seed", range(20))
def test_rank_row_against_scipy(oracle_mod, seed):
    rng = np.random.default_rng(5000 + seed)
    n = int(rng.integers(1, 520))
    x = np.round(rng.standard_normal(n), [None, 2, 1, 0][seed % 4] or 6).astype(np.float32)
    if seed % 2:
        x[rng.random(n) < 0.05] = np.nan
    r2, tie, K = oracle_mod.rank_row(x)
    ok = ~np.isnan(x)
    assert K == ok.sum()
    assert np.all(r2[~ok] == 0)
    ref = st.rankdata(x[ok].astype(np.float64), method="average")
    assert np.array_equal(r2[ok], np.rint(2 * ref).astype(np.int64))
    # tie sum from the run lengths counted independently
    _, counts = np.unique(x[ok], return_counts=True)
    assert tie == float(np.sum(counts.astype(np.int64) ** 3 - counts))
    # sum of 2*ranks = K(K+1); sum over samples of (eq^2 - 1) = sum(t^3 - t)
    assert r2.sum() == K * (K + 1)
    eq = np.array([np.sum(x[ok] == v) for v in x[ok]], dtype=np.int64)
    assert np.sum(eq * eq - 1) == tie


def test_negative_zero_ties_with_zero(oracle_mod):
    x = np.array([0.0, -0.0, 1.0, -1.0], dtype=np.float32)
    r2, tie, K = oracle_mod.rank_row(x)
    assert list(r2) == [5, 5, 8, 2] and tie == 6.0 and K == 4


@pytest.mark.parametrize("seed", range(20))
def test_invariances(oracle_mod, seed):
    rng = np.random.default_rng(6000 + seed)
    n = int(rng.integers(6, 100))
    x, g = _random_case(rng, n, tie_decimals=seed % 2 or None, missing=seed % 3 == 0)
    base = oracle_mod.kw_pair(x, g)
    # strictly increasing transform of the trait (exact in float32 ordering)
    y = np.where(np.isnan(x), np.nan, np.exp(x.astype(np.float64) / 4.0)).astype(np.float32)
    # exp/4 stays strictly increasing on float32 inputs in [-6, 6] only if no two
    # distinct inputs collapse: check that first, then compare.
    ok = ~np.isnan(x)
    if np.unique(y[ok]).size == np.unique(x[ok]).size:
        assert oracle_mod.kw_pair(y, g)["H"] == pytest.approx(base["H"], rel=1e-12, abs=1e-12)
    # doubling is exact in float32 and strictly increasing
    z = (x * 2).astype(np.float32)
    assert oracle_mod.kw_pair(z, g)["H"] == pytest.approx(base["H"], rel=1e-12, abs=1e-12)
    # joint permutation of samples
    perm = rng.permutation(n)
    assert oracle_mod.kw_pair(x[perm], g[perm])["H"] == pytest.approx(base["H"], rel=1e-12, abs=1e-12)
    # relabelling of genotype codes (keeping -1)
    lab = rng.permutation(3).astype(np.int8)
    g2 = np.where(g >= 0, lab[np.clip(g, 0, 2)], -1).astype(np.int8)
    assert oracle_mod.kw_pair(x, g2)["H"] == pytest.approx(base["H"], rel=1e-12, abs=1e-12)
    # one group only
    one = np.where(g >= 0, 1, -1).astype(np.int8)
    r = oracle_mod.kw_pair(x, one)
    assert r["H"] == 0 and r["p"] == 1 and r["df"] == 0


EXHAUSTIVE = [
    ([1, 2, 3, 4, 5, 6], [0, 0, 1, 1, 2, 2]),
    ([1, 1, 2, 3, 3, 3], [0, 1, 0, 1, 2, 2]),
    ([0.5, 0.5, 0.5, 2, 3, 3, 7], [0, 0, 1, 1, 1, 2, 2]),
    ([4, 1, 1, 2, 9, 9, 9, 3], [0, 1, 1, 1, 2, 2, 0, 0]),
    ([5, 3, 3, 1, 8, 2, 2, 2], [0, 0, 0, 2, 2, 2, 2, 2]),
]


@pytest.mark.parametrize("case", range(len(EXHAUSTIVE)))
def test_exhaustive_permutation_mean(oracle_mod, case):
    """Over all K! relabellings of samples the mean of the tie-corrected H is
    exactly k - 1 (k non-empty groups), with or without ties.  Each relabelling
    is one SNP row of a dense oracle scan."""
    x, g = EXHAUSTIVE[case]
    x = np.array(x, dtype=np.float32)
    g = np.array(g, dtype=np.int8)
    K = x.size
    k = np.unique(g).size
    perms = np.array(list(itertools.permutations(range(K))), dtype=np.int64)
    geno = g[perms].astype(np.int8)
    r = oracle_mod.scan(x[None, :], geno, 0.05)
    H = r["H"][0]
    assert np.all(r["df"][0] == k - 1)
    assert H.mean() == pytest.approx(k - 1, rel=1e-12)
    # the multiset is symmetric under relabelling: each distinct labelling of
    # group sizes appears prod(n_i!) times, so counts of each H value are
    # multiples of that factor
    fact = np.prod([math.factorial(int(np.sum(g == i))) for i in range(3)])
    _, counts = np.unique(np.round(H, 9), return_counts=True)
    assert np.all(counts % fact == 0)


def test_scan_matches_pairs_and_centred_sums(oracle_mod):
    import synth
    d = synth.config(1, T=7, S=40)
    r = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"])
    for a in range(7):
        for b in range(0, 40, 7):
            one = oracle_mod.kw_pair(d["expr"][a], d["geno"][b], d["pthresh"])
            assert r["H"][a, b] == one["H"] and r["p"][a, b] == one["p"]
            assert list(r["d"][a, b]) == one["d"]
    assert np.all(r["d"].sum(axis=2) == 0)
    assert np.all(r["n"].sum(axis=2) == r["K"])


def test_permuted_scan_equals_scan_of_permuted_expression(oracle_mod):
    import synth
    d = synth.config(4, T=5, S=30)
    perms = synth.make_perms(1307, 3, d["N"])
    for q in range(3):
        a = oracle_mod.scan(d["expr"], d["geno"], 1e-5, perm=perms[q])
        b = oracle_mod.scan(np.ascontiguousarray(d["expr"][:, perms[q]]), d["geno"], 1e-5)
        assert np.array_equal(a["H"], b["H"]) and np.array_equal(a["p"], b["p"])
        m = oracle_mod.perm_minp(d["expr"], d["geno"], perms[q:q + 1])
        assert np.array_equal(m[0], b["p"].min(axis=1))


def test_bad_genotype_code_raises(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.kw_pair(np.arange(4, dtype=np.float32), np.array([0, 1, 3, 2], np.int8))


def _read_fdr_golden():
    rows = {}
    for line in open(os.path.join(os.path.dirname(GOLDEN), "fdr_worked_example.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.rstrip("\n").split("\t")
        rows.setdefault(k, []).append(np.array([float(x) for x in v.split(",")]))
    return rows


def test_fdr_worked_example(oracle_mod):
    g = _read_fdr_golden()
    n_real, pc, fdr = oracle_mod.fdr_from_pvalues(g["real"][0], g["perm"], g["pthresh"][0][0],
                                                  g["thresholds"][0])
    assert np.array_equal(n_real, g["n_real"][0])
    assert np.array_equal(pc, np.stack(g["perm_counts"]))
    assert np.allclose(fdr, g["fdr"][0], equal_nan=True, rtol=0, atol=1e-15)


def test_fdr_of_identity_permutations_is_one(oracle_mod):
    """Randomised data identical to the real data: FDR = 1 wherever it is defined."""
    d = synth.config(4, T=12, S=150, N=30, seed=77)
    ident = np.tile(np.arange(d["N"], dtype=np.int32), (2, 1))
    thr = 0.05 * 10.0 ** -np.arange(0, 3, 0.5)
    n_real, pc, fdr = oracle_mod.fdr(d["expr"], d["geno"], ident, 0.05, thr)
    assert n_real[0] > 0
    assert np.array_equal(pc[0], n_real) and np.array_equal(pc[1], n_real)
    assert np.all(fdr[n_real > 0] == 1.0)


def test_fdr_counts_match_permuted_scans(oracle_mod):
    """The permuted counts are those of a scan of the column-permuted expression."""
    d = synth.config(4, T=10, S=120, N=40, seed=78)
    perms = synth.make_perms(5, 2, d["N"])
    thr = np.array([0.05, 0.01, 0.001])
    _, pc, _ = oracle_mod.fdr(d["expr"], d["geno"], perms, 0.05, thr)
    for q in range(2):
        p = oracle_mod.scan(np.ascontiguousarray(d["expr"][:, perms[q]]), d["geno"], 0.05)["p"]
        p = p[p < 0.05]
        assert list(pc[q]) == [int((p <= t).sum()) for t in thr]


def test_cis_window_mask(oracle_mod):
    """Pairs kept by the cis filter: |snp_pos - trait_pos| <= window, worked by hand."""
    rng = np.random.default_rng(3)
    expr = rng.standard_normal((3, 12)).astype(np.float32)
    geno = rng.integers(0, 3, size=(4, 12)).astype(np.int8)
    snp_pos = np.array([0, 10, 20, (1 << 40)], dtype=np.int64)
    trait_pos = np.array([5, 15, (1 << 40) + 3], dtype=np.int64)
    r = oracle_mod.scan_cis(expr, geno, 0.5, snp_pos, trait_pos, 5)
    want = np.array([[1, 1, 0, 0], [0, 1, 1, 0], [0, 0, 0, 1]], dtype=bool)
    assert np.array_equal(r["in_window"], want)
    full = oracle_mod.scan(expr, geno, 0.5)
    assert np.array_equal(r["hit"], full["hit"] & want)
    wide = oracle_mod.scan_cis(expr, geno, 0.5, snp_pos, trait_pos, 1 << 62)
    assert np.array_equal(wide["hit"], full["hit"])



def _load_multi():
    rows = []
    with open(os.path.join(os.path.dirname(GOLDEN), "kw_multiallelic_examples.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            vals, codes, mc, frac, df, d = line.rstrip("\n").split("\t")
            rows.append((np.array([float(v) for v in vals.split(",")], dtype=np.float32),
                         np.array([int(c) for c in codes.split(",")], dtype=np.int8), int(mc),
                         Fraction(frac), int(df), [int(v) for v in d.split(",")]))
    return rows


@pytest.mark.parametrize("case", range(4))
def test_multiallelic_worked_examples(oracle_mod, case):
    x, g, mc, H, df, d = _load_multi()[case]
    r = oracle_mod.kw_pair(x, g, max_code=mc)
    assert r["df"] == df and r["d"] == d
    assert r["H"] == pytest.approx(float(H), rel=1e-13, abs=1e-13)
    assert r["p"] == pytest.approx(_mp_tail(H, df), rel=1e-12)


@pytest.mark.parametrize("df", range(1, 9))
def test_chi2_tail_all_df(oracle_mod, df):
    """Closed forms of Q(df/2, H/2) against scipy's chi2.sf and gammaincc."""
    for H in [1e-6, 0.3, 1.0, 4.7, 12.0, 31.5, 80.0, 300.0]:
        want = st.chi2.sf(H, df)
        assert oracle_mod.chi2_upper(H, df) == pytest.approx(want, rel=1e-11, abs=1e-300)
        assert oracle_mod.chi2_upper(H, df) == pytest.approx(sps.gammaincc(df / 2, H / 2), rel=1e-11,
                                                             abs=1e-300)


@pytest.mark.parametrize("mc", [3, 4])
def test_multiallelic_matches_scipy(oracle_mod, mc):
    rng = np.random.default_rng(100 + mc)
    checked = 0
    for j in range(60):
        n = int(rng.integers(8, 90))
        x = np.round(rng.standard_normal(n), j % 3).astype(np.float32)
        g = rng.integers(0, mc + 1, n).astype(np.int8)
        if j % 2:
            x[rng.random(n) < 0.1] = np.nan
            g[rng.random(n) < 0.1] = -1
        use = (g >= 0) & ~np.isnan(x)
        groups = [x[use & (g == k)].astype(np.float64) for k in range(mc + 1)]
        groups = [a for a in groups if a.size]
        if len(groups) < 2 or np.unique(np.concatenate(groups)).size < 2:
            continue
        s = st.kruskal(*groups)
        r = oracle_mod.kw_pair(x, g, max_code=mc)
        assert r["df"] == len(groups) - 1
        assert r["H"] == pytest.approx(s.statistic, rel=1e-9)
        assert r["p"] == pytest.approx(s.pvalue, rel=1e-9)
        assert r["H_alt"] == pytest.approx(r["H"], rel=1e-11, abs=1e-11)
        checked += 1
    assert checked > 40


def test_multiallelic_exhaustive_permutation_mean(oracle_mod):
    """Four groups, N = 7 with ties: over all 7! relabellings the mean H is k - 1 = 3."""
    x = np.array([1, 2, 2, 3, 5, 5, 8], dtype=np.float32)
    g = np.array([0, 0, 1, 1, 2, 3, 3], dtype=np.int8)
    perms = np.array(list(itertools.permutations(range(7))), dtype=np.int64)
    r = oracle_mod.scan(x[None, :], g[perms].astype(np.int8), 0.05, max_code=3)
    assert np.all(r["df"][0] == 3)
    assert r["H"][0].mean() == pytest.approx(3.0, rel=1e-12)


def test_biallelic_data_gives_the_same_results_as_multiallelic_mode(oracle_mod):
    d = synth.config(1, T=6, S=40, seed=5)
    a = oracle_mod.scan(d["expr"], d["geno"], 1e-3)
    b = oracle_mod.scan(d["expr"], d["geno"], 1e-3, max_code=4)
    assert np.array_equal(a["H"], b["H"]) and np.array_equal(a["p"], b["p"])
    assert np.array_equal(a["d"], b["d"][..., :3]) and np.all(b["d"][..., 3:] == 0)


def _load_param():
    rows = []
    with open(os.path.join(os.path.dirname(GOLDEN), "parametric_worked_examples.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            vals, codes, model, frac, d1, d2 = line.rstrip("\n").split("\t")
            rows.append((np.array([float(v) for v in vals.split(",")]),
                         np.array([int(c) for c in codes.split(",")], dtype=np.int8), model,
                         Fraction(frac), int(d1), int(d2)))
    return rows


@pytest.mark.parametrize("case", range(4))
def test_parametric_worked_examples(oracle_mod, case):
    x, g, model, val, d1, d2 = _load_param()[case]
    stat, p = oracle_mod.parametric_pair(x, g, model)
    if model == "anova":
        assert stat == pytest.approx(float(val), rel=1e-13)
        assert p == pytest.approx(st.f.sf(float(val), d1, d2), rel=1e-12)
    else:
        assert stat * stat == pytest.approx(float(val), rel=1e-13)
        # the two-sided t tail equals the F(1, K-2) tail of t^2
        assert p == pytest.approx(st.f.sf(float(val), 1, d2), rel=1e-10)


def test_parametric_matches_scipy_routines(oracle_mod):
    """ANOVA against scipy's f_oneway, linear against scipy's linregress."""
    rng = np.random.default_rng(91)
    n_checked = 0
    for j in range(40):
        n = int(rng.integers(8, 120))
        x = rng.standard_normal(n) + 3.0 * (j % 5)
        g = rng.integers(0, 3, n).astype(np.int8)
        if j % 3 == 0:
            g[rng.random(n) < 0.1] = -1
        use = g >= 0
        groups = [x[use & (g == c)] for c in range(3) if np.any(use & (g == c))]
        if len(groups) < 2:
            continue
        F, pF = oracle_mod.parametric_pair(x, g, "anova")
        ref = st.f_oneway(*groups)
        assert F == pytest.approx(ref.statistic, rel=1e-10) and pF == pytest.approx(ref.pvalue, rel=1e-9)
        t, pt = oracle_mod.parametric_pair(x, g, "linear")
        lr = st.linregress(g[use].astype(float), x[use])
        assert pt == pytest.approx(lr.pvalue, rel=1e-9)
        assert t == pytest.approx(lr.slope / lr.stderr, rel=1e-9)
        n_checked += 1
    assert n_checked > 30


def test_parametric_invariances(oracle_mod):
    """Both statistics are invariant under x -> a x + b (a > 0); the linear t flips
    sign with the dosage direction; ANOVA ignores group labels."""
    rng = np.random.default_rng(92)
    x = rng.standard_normal(50)
    g = rng.integers(0, 3, 50).astype(np.int8)
    for model in ("anova", "linear"):
        s0, p0 = oracle_mod.parametric_pair(x, g, model)
        s1, p1 = oracle_mod.parametric_pair(7.0 * x - 300.0, g, model)
        assert s1 == pytest.approx(s0, rel=1e-9) and p1 == pytest.approx(p0, rel=1e-9)
    t0, _ = oracle_mod.parametric_pair(x, g, "linear")
    t1, _ = oracle_mod.parametric_pair(x, (2 - g).astype(np.int8), "linear")
    assert t1 == pytest.approx(-t0, rel=1e-12)
    F0, _ = oracle_mod.parametric_pair(x, g, "anova")
    F1, _ = oracle_mod.parametric_pair(x, np.array([1, 2, 0], np.int8)[g], "anova")
    assert F1 == pytest.approx(F0, rel=1e-12)
