"""Batched forms through the C ABI: permutation null (per-permutation, per-trait
minimum p), several cohorts of uneven sample counts in one launch, and the
bounded device-side wait."""
import numpy as np
import pytest

import synth
from kwcheck import check_hits

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kx():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1307_3519_gb300 import build
    build.build()
    import paper_1307_3519_gb300 as k
    ctx = k.Krux(0)
    yield ctx
    ctx.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("T,S,P,N", [(200, 3000, 4, 102), (131, 700, 3, 60), (64, 1000, 2, 150),
                                     (40, 300, 2, 300)])
def test_permutation_minp(kx, oracle_mod, T, S, P, N):
    d = synth.config(4, T=T, S=S, N=N, seed=T + S)
    perms = synth.make_perms(1307, P, N)
    pth = 1e-3
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_permute(rs, _dev(d["geno"]), _dev(perms), pth, capacity=T * S)
    want = oracle_mod.perm_minp(d["expr"], d["geno"], perms)
    got = res["minp"].cpu().numpy()
    assert got.shape == want.shape
    assert np.all(np.abs(got - want) <= 1e-6 * want), \
        f"max rel err {np.max(np.abs(got - want) / want)}"
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    check_hits(res, orc, np.arange(T), np.arange(S), pth, must_have_hits=False)
    assert res["n_hits"] == int(orc["hit"].sum())


@pytest.mark.parametrize("nan", [0.0, 0.02])
def test_permutation_minp_with_seed_pass(kx, oracle_mod, nan):
    """Enough SNPs (70,000 > 4 x 16,384) for the seed pass that primes the minimum-p
    keys with lower bounds before the main launch (traits with NaN sit it out and
    take the exact per-pair path); every (permutation, trait) minimum p against the
    oracle, on LD-block genotypes (many exact SNP copies)."""
    d = synth.config(4, T=70, S=70000, seed=91)
    if nan > 0:
        synth.add_missing_expression(np.random.default_rng(5), d["expr"], nan)
    perms = synth.make_perms(1307, 2, d["N"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_permute(rs, _dev(d["geno"]), _dev(perms), 1e-5, capacity=70 * 70000)
    want = oracle_mod.perm_minp(d["expr"], d["geno"], perms)
    got = res["minp"].cpu().numpy()
    assert got.shape == want.shape
    assert np.all(np.abs(got - want) <= 1e-6 * want), np.max(np.abs(got - want) / want)


def test_permutation_minp_with_nan_expression(kx, oracle_mod):
    """NaN expression values move with the permuted columns: each permutation's
    group sizes exclude the samples whose permuted value is NaN."""
    T, S, P, N = 90, 800, 3, 80
    d = synth.config(3, T=T, S=S, N=N, seed=91)
    geno = np.where(d["geno"] < 0, 0, d["geno"]).astype(np.int8)
    assert np.isnan(d["expr"]).any()
    perms = synth.make_perms(17, P, N)
    pth = 1e-3
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_permute(rs, _dev(geno), _dev(perms), pth, capacity=T * S)
    want = oracle_mod.perm_minp(d["expr"], geno, perms)
    got = res["minp"].cpu().numpy()
    assert np.all(np.abs(got - want) <= 1e-6 * want), \
        f"max rel err {np.max(np.abs(got - want) / want)}"
    orc = oracle_mod.scan(d["expr"], geno, pth)
    check_hits(res, orc, np.arange(T), np.arange(S), pth, must_have_hits=False)


def test_permutation_rejects_bad_rows(kx):
    import paper_1307_3519_gb300 as k
    d = synth.config(4, T=10, S=50, seed=1)
    perms = synth.make_perms(3, 2, d["N"])
    perms[1, 0] = perms[1, 1]
    rs = kx.krux_rank(_dev(d["expr"]))
    with pytest.raises(k.KruxError) as e:
        kx.krux_permute(rs, _dev(d["geno"]), _dev(perms), 1e-3, capacity=10)
    assert e.value.status == k.KRUX_EINVAL


def test_grouped_cohorts(kx, oracle_mod):
    """Cohorts of uneven sample counts in one persistent launch, each against its
    own genotypes (the multi-cohort workload at reduced T and S)."""
    Ns = [48, 75, 102, 150, 200, 300, 500]
    rng = np.random.default_rng(5)
    cohorts, data = [], []
    for n_c in Ns:
        g, _ = synth.hwe_genotypes(rng, 700, n_c, 0.05, 0.5)
        e = synth.expression_lognormal(rng, 150, n_c)
        data.append((e, g))
        cohorts.append(dict(rs=kx.krux_rank(_dev(e)), geno=_dev(g), capacity=150 * 700))
    pth = 1e-2
    out = kx.krux_scan_grouped(cohorts, pth)
    for (e, g), res in zip(data, out):
        orc = oracle_mod.scan(e, g, pth)
        check_hits(res, orc, np.arange(150), np.arange(700), pth)
        assert res["n_hits"] == int(orc["hit"].sum())


def test_grouped_cohorts_with_missing_values(kx, oracle_mod):
    """Cohorts of different N in one launch, each with missing-genotype patterns and
    NaN expression: the buckets of every cohort are re-ranked by one launch and
    share one tensor map per cohort, groups of different width share the packed B
    buffer, and the traits with NaN take the exact-size hot test."""
    Ns = [60, 102, 150]
    rng = np.random.default_rng(17)
    cohorts, data = [], []
    for n_c in Ns:
        g, _ = synth.hwe_genotypes(rng, 900, n_c, 0.05, 0.5)
        synth.add_missing_genotypes(rng, g, snp_frac=0.15, n_patterns=9, per_pattern=2)
        e = synth.expression_lognormal(rng, 140, n_c)
        synth.add_missing_expression(rng, e, 0.02)
        data.append((e, g))
        cohorts.append(dict(rs=kx.krux_rank(_dev(e)), geno=_dev(g), capacity=140 * 900))
    pth = 1e-2
    out = kx.krux_scan_grouped(cohorts, pth)
    for (e, g), res in zip(data, out):
        orc = oracle_mod.scan(e, g, pth)
        check_hits(res, orc, np.arange(140), np.arange(900), pth)


def test_bounded_wait_reports_timeout_and_context_survives(kx, oracle_mod):
    """With a one-cycle wait limit the first wait that has to spin gives up: the
    kernel drains its copies, frees TMEM and the call returns KRUX_ETIMEOUT.  The
    context stays usable and the next call with the default limit is correct."""
    import paper_1307_3519_gb300 as k
    d = synth.config(1, T=300, S=4000, seed=12)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    kx.set_wait_limit(1)
    try:
        with pytest.raises(k.KruxError) as e:
            kx.krux_scan(rs, g, 1e-3, capacity=300 * 4000)
        assert e.value.status == k.KRUX_ETIMEOUT
    finally:
        kx.set_wait_limit(0)
    res = kx.krux_scan(rs, g, 1e-3, capacity=300 * 4000)
    orc = oracle_mod.scan(d["expr"], d["geno"], 1e-3)
    check_hits(res, orc, np.arange(300), np.arange(4000), 1e-3)


@pytest.mark.parametrize("T,S,P,N,nan", [(150, 2500, 3, 102, False), (70, 900, 2, 75, True)])
def test_permutation_fdr_histogram(kx, oracle_mod, T, S, P, N, nan):
    """Per-permutation counts of p' < P_c by -log10 p bin, and the real data's
    row, against the oracle's p of every pair; the FDR curve from it equals the
    definition evaluated by the oracle."""
    from paper_1307_3519_gb300.fdr import fdr_curve
    d = synth.config(3 if nan else 4, T=T, S=S, N=N, seed=T * 7 + S)
    expr = d["expr"]
    geno = np.where(d["geno"] < 0, 0, d["geno"]).astype(np.int8)  # complete genotypes
    perms = synth.make_perms(11, P, N)
    pth, w, bins = 1e-2, 0.2, 16
    rs = kx.krux_rank(_dev(expr))
    res = kx.krux_permute(rs, _dev(geno), _dev(perms), pth, capacity=T * S, fdr_bins=bins,
                          fdr_bin_width=w)
    got = res["fdr_hist"].cpu().numpy()
    rows = [oracle_mod.scan(expr, geno, pth)["p"]]
    rows += [oracle_mod.scan(expr, geno, pth, perm=perms[q])["p"] for q in range(P)]
    l0 = -np.log10(pth)
    for q, p in enumerate(rows):
        p = p[p < pth]
        x = (-np.log10(p) - l0) / w
        want = np.bincount(np.clip(np.floor(x), 0, bins - 1).astype(np.int64), minlength=bins)
        near = np.abs(x - np.round(x)) < 1e-9
        assert np.sum(np.abs(got[q] - want)) <= 2 * int(near.sum()), (q, got[q], want)
        assert got[q].sum() == p.size
    c = fdr_curve(got, pth, w)
    n_real, pc, fdr = oracle_mod.fdr_from_pvalues(rows[0], rows[1:], pth, c["threshold"])
    assert np.array_equal(c["n_real"], n_real) and np.array_equal(c["mean_perm"] * P, pc.sum(axis=0))
    assert np.allclose(c["fdr"], fdr, rtol=1e-12, atol=0, equal_nan=True)


def test_plain_forms_are_the_default(kx):
    """Without any tuning, complete data take the plain scan form (0) and a
    permutation batch its two-sided variant (4); NaN expression takes the plain
    form's NaN variant (5), unless more than one trait in 128 has more than six NaN
    samples (the general form, 3); a permutation batch with NaN takes the
    permutation form (2)."""
    import paper_1307_3519_gb300 as k
    ctx = k.Krux(0)
    ctx.set_profiling(True)
    d = synth.config(4, T=300, S=5000, seed=3)
    rs, g, pm = ctx.krux_rank(_dev(d["expr"])), _dev(d["geno"]), _dev(d["perms"][:3])
    ctx.krux_scan(rs, g, 1e-4, capacity=300 * 5000)
    assert ctx.profile()["scan_form"] == 0
    ctx.krux_permute(rs, g, pm, 1e-4, capacity=300 * 5000, fdr_bins=8)
    assert ctx.profile()["scan_form"] == 4
    x = d["expr"].copy()
    x[5, 7] = np.nan
    rsn = ctx.krux_rank(_dev(x))
    ctx.krux_scan(rsn, g, 1e-4, capacity=300 * 5000)
    assert ctx.profile()["scan_form"] == 5
    ctx.krux_permute(rsn, g, pm, 1e-4, capacity=300 * 5000)
    assert ctx.profile()["scan_form"] == 2
    x[200:203, :7] = np.nan  # 3 of 300 traits with 7 NaN samples
    rsm = ctx.krux_rank(_dev(x))
    ctx.krux_scan(rsm, g, 1e-4, capacity=300 * 5000)
    assert ctx.profile()["scan_form"] == 3
    ctx.close()
