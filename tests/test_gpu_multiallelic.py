"""Markers with up to five genotype groups (codes 0..4, section "Input data":
any number of alleles, varying between markers) through the C ABI, against the
FP64 oracle."""
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


def _sorted(res):
    h = res["hits"].cpu().numpy()
    o = np.lexsort((h[:, 0], h[:, 1]))
    return h[o], res["H"].cpu().numpy()[o], res["p"].cpu().numpy()[o]


@pytest.mark.parametrize("T,S,N,pth", [(300, 2000, 102, 1e-3), (131, 777, 60, 1e-2),
                                       (200, 900, 150, 1e-3), (70, 400, 500, 1e-2)])
def test_multiallelic_scan(kx, oracle_mod, T, S, N, pth):
    rng = np.random.default_rng(T + S + N)
    geno = synth.multiallelic_genotypes(rng, S, N)
    expr = synth.expression_rounded_normal(rng, T, N)
    rs = kx.krux_rank(_dev(expr))
    res = kx.krux_scan(rs, _dev(geno), pth, capacity=T * S, multiallelic=True)
    orc = oracle_mod.scan(expr, geno, pth, max_code=4)
    assert orc["df"].max() >= 3
    check_hits(res, orc, np.arange(T), np.arange(S), pth)
    assert res["n_hits"] == int(orc["hit"].sum())


def test_multiallelic_planted_signal_in_all_df(kx, oracle_mod):
    """Hits of every df 1..4: a rank shift in one group of each marker."""
    rng = np.random.default_rng(9)
    T, S, N = 256, 600, 120
    geno = synth.multiallelic_genotypes(rng, S, N)
    expr = rng.standard_normal((T, N)).astype(np.float32)
    for t in range(0, T, 3):  # trait t follows marker t: shift the samples of code 0
        expr[t] += 1.2 * (geno[t % S] == 0)
    rs = kx.krux_rank(_dev(expr))
    res = kx.krux_scan(rs, _dev(geno), 1e-4, capacity=T * S, multiallelic=True)
    orc = oracle_mod.scan(expr, geno, 1e-4, max_code=4)
    assert set(np.unique(orc["df"][orc["hit"]])) >= {1, 2, 3, 4}
    check_hits(res, orc, np.arange(T), np.arange(S), 1e-4)


def test_biallelic_data_same_in_both_forms(kx):
    d = synth.config(1, T=300, S=3000, seed=81)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    a = kx.krux_scan(rs, g, 1e-3, capacity=300 * 3000)
    b = kx.krux_scan(rs, g, 1e-3, capacity=300 * 3000, multiallelic=True)
    assert a["n_hits"] == b["n_hits"] > 0
    for x, y in zip(_sorted(a), _sorted(b)):
        assert np.array_equal(x, y)


def test_multiallelic_missing_genotypes(kx, oracle_mod):
    rng = np.random.default_rng(83)
    T, S, N = 150, 1200, 102
    geno = synth.multiallelic_genotypes(rng, S, N)
    synth.add_missing_genotypes(rng, geno, snp_frac=0.1, n_patterns=12, per_pattern=2)
    expr = synth.expression_lognormal(rng, T, N)
    rs = kx.krux_rank(_dev(expr))
    res = kx.krux_scan(rs, _dev(geno), 1e-3, capacity=T * S, multiallelic=True)
    orc = oracle_mod.scan(expr, geno, 1e-3, max_code=4)
    check_hits(res, orc, np.arange(T), np.arange(S), 1e-3)


def test_multiallelic_grouped_cis_and_graph(kx, oracle_mod):
    rng = np.random.default_rng(84)
    data, cohorts = [], []
    for n_c in (48, 102, 300):
        gn = synth.multiallelic_genotypes(rng, 500, n_c)
        e = synth.expression_lognormal(rng, 140, n_c)
        data.append((e, gn))
        cohorts.append(dict(rs=kx.krux_rank(_dev(e)), geno=_dev(gn), capacity=140 * 500))
    out = kx.krux_scan_grouped(cohorts, 1e-2, multiallelic=True)
    graph = kx.graph_grouped(cohorts, 1e-2, multiallelic=True)
    graph.launch()
    gout = graph.wait()
    for (e, gn), r, q in zip(data, out, gout):
        orc = oracle_mod.scan(e, gn, 1e-2, max_code=4)
        check_hits(r, orc, np.arange(140), np.arange(500), 1e-2)
        for x, y in zip(_sorted(r), _sorted(q)):
            assert np.array_equal(x, y)
    graph.close()
    e, gn = data[1]
    snp_pos, trait_pos = synth.genome_positions(np.random.default_rng(85), 500, 140, n_chrom=1,
                                                chrom_len=2_000_000)
    res = kx.krux_scan_cis(cohorts[1]["rs"], cohorts[1]["geno"], _dev(snp_pos), _dev(trait_pos),
                           300_000, 1e-2, capacity=140 * 500, multiallelic=True)
    orc = oracle_mod.scan(e, gn, 1e-2, max_code=4)
    orc["hit"] &= np.abs(trait_pos[:, None] - snp_pos[None, :]) <= 300_000
    check_hits(res, orc, np.arange(140), np.arange(500), 1e-2, must_have_hits=False)


def test_multiallelic_codes_checked(kx):
    import paper_1307_3519_gb300 as k
    rng = np.random.default_rng(86)
    geno = synth.multiallelic_genotypes(rng, 50, 40)
    expr = synth.expression_lognormal(rng, 10, 40)
    rs = kx.krux_rank(_dev(expr))
    with pytest.raises(k.KruxError) as e:  # codes 3, 4 need the flag
        kx.krux_scan(rs, _dev(geno), 1e-3, capacity=500)
    assert e.value.status == k.KRUX_EINVAL
    bad = geno.copy()
    bad[3, 3] = 5
    with pytest.raises(k.KruxError) as e:
        kx.krux_scan(rs, _dev(bad), 1e-3, capacity=500, multiallelic=True)
    assert e.value.status == k.KRUX_EINVAL
