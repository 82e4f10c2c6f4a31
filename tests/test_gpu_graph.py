"""CUDA-graph replays and the autotuner through the C ABI: a captured scan,
permutation batch and multi-cohort launch replayed on new inputs of the same
shapes give what the direct calls (and the FP64 oracle) give; inputs a replay
cannot scan are reported, not scanned."""
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


def _same(a, b):
    ha, Ha, pa = _sorted(a)
    hb, Hb, pb = _sorted(b)
    assert a["n_hits"] == b["n_hits"]
    assert np.array_equal(ha, hb)
    assert np.array_equal(Ha, Hb) and np.array_equal(pa, pb)


def test_graph_scan_replays_new_genotypes(kx, oracle_mod):
    d1 = synth.config(1, T=300, S=3000, seed=21)
    d2 = synth.config(1, T=300, S=3000, seed=22)
    pth = 1e-3
    rs = kx.krux_rank(_dev(d1["expr"]))
    g = _dev(d1["geno"])
    graph = kx.graph_scan(rs, g, pth, capacity=300 * 3000)
    for d in (d1, d2, d1):
        g.copy_(_dev(d["geno"]))
        graph.launch()
        got = graph.wait()[0]
        direct = kx.krux_scan(rs, g, pth, capacity=300 * 3000)
        _same(got, direct)
        orc = oracle_mod.scan(d1["expr"], d["geno"], pth)
        check_hits(got, orc, np.arange(300), np.arange(3000), pth)
    graph.close()


def test_graph_dense_output(kx, oracle_mod):
    d = synth.config(1, T=130, S=700, seed=23)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    graph = kx.graph_scan(rs, g, 1e-3, capacity=130 * 700, dense=True)
    graph.launch()
    graph.wait()
    direct = kx.krux_scan(rs, g, 1e-3, capacity=130 * 700, dense=True)
    assert np.array_equal(graph.dense[0].cpu().numpy(), direct["dense_H"].cpu().numpy())
    assert np.array_equal(graph.dense[1].cpu().numpy(), direct["dense_p"].cpu().numpy())
    graph.close()


@pytest.mark.parametrize("nan", [False, True])
def test_graph_permute_matches_direct(kx, oracle_mod, nan):
    T, S, P, N = 150, 1500, 3, 102
    d = synth.config(3 if nan else 4, T=T, S=S, N=N, seed=31)
    geno = np.where(d["geno"] < 0, 0, d["geno"]).astype(np.int8)
    perms = _dev(synth.make_perms(5, P, N))
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(geno)
    pth = 1e-3
    graph = kx.graph_permute(rs, g, perms, pth, capacity=T * S, fdr_bins=12, fdr_bin_width=0.25)
    for seed in (5, 6):
        perms.copy_(_dev(synth.make_perms(seed, P, N)))
        graph.launch()
        got = graph.wait()[0]
        direct = kx.krux_permute(rs, g, perms, pth, capacity=T * S, fdr_bins=12, fdr_bin_width=0.25)
        _same(got, direct)
        assert np.array_equal(graph.minp.cpu().numpy(), direct["minp"].cpu().numpy())
        assert np.array_equal(graph.fdr_hist.cpu().numpy(), direct["fdr_hist"].cpu().numpy())
        want = oracle_mod.perm_minp(d["expr"], geno, perms.cpu().numpy())
        gm = graph.minp.cpu().numpy()
        assert np.all(np.abs(gm - want) <= 1e-6 * want)
    graph.close()


def test_graph_permute_with_seed_pass(kx, oracle_mod):
    """More than 65,536 SNPs: the direct call and the graph both run the seed pass
    over the first 16,384 SNPs and the main launch back to back; their minima,
    hits and FDR histogram agree exactly, and the minima match the oracle."""
    T, S, P, N = 128, 70000, 4, 102
    d = synth.config(4, T=T, S=S, N=N, seed=41)
    perms = _dev(synth.make_perms(7, P, N))
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    pth = 1e-4
    graph = kx.graph_permute(rs, g, perms, pth, capacity=T * S, fdr_bins=10, fdr_bin_width=0.5)
    graph.launch()
    got = graph.wait()[0]
    direct = kx.krux_permute(rs, g, perms, pth, capacity=T * S, fdr_bins=10, fdr_bin_width=0.5)
    _same(got, direct)
    assert np.array_equal(graph.minp.cpu().numpy(), direct["minp"].cpu().numpy())
    assert np.array_equal(graph.fdr_hist.cpu().numpy(), direct["fdr_hist"].cpu().numpy())
    sel = np.arange(0, T, 8)
    want = oracle_mod.perm_minp(d["expr"][sel], d["geno"], perms.cpu().numpy())
    gm = direct["minp"].cpu().numpy()[:, sel]
    assert np.all(np.abs(gm - want) <= 1e-6 * want)
    graph.close()


def test_graph_grouped_cohorts(kx, oracle_mod):
    rng = np.random.default_rng(41)
    cohorts, data = [], []
    for n_c in (48, 102, 300):
        gn, _ = synth.hwe_genotypes(rng, 600, n_c, 0.05, 0.5)
        e = synth.expression_lognormal(rng, 140, n_c)
        data.append((e, gn))
        cohorts.append(dict(rs=kx.krux_rank(_dev(e)), geno=_dev(gn), capacity=140 * 600))
    pth = 1e-2
    graph = kx.graph_grouped(cohorts, pth)
    graph.launch()
    got = graph.wait()
    direct = kx.krux_scan_grouped(cohorts, pth)
    for (e, gn), a, b in zip(data, got, direct):
        _same(a, b)
        check_hits(a, oracle_mod.scan(e, gn, pth), np.arange(140), np.arange(600), pth)
    graph.close()


def test_graph_refuses_and_reports_missing_genotypes(kx):
    import paper_1307_3519_gb300 as k
    d = synth.config(1, T=64, S=500, seed=51)
    rs = kx.krux_rank(_dev(d["expr"]))
    bad = d["geno"].copy()
    bad[7, 3] = -1
    with pytest.raises(k.KruxError) as e:
        kx.graph_scan(rs, _dev(bad), 1e-3, capacity=64 * 500)
    assert e.value.status == k.KRUX_EUNSUPPORTED
    g = _dev(d["geno"])
    graph = kx.graph_scan(rs, g, 1e-3, capacity=64 * 500)
    g.copy_(_dev(bad))
    graph.launch()
    with pytest.raises(k.KruxError) as e:
        graph.wait()
    assert e.value.status == k.KRUX_EUNSUPPORTED
    graph.close()


def test_graph_replay_reports_out_of_range_permutation(kx):
    import paper_1307_3519_gb300 as k
    d = synth.config(4, T=64, S=400, seed=52)
    perms = _dev(synth.make_perms(9, 2, d["N"]))
    rs = kx.krux_rank(_dev(d["expr"]))
    graph = kx.graph_permute(rs, _dev(d["geno"]), perms, 1e-3, capacity=64 * 400)
    perms[1, 5] = d["N"] + 7  # outside 0..N-1: the gather reads zeros and reports it
    graph.launch()
    with pytest.raises(k.KruxError) as e:
        graph.wait()
    assert e.value.status == k.KRUX_EINVAL
    graph.close()


def test_autotune_picks_a_shape_and_scans_stay_exact(kx, oracle_mod):
    d = synth.config(1, T=400, S=5000, N=102, seed=61)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    shape = kx.autotune(rs, g, 1e-3)
    assert len(shape) == 4 and shape[0] in (-1, 0, 1)
    res = kx.krux_scan(rs, g, 1e-3, capacity=400 * 5000)
    check_hits(res, oracle_mod.scan(d["expr"], d["geno"], 1e-3), np.arange(400), np.arange(5000), 1e-3)
