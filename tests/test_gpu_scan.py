"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import synth
from kwcheck import check_dense, check_hits

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


# ---------------------------------------------------------------- rank transform
@pytest.mark.parametrize("T,N,decimals,nan", [(1, 1, 2, 0.0), (7, 5, 1, 0.0), (129, 60, 2, 0.0),
                                              (300, 102, None, 0.02), (40, 250, 1, 0.05),
                                              (33, 512, 0, 0.0), (16, 511, None, 0.3)])
def test_rank_bit_exact(kx, oracle_mod, T, N, decimals, nan):
    rng = np.random.default_rng(T * 1000 + N)
    x = rng.standard_normal((T, N))
    if decimals is not None:
        x = np.round(x, decimals)
    x = x.astype(np.float32)
    x[rng.random((T, N)) < nan] = np.nan
    if T > 3:
        x[0] = 1.5            # all tied
        x[1, : N // 2] = -0.0 # signed zeros tie with zeros
        x[1, N // 2:] = 0.0
    rs = kx.krux_rank(_dev(x))
    c, tie, K = (a.cpu().numpy() for a in kx.export(rs))
    for t in range(T):
        r2, otie, oK = oracle_mod.rank_row(x[t])
        assert K[t] == oK
        assert tie[t] == int(otie)
        ok = ~np.isnan(x[t])
        assert np.array_equal(c[t][ok], r2[ok] - (oK + 1)), f"trait {t}"
        assert np.all(c[t][~ok] == 0)


# ---------------------------------------------------------------- fused scan
def test_workload1_dense_and_hits(kx, oracle_mod):
    """Full 60-sample workload: every pair's H and p densely, plus the hit list."""
    d = synth.config(1)
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=200_000, dense=True)
    check_dense(res["dense_H"].cpu().numpy(), res["dense_p"].cpu().numpy(), orc)
    check_hits(res, orc, np.arange(d["T"]), np.arange(d["S"]), d["pthresh"])
    res2 = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=200_000)
    check_hits(res2, orc, np.arange(d["T"]), np.arange(d["S"]), d["pthresh"])
    assert res2["n_hits"] == res["n_hits"] == int(orc["hit"].sum())


@pytest.mark.parametrize("N,T,S,pth", [(5, 3, 1, 0.3), (17, 129, 65, 0.05), (33, 200, 300, 0.02),
                                       (60, 257, 1000, 1e-3), (102, 300, 2500, 1e-3),
                                       (150, 131, 700, 1e-3), (200, 128, 640, 1e-2),
                                       (256, 100, 333, 1e-2), (300, 129, 300, 1e-2),
                                       (400, 64, 200, 1e-2), (512, 33, 150, 1e-2)])
def test_scan_hits_ragged(kx, oracle_mod, N, T, S, pth):
    d = synth.config(2, T=T, S=S, N=N, seed=7 * N + S)
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=T * S)
    check_hits(res, orc, np.arange(T), np.arange(S), pth, must_have_hits=False)
    assert res["n_hits"] == int(orc["hit"].sum())


def test_plain_form_matches(kx, oracle_mod):
    d = synth.config(2, T=300, S=3000, seed=11)
    pth = 1e-3
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    a = kx.krux_scan(rs, g, pth, capacity=300 * 3000)
    b = kx.krux_scan_plain(rs, g, pth, capacity=300 * 3000)
    check_hits(a, orc, np.arange(300), np.arange(3000), pth)
    check_hits(b, orc, np.arange(300), np.arange(3000), pth)
    bd = kx.krux_scan_plain(rs, g, pth, capacity=300 * 3000, dense=True)
    check_dense(bd["dense_H"].cpu().numpy(), bd["dense_p"].cpu().numpy(), orc)


def test_slices_and_overflow(kx, oracle_mod):
    d = synth.config(1, T=100, S=900, seed=5)
    pth = 0.02
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    total = int(orc["hit"].sum())
    assert total > 50
    parts = []
    for b, e in [(0, 130), (130, 131), (131, 900)]:
        r = kx.krux_scan(rs, g, pth, capacity=100 * 900, snp_begin=b, snp_end=e)
        sub = {k: v[:, b:e] for k, v in orc.items()}
        check_hits(r, sub, np.arange(100), np.arange(b, e), pth, must_have_hits=False)
        parts.append(r["n_hits"])
    assert sum(parts) == total
    small = kx.krux_scan(rs, g, pth, capacity=10)
    assert small["overflow"] and small["n_hits"] == total and small["hits"].shape[0] == 10
    zero = kx.krux_scan(rs, g, pth, capacity=0)
    assert zero["n_hits"] == total


def test_hits_past_the_staging_segments(kx, oracle_mod):
    """Many hits per warp and a capacity of a third of them: each warp's staging
    segment (sized from the capacity) holds about half of its hits, so the rest go
    to the list through the global counter and the list ends up mixed.  The count
    stays exact and every record kept must be an oracle hit with exact rank sums
    and FP64 H and p."""
    from kwcheck import gpu_hits_np, H_RTOL, H_ATOL, P_RTOL
    d = synth.config(2, T=256, S=4000, seed=12)
    pth = 0.05
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    total = int(orc["hit"].sum())
    assert total > 20000
    rs = kx.krux_rank(_dev(d["expr"]))
    cap = total // 3
    res = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=cap)
    assert res["overflow"] and res["n_hits"] == total and res["hits"].shape[0] == cap
    h, H, p = gpu_hits_np(res)
    t, snp = h[:, 0], h[:, 1]
    assert len(set(zip(t.tolist(), snp.tolist()))) == cap, "duplicate records"
    assert orc["hit"][t, snp].all(), "a record that is not a hit"
    assert np.array_equal(h[:, 2], orc["d"][t, snp, 0]) and np.array_equal(h[:, 3], orc["d"][t, snp, 1])
    oh, op = orc["H"][t, snp], orc["p"][t, snp]
    assert np.all(np.abs(H - oh) <= H_RTOL * np.abs(oh) + H_ATOL)
    assert np.all(np.abs(p - op) <= P_RTOL * op)


def test_degenerate_inputs(kx, oracle_mod):
    """Monomorphic SNPs, all-tied traits, a single sample group and S = 0."""
    d = synth.config(1, T=40, S=200, seed=3)
    x, g = d["expr"].copy(), d["geno"].copy()
    x[0] = 0.25
    x[1, :] = np.arange(60, dtype=np.float32)
    g[0] = 1
    g[1] = 0
    g[2, :30] = 2
    g[2, 30:] = 0
    pth = 0.05
    orc = oracle_mod.scan(x, g, pth)
    rs = kx.krux_rank(_dev(x))
    res = kx.krux_scan(rs, _dev(g), pth, capacity=40 * 200, dense=True)
    check_dense(res["dense_H"].cpu().numpy(), res["dense_p"].cpu().numpy(), orc)
    check_hits(res, orc, np.arange(40), np.arange(200), pth)
    empty = kx.krux_scan(rs, _dev(g[:0]), pth, capacity=10)
    assert empty["n_hits"] == 0


def test_bad_genotype_code(kx):
    import paper_1307_3519_gb300 as k
    d = synth.config(1, T=10, S=20, seed=1)
    g = d["geno"].copy()
    g[5, 7] = 3
    rs = kx.krux_rank(_dev(d["expr"]))
    with pytest.raises(k.KruxError) as e:
        kx.krux_scan(rs, _dev(g), 0.01, capacity=100)
    assert e.value.status == k.KRUX_EINVAL


def test_nan_expression(kx, oracle_mod):
    d = synth.config(2, T=260, S=1500, seed=21)
    x = d["expr"].copy()
    rng = np.random.default_rng(4)
    x[rng.random(x.shape) < 0.02] = np.nan
    x[3, :90] = np.nan          # a trait with many missing values
    x[4, :101] = np.nan         # one present sample: degenerate
    pth = 1e-3
    orc = oracle_mod.scan(x, d["geno"], pth)
    rs = kx.krux_rank(_dev(x))
    res = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=260 * 1500)
    check_hits(res, orc, np.arange(260), np.arange(1500), pth)
    dn = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=260 * 1500, dense=True)
    check_dense(dn["dense_H"].cpu().numpy(), dn["dense_p"].cpu().numpy(), orc)


@pytest.mark.parametrize("with_missing_geno", [False, True])
def test_nan_counts_per_trait(kx, oracle_mod, with_missing_geno):
    """Traits with 0..20 NaN samples (trait t has t mod 21): up to 15 per trait
    the hot test works on each pair's exact group sizes, beyond that every pair
    takes the rare path; with missing-genotype patterns the buckets' re-ranked
    sets carry the same NaN lists.  The hit set must be the oracle's, so that a
    hot test that drops a true hit fails here."""
    d = synth.config(2, T=168, S=2100, seed=33)
    x = d["expr"].copy()
    g = d["geno"].copy()
    rng = np.random.default_rng(9)
    for t in range(x.shape[0]):
        x[t, rng.choice(x.shape[1], t % 21, replace=False)] = np.nan
    if with_missing_geno:
        synth.add_missing_genotypes(rng, g, snp_frac=0.2, n_patterns=12, per_pattern=3)
    pth = 2e-3
    orc = oracle_mod.scan(x, g, pth)
    rs = kx.krux_rank(_dev(x))
    res = kx.krux_scan(rs, _dev(g), pth, capacity=168 * 2100)
    check_hits(res, orc, np.arange(168), np.arange(2100), pth)


@pytest.mark.parametrize("with_missing_geno", [False, True])
def test_nan_plain_form_variant(kx, oracle_mod, with_missing_geno):
    """The plain form's NaN variant: traits with 0..6 NaN samples (trait t has t
    mod 7) take the coefficient set of their count, and three traits have more (9,
    30, and 101 of 102: degenerate), so that every pair of theirs reaches the exact
    test with its exact group sizes.  Nine trait tiles (the last ragged); three
    traits in 1030 beyond the sets: the call takes form 5, and its hit set must be
    the oracle's."""
    d = synth.config(2, T=1030, S=2100, seed=35)
    x = d["expr"].copy()
    g = d["geno"].copy()
    rng = np.random.default_rng(11)
    for t in range(x.shape[0]):
        c = {5: 9, 6: 30, 13: 101}.get(t, t % 7)
        x[t, rng.choice(x.shape[1], c, replace=False)] = np.nan
    if with_missing_geno:
        synth.add_missing_genotypes(rng, g, snp_frac=0.2, n_patterns=12, per_pattern=3)
    pth = 2e-3
    orc = oracle_mod.scan(x, g, pth)
    import paper_1307_3519_gb300 as k
    ctx = k.Krux(0)
    ctx.set_profiling(True)
    rs = ctx.krux_rank(_dev(x))
    res = ctx.krux_scan(rs, _dev(g), pth, capacity=1030 * 2100)
    assert ctx.profile()["scan_form"] == 5
    check_hits(res, orc, np.arange(1030), np.arange(2100), pth)
    ctx.close()


@pytest.mark.parametrize("N", [60, 150, 250])
def test_nan_expression_other_widths(kx, oracle_mod, N):
    """NaN expression at other sample counts: the NaN variant of the plain form where
    its coefficient sets fit shared memory beside the wider operands, the general
    form where they do not (the plan is made again); the hit set is the oracle's
    either way."""
    d = synth.config(2, T=260, S=1400, N=N, seed=40 + N)
    x = d["expr"].copy()
    rng = np.random.default_rng(N)
    x[rng.random(x.shape) < 0.015] = np.nan
    pth = 2e-3
    orc = oracle_mod.scan(x, d["geno"], pth)
    import paper_1307_3519_gb300 as k
    ctx = k.Krux(0)
    ctx.set_profiling(True)
    rs = ctx.krux_rank(_dev(x))
    res = ctx.krux_scan(rs, _dev(d["geno"]), pth, capacity=260 * 1400)
    assert ctx.profile()["scan_form"] in (3, 5)
    check_hits(res, orc, np.arange(260), np.arange(1400), pth)
    ctx.close()


def test_missing_genotypes(kx, oracle_mod):
    """Missing-value workload at reduced size: -1 genotypes in missing-sample
    patterns and NaN expression; ranks over the samples present in both."""
    d = synth.config(3, T=300, S=4000)
    pth = 1e-3
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=300 * 4000)
    check_hits(res, orc, np.arange(300), np.arange(4000), pth)
    dn = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=300 * 4000, dense=True)
    check_dense(dn["dense_H"].cpu().numpy(), dn["dense_p"].cpu().numpy(), orc)


def _as_res(out):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(out[k])) for k in ("hits", "H", "p")}


def test_host_end_to_end(kx, oracle_mod):
    d = synth.config(1, T=50, S=400, seed=8)
    out = kx.krux_scan_host(d["expr"], d["geno"], 0.01, capacity=50 * 400)
    orc = oracle_mod.scan(d["expr"], d["geno"], 0.01)
    assert out["n_hits"] == int(orc["hit"].sum())
    check_hits(_as_res(out), orc, np.arange(50), np.arange(400), 0.01)


def test_host_entry_strided_pinned_missing(kx, oracle_mod):
    """krux_scan_host on page-locked host buffers whose leading dimensions exceed
    N (the 2-D copies), with missing genotypes and NaN expression, against the
    oracle; then a capacity below the hit count: KRUX_EOVERFLOW, the exact count
    and real hit records."""
    import torch
    d = synth.config(3, T=300, S=4000, seed=21)
    T, S, N = d["expr"].shape[0], d["geno"].shape[0], d["expr"].shape[1]
    pth = 1e-3
    e_h = torch.zeros((T, N + 5), dtype=torch.float32).pin_memory()
    g_h = torch.zeros((S, N + 3), dtype=torch.int8).pin_memory()
    e_h[:, :N] = torch.from_numpy(d["expr"])
    g_h[:, :N] = torch.from_numpy(d["geno"])
    out = kx.krux_scan_host(e_h[:, :N], g_h[:, :N], pth, capacity=T * S)
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    assert not out["overflow"] and out["n_hits"] == out["hits"].shape[0]
    check_hits(_as_res(out), orc, np.arange(T), np.arange(S), pth)
    cap = out["n_hits"] // 3
    small = kx.krux_scan_host(d["expr"], d["geno"], pth, capacity=cap)
    assert small["overflow"] and small["n_hits"] == out["n_hits"] and small["hits"].shape[0] == cap
    key = lambda h: h[:, 0].astype(np.int64) * S + h[:, 1]
    full = dict(zip(key(out["hits"]).tolist(), map(tuple, out["hits"].tolist())))
    assert all(full[k_] == tuple(r) for k_, r in zip(key(small["hits"]).tolist(), small["hits"].tolist()))
    # page-locked outputs: the kernels write them directly; the same records
    n = out["n_hits"]
    outs = (torch.zeros((n, 4), dtype=torch.int32).pin_memory(),
            torch.zeros(n, dtype=torch.float64).pin_memory(), torch.zeros(n, dtype=torch.float64).pin_memory())
    pin = kx.krux_scan_host(e_h[:, :N], g_h[:, :N], pth, capacity=n, out=outs)
    assert not pin["overflow"] and pin["n_hits"] == n
    a, b = np.argsort(key(pin["hits"])), np.argsort(key(out["hits"]))
    assert np.array_equal(pin["hits"][a], out["hits"][b])
    assert np.array_equal(pin["H"][a], out["H"][b]) and np.array_equal(pin["p"][a], out["p"][b])
    # and past their capacity: the exact count, real records
    outs2 = tuple(t[: n // 2] for t in outs)
    pin2 = kx.krux_scan_host(e_h[:, :N], g_h[:, :N], pth, capacity=n // 2, out=outs2)
    assert pin2["overflow"] and pin2["n_hits"] == n
    assert all(full[k_] == tuple(r) for k_, r in zip(key(pin2["hits"]).tolist(), pin2["hits"].tolist()))


def test_host_entry_large_with_missing(kx, oracle_mod):
    """krux_scan_host at 300,000 SNPs with missing genotypes (196-odd pattern
    buckets) and NaN expression: the same hit set, rank sums, H and p as the
    device-side krux_scan on the same inputs, the oracle's on sampled traits, and
    with a capacity below the hit count KRUX_EOVERFLOW, the exact count and real
    records."""
    import torch
    d = synth.config(3, T=256, S=300000, seed=23)
    x, g = d["expr"], d["geno"]
    T, S = x.shape[0], g.shape[0]
    pth = 1e-4
    out = kx.krux_scan_host(x, g, pth, capacity=T * 2000)
    assert not out["overflow"] and out["n_hits"] > 0
    rs = kx.krux_rank(_dev(x))
    ref = kx.krux_scan(rs, _dev(g), pth, capacity=T * 2000)
    rs.free()
    key = lambda h: h[:, 0].astype(np.int64) * S + h[:, 1]
    a = np.argsort(key(out["hits"]))
    rh = ref["hits"].cpu().numpy()
    b = np.argsort(key(rh))
    assert out["n_hits"] == ref["n_hits"]
    assert np.array_equal(out["hits"][a], rh[b])
    assert np.array_equal(out["H"][a], ref["H"].cpu().numpy()[b])
    assert np.array_equal(out["p"][a], ref["p"].cpu().numpy()[b])
    sel = np.arange(0, T, 37)
    orc = oracle_mod.scan(x[sel], g, pth)
    check_hits(_as_res(out), orc, sel, np.arange(S), pth)
    cap = out["n_hits"] // 3
    small = kx.krux_scan_host(x, g, pth, capacity=cap)
    assert small["overflow"] and small["n_hits"] == out["n_hits"] and small["hits"].shape[0] == cap
    full = dict(zip(key(out["hits"]).tolist(), map(tuple, out["hits"].tolist())))
    assert all(full[k_] == tuple(r) for k_, r in zip(key(small["hits"]).tolist(), small["hits"].tolist()))


@pytest.mark.parametrize("layout,nc,nA,ka", [(0, 0, 0, 0), (1, 0, 0, 0), (1, 2, 4, 0), (0, 3, 3, 0),
                                             (1, 1, 2, 0), (1, 4, 2, 0), (1, 2, 4, 64), (0, 2, 3, 64),
                                             (1, 1, 4, 64), (1, 4, 3, 64)])
@pytest.mark.parametrize("N", [60, 102, 150])
def test_tile_shapes(kx, oracle_mod, layout, nc, nA, ka, N):
    """Every shared-memory layout and pipeline shape the tuner may pick (whole-K
    rank stages or K blocks of 64 samples) gives the oracle's hit set and exact
    rank sums."""
    import paper_1307_3519_gb300 as k
    d = synth.config(2, T=270, S=1300, N=N, seed=N + 3 * nc + layout)
    pth = 2e-3
    orc = oracle_mod.scan(d["expr"], d["geno"], pth)
    rs = kx.krux_rank(_dev(d["expr"]))
    kx.set_tuning(layout, nc, nA, ka)
    try:
        res = kx.krux_scan(rs, _dev(d["geno"]), pth, capacity=270 * 1300)
    except k.KruxError as e:
        kx.set_tuning(-1, 0, 0, 0)
        assert e.status == k.KRUX_EINVAL  # shape does not fit this N
        return
    finally:
        kx.set_tuning(-1, 0, 0, 0)
    check_hits(res, orc, np.arange(270), np.arange(1300), pth, must_have_hits=False)
    assert res["n_hits"] == int(orc["hit"].sum())


@pytest.mark.parametrize("window", [0, 200_000, 1_000_000, 1 << 50])
def test_cis_scan(kx, oracle_mod, window):
    """cis scan: the hits of the full scan within the window, nothing else; the
    work is pruned to the trait tiles the window reaches."""
    import synth as sy
    T, S = 300, 4000
    d = sy.config(2, T=T, S=S, seed=71)
    snp_pos, trait_pos = sy.genome_positions(np.random.default_rng(72), S, T, n_chrom=2,
                                             chrom_len=4_000_000)
    rs = kx.krux_rank(_dev(d["expr"]))
    g = _dev(d["geno"])
    res = kx.krux_scan_cis(rs, g, _dev(snp_pos), _dev(trait_pos), window, 1e-4, capacity=T * S)
    orc = oracle_mod.scan_cis(d["expr"], d["geno"], 1e-4, snp_pos, trait_pos, window)
    check_hits(res, orc, np.arange(T), np.arange(S), 1e-4, must_have_hits=False)
    assert res["n_hits"] == int(orc["hit"].sum())


def test_cis_scan_rejects_unsorted_coordinates(kx):
    import paper_1307_3519_gb300 as k
    import synth as sy
    d = sy.config(1, T=20, S=100, seed=73)
    snp_pos, trait_pos = sy.genome_positions(np.random.default_rng(74), 100, 20)
    snp_pos[3] = snp_pos[4] + 5  # no longer nondecreasing
    rs = kx.krux_rank(_dev(d["expr"]))
    with pytest.raises(k.KruxError) as e:
        kx.krux_scan_cis(rs, _dev(d["geno"]), _dev(snp_pos), _dev(trait_pos), 1000, 1e-3, capacity=10)
    assert e.value.status == k.KRUX_EINVAL
