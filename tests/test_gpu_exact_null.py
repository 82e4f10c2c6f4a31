"""The CUDA path over the exact permutation distribution at N <= 8, and SNP
shards of one call merged on the host.

Exhaustive null: for a sample of K = 7 or 8 values (with ties) and a genotype
labelling with 2 or 3 groups, all K! relabellings are scanned densely through
krux_rank + krux_scan, once as K! permuted genotype rows against the one trait
and once as K! permuted expression rows against the one marker.  The GPU's H
must equal the oracle's pair by pair (hence as a multiset) to 1e-12 relative,
and its mean over the K! relabellings must be k - 1 (k non-empty groups), the
exact expectation of the tie-corrected statistic under the permutation null
(section "P-value calculation and empirical FDR correction" relies on that null).

Shards (section "Data slicing": a slice of markers is an independent job): a
scan and a permutation batch run over two SNP slices one after the other must
merge (hit lists concatenated, min-p tables by element-wise minimum) into exactly
the unsharded call's results."""
import itertools

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

CASES = [
    ([0.5, 0.5, 0.5, 2, 3, 3, 7], [0, 0, 1, 1, 1, 2, 2]),
    ([4, 1, 1, 2, 9, 9, 9, 3], [0, 1, 1, 1, 2, 2, 0, 0]),
    ([5, 3, 3, 1, 8, 2, 2, 2], [0, 0, 0, 2, 2, 2, 2, 2]),
    ([1, 2, 2, 3, 4, 4, 4, 5], [0, 0, 0, 1, 1, 1, 1, 0]),
]


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


def _dense(kx, expr, geno, pth):
    rs = kx.krux_rank(_dev(expr))
    r = kx.krux_scan(rs, _dev(geno), pth, capacity=expr.shape[0] * geno.shape[0], dense=True)
    rs.free()
    return r["dense_H"].cpu().numpy(), r["dense_p"].cpu().numpy(), r


def _close(a, b):
    return np.all(np.abs(a - b) <= 1e-12 * np.abs(b) + 1e-12)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_exhaustive_relabellings(kx, oracle_mod, case):
    x, g = CASES[case]
    x = np.array(x, dtype=np.float32)
    g = np.array(g, dtype=np.int8)
    K = x.size
    k = np.unique(g).size
    perms = np.array(list(itertools.permutations(range(K))), dtype=np.int64)
    pth = 0.05
    # K! genotype rows against one trait
    geno = np.ascontiguousarray(g[perms])
    H, p, r = _dense(kx, x[None, :], geno, pth)
    orc = oracle_mod.scan(x[None, :], geno, pth)
    assert _close(H, orc["H"]) and _close(p, orc["p"])
    assert _close(np.sort(H[0]), np.sort(orc["H"][0]))  # the multiset
    assert H[0].mean() == pytest.approx(k - 1, rel=1e-12)
    assert r["n_hits"] == int(orc["hit"].sum())
    # K! expression rows (ranked on the GPU) against the marker and a relabelled copy
    expr = np.ascontiguousarray(x[perms])
    geno2 = np.stack([g, g[::-1]]).astype(np.int8)
    H2, p2, r2 = _dense(kx, expr, geno2, pth)
    orc2 = oracle_mod.scan(expr, geno2, pth)
    assert _close(H2, orc2["H"]) and _close(p2, orc2["p"])
    for j in range(2):
        assert H2[:, j].mean() == pytest.approx(k - 1, rel=1e-12)
    # the two orientations give the same multiset (relabelling samples of the
    # trait or of the marker is the same permutation group)
    assert _close(np.sort(H2[:, 0]), np.sort(H[0]))
    assert r2["n_hits"] == int(orc2["hit"].sum())


def _hits_np(r, offset=0):
    h = r["hits"].cpu().numpy().astype(np.int64)
    h[:, 1] += offset
    return h, r["H"].cpu().numpy(), r["p"].cpu().numpy()


def test_snp_shards_merge_to_the_unsharded_call(kx):
    from paper_1307_3519_gb300 import shard
    d = synth.config(4, T=2000, S=80000, seed=77)
    S = d["S"]
    pth = d["pthresh"]
    rs = kx.krux_rank(_dev(d["expr"]))
    geno = _dev(d["geno"])
    perms = _dev(d["perms"])
    cap = 5_000_000
    # the fused scan: whole call vs two slices given by snp_begin / snp_end
    whole = shard.merge_hits([_hits_np(kx.krux_scan(rs, geno, pth, capacity=cap))])
    parts = []
    for w in range(2):
        b, e = shard.shard_bounds(S, w, 2)
        parts.append(_hits_np(kx.krux_scan(rs, geno, pth, capacity=cap, snp_begin=b, snp_end=e)))
    merged = shard.merge_hits(parts)
    assert whole[0].shape[0] > 0
    for a, b in zip(whole, merged):
        assert np.array_equal(a, b)
    # the permutation batch: whole call (80,000 SNPs, with its seed pass) vs the
    # two shards' own calls on their row slices
    r = kx.krux_permute(rs, geno, perms, pth, capacity=cap)
    whole_minp = r["minp"].cpu().numpy()
    whole_hits = shard.merge_hits([_hits_np(r)])
    mins, hparts = [], []
    for w in range(2):
        b, e = shard.shard_bounds(S, w, 2)
        rp = kx.krux_permute(rs, geno[b:e], perms, pth, capacity=cap)
        mins.append(rp["minp"].cpu().numpy())
        hparts.append(_hits_np(rp, offset=b))
    assert np.array_equal(shard.merge_minp(mins), whole_minp)
    for a, b in zip(whole_hits, shard.merge_hits(hparts)):
        assert np.array_equal(a, b)
    rs.free()
