"""Parity at the full workload sizes, in the configuration bench.py times.

The CUDA path scans each full workload; the FP64 oracle recomputes, one pair
at a time, every SNP of a sample of traits (traits with and without hits), and
the hit sets, exact rank sums and FP64 H / p of those traits must agree."""
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


def _restrict(res, traits):
    """GPU hit list restricted to `traits` (as a result dict check_hits takes)."""
    h = res["hits"]
    import torch
    sel = torch.isin(h[:, 0].long(), torch.as_tensor(traits, device=h.device))
    return dict(hits=h[sel], H=res["H"][sel], p=res["p"][sel])


def _sample_traits(res, T, rng, n_hit=3, n_other=2):
    counts = np.bincount(res["hits"][:, 0].cpu().numpy(), minlength=T)
    with_hits = np.nonzero(counts)[0]
    pick = list(rng.choice(with_hits, size=min(n_hit, with_hits.size), replace=False))
    pick += list(rng.choice(np.nonzero(counts == 0)[0], size=n_other, replace=False))
    return np.sort(np.array(pick, dtype=np.int64))


def test_paper_scale_workload(kx, oracle_mod):
    """20,000 traits x 500,000 SNPs x 102 samples, hits at p < 1e-5."""
    d = synth.config(2)
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=50_000_000)
    assert not res["overflow"] and res["n_hits"] > 0
    traits = _sample_traits(res, d["T"], np.random.default_rng(2))
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"], traits=traits)
    check_hits(_restrict(res, traits), orc, traits, np.arange(d["S"]), d["pthresh"])


def test_missing_value_workload(kx, oracle_mod):
    """5,000 traits x 100,000 SNPs with missing-genotype patterns and NaN expression."""
    d = synth.config(3)
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=10_000_000)
    assert not res["overflow"]
    traits = _sample_traits(res, d["T"], np.random.default_rng(3))
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"], traits=traits)
    check_hits(_restrict(res, traits), orc, traits, np.arange(d["S"]), d["pthresh"])


def test_permutation_workload(kx, oracle_mod):
    """20,000 traits x 200,000 SNPs, 16 permutations: per-permutation minimum p of
    sampled traits and the unpermuted hits."""
    d = synth.config(4)
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_permute(rs, _dev(d["geno"]), _dev(d["perms"]), d["pthresh"], capacity=50_000_000)
    assert not res["overflow"]
    traits = _sample_traits(res, d["T"], np.random.default_rng(4), n_hit=2, n_other=1)
    want = oracle_mod.perm_minp(d["expr"], d["geno"], d["perms"], traits=traits)
    got = res["minp"].cpu().numpy()[:, traits]
    assert np.all(np.abs(got - want) <= 1e-6 * want), f"max rel err {np.max(np.abs(got - want) / want)}"
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"], traits=traits)
    check_hits(_restrict(res, traits), orc, traits, np.arange(d["S"]), d["pthresh"])


def test_multi_cohort_workload(kx, oracle_mod):
    """8 cohorts (N = 48 .. 500), 15,000 traits x 300,000 SNPs each, in one
    grouped persistent launch; hits at p < 1e-5."""
    d = synth.config(5)
    cohorts = []
    for c in d["cohorts"]:
        cohorts.append(dict(rs=kx.krux_rank(_dev(c["expr"])), geno=_dev(c["geno"]), capacity=5_000_000))
    out = kx.krux_scan_grouped(cohorts, d["pthresh"])
    rng = np.random.default_rng(5)
    for c, res in zip(d["cohorts"], out):
        assert not res["overflow"]
        traits = np.sort(rng.choice(d["T"], size=2, replace=False))
        orc = oracle_mod.scan(c["expr"], c["geno"], d["pthresh"], traits=traits)
        check_hits(_restrict(res, traits), orc, traits, np.arange(d["S"]), d["pthresh"],
                   must_have_hits=False)
        assert res["n_hits"] > 0
