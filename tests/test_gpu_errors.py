"""Largest relative error of the reported H and p against the FP64 oracle, per
workload (at sizes the oracle covers completely), printed and bounded by 1e-6.

Workloads 1 and 3 compare every pair through the dense output, the others every
reported hit; workload 4 also compares the per-(permutation, trait) minimum p."""
import numpy as np
import pytest

import synth
from kwcheck import gpu_hits_np

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


def _rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nz = b != 0
    return float(np.max(np.abs(a[nz] - b[nz]) / np.abs(b[nz]))) if nz.any() else 0.0


def _hit_errors(res, orc):
    h, H, p = gpu_hits_np(res)
    oh, op = orc["H"][h[:, 0], h[:, 1]], orc["p"][h[:, 0], h[:, 1]]
    return _rel(H, oh), _rel(p, op), h.shape[0]


def _report(name, eH, ep, n):
    print(f"\nerrors {name}: H max rel {eH:.2e}, p max rel {ep:.2e} over {n} pairs")
    assert eH <= 1e-6 and ep <= 1e-6


def test_errors_plain_dense(kx, oracle_mod):
    d = synth.config(1)
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=d["T"] * d["S"], dense=True)
    dH, dp = res["dense_H"].cpu().numpy(), res["dense_p"].cpu().numpy()
    big = orc["H"] > 1e-3  # the oracle's Eq. 2 form cancels for tiny H (absolute 1e-10 there)
    _report("workload 1 (all pairs, dense)", _rel(dH[big], orc["H"][big]), _rel(dp, orc["p"]),
            dH.size)


def test_errors_paper_scale_generator(kx, oracle_mod):
    d = synth.config(2, T=256, S=20000)
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=d["T"] * d["S"])
    _report("workload 2 (hits)", *_hit_errors(res, orc))


def test_errors_missing_values_dense(kx, oracle_mod):
    d = synth.config(3, T=300, S=4000)
    orc = oracle_mod.scan(d["expr"], d["geno"], d["pthresh"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_scan(rs, _dev(d["geno"]), d["pthresh"], capacity=d["T"] * d["S"], dense=True)
    dH, dp = res["dense_H"].cpu().numpy(), res["dense_p"].cpu().numpy()
    big = orc["H"] > 1e-3
    _report("workload 3 (all pairs, dense)", _rel(dH[big], orc["H"][big]), _rel(dp, orc["p"]),
            dH.size)


def test_errors_permutations(kx, oracle_mod):
    d = synth.config(4, T=200, S=3000)
    perms = synth.make_perms(1307, 4, d["N"])
    rs = kx.krux_rank(_dev(d["expr"]))
    res = kx.krux_permute(rs, _dev(d["geno"]), _dev(perms), 1e-3, capacity=d["T"] * d["S"])
    orc = oracle_mod.scan(d["expr"], d["geno"], 1e-3)
    eH, ep, n = _hit_errors(res, orc)
    _report("workload 4 (unpermuted hits)", eH, ep, n)
    want = oracle_mod.perm_minp(d["expr"], d["geno"], perms)
    got = res["minp"].cpu().numpy()
    e = _rel(got, want)
    print(f"errors workload 4 (minimum p of {got.size} permutation-trait pairs): max rel {e:.2e}")
    assert e <= 1e-6


def test_errors_cohorts(kx, oracle_mod):
    rng = np.random.default_rng(11)
    cohorts, data = [], []
    for n_c in (48, 150, 500):
        g, _ = synth.hwe_genotypes(rng, 600, n_c, 0.05, 0.5)
        e = synth.expression_lognormal(rng, 100, n_c)
        data.append((e, g))
        cohorts.append(dict(rs=kx.krux_rank(_dev(e)), geno=_dev(g), capacity=100 * 600))
    out = kx.krux_scan_grouped(cohorts, 1e-2)
    eH = ep = 0.0
    n = 0
    for (e, g), res in zip(data, out):
        a, b, k = _hit_errors(res, oracle_mod.scan(e, g, 1e-2))
        eH, ep, n = max(eH, a), max(ep, b), n + k
    _report("workload 5 (cohorts N = 48, 150, 500; hits)", eH, ep, n)
