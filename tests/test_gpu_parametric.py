"""Parametric comparison statistics on the same tiles (one-way ANOVA F and
dosage-regression t) through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import synth

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


def _check(res, orc, pth):
    h = res["hits"].cpu().numpy().astype(np.int64)
    stat = res["stat"].cpu().numpy()
    p = res["p"].cpu().numpy()
    got = np.zeros_like(orc["hit"])
    got[h[:, 0], h[:, 1]] = True
    band = np.abs(orc["p"] / pth - 1.0) < 1e-9
    diff = (got != orc["hit"]) & ~band
    assert not diff.any(), f"hit sets differ at {np.argwhere(diff)[:5].tolist()}"
    assert np.all(h[:, 2:] == 0)
    os_, op = orc["stat"][h[:, 0], h[:, 1]], orc["p"][h[:, 0], h[:, 1]]
    assert np.all(np.abs(stat - os_) <= 1e-6 * np.abs(os_)), "statistic differs"
    assert np.all(np.abs(p - op) <= 1e-6 * op), "p differs"
    assert res["n_hits"] == int(orc["hit"].sum())


@pytest.mark.parametrize("model", ["anova", "linear"])
@pytest.mark.parametrize("T,S,N,pth", [(150, 800, 102, 1e-3), (131, 555, 60, 1e-2)])
def test_parametric_scan(kx, oracle_mod, model, T, S, N, pth):
    d = synth.config(2, T=T, S=S, N=N, seed=T + S)
    geno = np.where(d["geno"] < 0, 0, d["geno"]).astype(np.int8)
    res = kx.krux_scan_parametric(_dev(d["expr"]), _dev(geno), model, pth, capacity=T * S)
    orc = oracle_mod.parametric_scan(d["expr"], geno, pth, model)
    assert orc["hit"].sum() > 0
    _check(res, orc, pth)


def test_parametric_rejects_nan_and_missing(kx):
    import paper_1307_3519_gb300 as k
    d = synth.config(1, T=10, S=60, seed=95)
    e = d["expr"].copy()
    e[2, 3] = np.nan
    with pytest.raises(k.KruxError) as err:
        kx.krux_scan_parametric(_dev(e), _dev(d["geno"]), "anova", 1e-3, capacity=100)
    assert err.value.status == k.KRUX_EINVAL
    g = d["geno"].copy()
    g[5, 5] = -1
    with pytest.raises(k.KruxError) as err:
        kx.krux_scan_parametric(_dev(d["expr"]), _dev(g), "linear", 1e-3, capacity=100)
    assert err.value.status == k.KRUX_EUNSUPPORTED
