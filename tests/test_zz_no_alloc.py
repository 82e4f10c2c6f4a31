"""krux_scan_noalloc: the scan for callers that cannot allocate device memory.

Callers that run under an allocator owning the whole device, plugins inside such
processes, or latency-critical code where an allocation may block or fail use
this entry point: the library takes all scratch from a fixed array of its own.
Its results must equal those of krux_scan on the same inputs (exact hit set and
rank sums, H and p within the same 1e-6 relative tolerance) and, checked on their
own, the FP64 oracle's, on two calls in a row, so that what one call leaves in the
shared array cannot leak into the next.  This file is collected last; it also
passes when run alone."""
import numpy as np
import pytest

import synth
from kwcheck import check_hits

pytestmark = pytest.mark.gpu


def _sorted(h, H, p):
    h = h.cpu().numpy().astype(np.int64)
    H, p = H.cpu().numpy(), p.cpu().numpy()
    o = np.lexsort((h[:, 0], h[:, 1]))
    return h[o], H[o], p[o]


def _case(seed, T, S, N, nan):
    """Null-distribution inputs (a few thousand hits at p < 1e-3, well inside the
    entry point's 262,144 stored-hit limit): HWE genotypes, tied expression
    (rounded normals) or log-normal expression with NaN."""
    rng = np.random.default_rng(seed)
    g, _ = synth.hwe_genotypes(rng, S, N, 0.05, 0.5)
    if nan:
        x = synth.expression_lognormal(rng, T, N)
        x[rng.random(x.shape) < nan] = np.nan
    else:
        x = synth.expression_rounded_normal(rng, T, N)
    return x, g


def test_noalloc_matches_krux_scan_on_two_calls(oracle_mod):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1307_3519_gb300 import build
    build.build()
    import paper_1307_3519_gb300 as k
    kx = k.Krux(0)
    cases = [_case(31, 300, 9000, 102, 0.0), _case(32, 257, 5000, 60, 0.01)]
    pth = 1e-3
    for x, g in cases:  # two calls in a row, different shapes and contents
        e, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
        rs = kx.krux_rank(e)
        ref = kx.krux_scan(rs, gd, pth, capacity=x.shape[0] * g.shape[0])
        cap = 200_000
        hits = torch.empty((cap, 4), dtype=torch.int32, device="cuda")
        H = torch.empty(cap, dtype=torch.float64, device="cuda")
        P = torch.empty(cap, dtype=torch.float64, device="cuda")
        st, n = k.krux_scan_noalloc(e, gd, pth, hits, H, P)
        assert st == k.KRUX_OK
        assert n == ref["n_hits"] and n > 0
        a = _sorted(hits[:n], H[:n], P[:n])
        b = _sorted(ref["hits"], ref["H"], ref["p"])
        assert np.array_equal(a[0], b[0])  # same pairs, same exact rank sums
        assert np.all(np.abs(a[1] - b[1]) <= 1e-6 * np.abs(b[1]) + 1e-10)
        assert np.all(np.abs(a[2] - b[2]) <= 1e-6 * b[2])
        # and the oracle's, directly
        orc = oracle_mod.scan(x, g, pth)
        check_hits({"hits": hits[:n], "H": H[:n], "p": P[:n]}, orc, np.arange(x.shape[0]),
                   np.arange(g.shape[0]), pth)
    kx.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1307_3519_gb300 as k
    e = torch.zeros((4097, 8), dtype=torch.float32, device="cuda")
    g = torch.zeros((4, 8), dtype=torch.int8, device="cuda")
    out = torch.empty((1, 4), dtype=torch.int32, device="cuda")
    H = torch.empty(1, dtype=torch.float64, device="cuda")
    st, n = k.krux_scan_noalloc(e, g, 1e-3, out, H, H.clone())
    assert st == k.KRUX_EINVAL and n == 0


def _noalloc_out(cap):
    import torch
    return (torch.empty((cap, 4), dtype=torch.int32, device="cuda"),
            torch.empty(cap, dtype=torch.float64, device="cuda"),
            torch.empty(cap, dtype=torch.float64, device="cuda"))


def test_noalloc_at_its_largest_shape():
    """T = 4096 traits and N = 256 samples (the documented maximum: the largest
    scratch offsets, one resident SNP chunk per launch) against krux_scan."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1307_3519_gb300 as k
    x, g = _case(33, 4096, 300, 256, 0.0)
    e, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    kx = k.Krux(0)
    rs = kx.krux_rank(e)
    ref = kx.krux_scan(rs, gd, 1e-3, capacity=4096 * 300)
    hits, H, P = _noalloc_out(20_000)
    st, n = k.krux_scan_noalloc(e, gd, 1e-3, hits, H, P)
    assert st == k.KRUX_OK and n == ref["n_hits"] and n > 0
    a = _sorted(hits[:n], H[:n], P[:n])
    b = _sorted(ref["hits"], ref["H"], ref["p"])
    assert np.array_equal(a[0], b[0])
    assert np.all(np.abs(a[1] - b[1]) <= 1e-6 * np.abs(b[1]) + 1e-10)
    assert np.all(np.abs(a[2] - b[2]) <= 1e-6 * b[2])
    kx.close()


def test_noalloc_stored_hit_limit():
    """More hits than the 262,144 records the entry point stores: KRUX_EOVERFLOW,
    the exact total, and every stored record one of krux_scan's hits with the
    same rank sums."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1307_3519_gb300 as k
    x, g = _case(34, 1024, 2000, 60, 0.0)
    e, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    kx = k.Krux(0)
    rs = kx.krux_rank(e)
    pth = 0.3
    ref = kx.krux_scan(rs, gd, pth, capacity=1024 * 2000)
    assert ref["n_hits"] > 262_144
    hits, H, P = _noalloc_out(400_000)
    st, n = k.krux_scan_noalloc(e, gd, pth, hits, H, P)
    assert st == k.KRUX_EOVERFLOW and n == ref["n_hits"]
    got = hits[:262_144].cpu().numpy().astype(np.int64)
    want = ref["hits"].cpu().numpy().astype(np.int64)
    key = lambda h: h[:, 0] * 10_000_000 + h[:, 1]
    order = np.argsort(key(want))
    pos = np.searchsorted(key(want)[order], key(got))
    assert np.all(pos < want.shape[0])
    match = want[order][pos]
    assert np.array_equal(match, got)  # a real hit, same pair and rank sums
    assert np.unique(key(got)).size == got.shape[0]  # no record twice
    kx.close()


def test_noalloc_rejects_missing_genotypes():
    """One -1 code: the entry point scans complete genotypes only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1307_3519_gb300 as k
    x, g = _case(35, 200, 500, 60, 0.0)
    g[123, 7] = -1
    e, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    hits, H, P = _noalloc_out(1000)
    st, n = k.krux_scan_noalloc(e, gd, 1e-3, hits, H, P)
    assert st == k.KRUX_EUNSUPPORTED
