"""Comparison of CUDA-path results with the FP64 oracle (test helper).

Tolerances: rank sums (d0, d1), hit indices and ranks are compared exactly.
H and p are compared within 1e-6 relative.  H also gets an absolute slack of
1e-10: the oracle evaluates Eq. 2 as 12/(K(K+1)) sum S_i^2/N_i - 3(K+1), whose
cancellation leaves an absolute error of a few 3(K+1) * 2^-52 (below 1e-12 for
K <= 512) when H itself is tiny.  Pairs whose oracle p lies within 1e-12
relative of P_c are boundary-ambiguous (their side of the threshold depends on
the last bit of an FP64 evaluation) and are excluded from the hit-set
comparison; they are counted and the count is returned."""
import numpy as np

H_RTOL, H_ATOL, P_RTOL = 1e-6, 1e-10, 1e-6


def gpu_hits_np(res):
    h = res["hits"].cpu().numpy().astype(np.int64)
    H = res["H"].cpu().numpy()
    p = res["p"].cpu().numpy()
    order = np.lexsort((h[:, 0], h[:, 1]))
    return h[order], H[order], p[order]


def check_hits(res, orc, traits, snps, pthresh, must_have_hits=True):
    """res: GPU result restricted to `traits` x `snps` (global indices, sorted);
    orc: oracle.scan over the same selection.  Asserts identical hit sets
    (outside the boundary band), exact d0/d1 and H/p within tolerance."""
    h, H, p = gpu_hits_np(res)
    traits = np.asarray(traits)
    snps = np.asarray(snps)
    tpos = -np.ones(int(traits.max()) + 1 if traits.size else 1, dtype=np.int64)
    tpos[traits] = np.arange(traits.size)
    spos = -np.ones(int(snps.max()) + 1 if snps.size else 1, dtype=np.int64)
    spos[snps] = np.arange(snps.size)
    keep = (h[:, 0] < tpos.size) & (h[:, 1] < spos.size)
    keep[keep] &= (tpos[h[keep, 0]] >= 0) & (spos[h[keep, 1]] >= 0)
    h, H, p = h[keep], H[keep], p[keep]
    a, b = tpos[h[:, 0]], spos[h[:, 1]]
    op = orc["p"]
    band = np.abs(op / pthresh - 1.0) < 1e-12
    gpu_set = np.zeros_like(orc["hit"])
    gpu_set[a, b] = True
    assert len(set(zip(a.tolist(), b.tolist()))) == a.size, "duplicate hit records"
    diff = (gpu_set != orc["hit"]) & ~band
    assert not diff.any(), f"hit sets differ at {np.argwhere(diff)[:10].tolist()} " \
                           f"(gpu {gpu_set.sum()}, oracle {orc['hit'].sum()})"
    if must_have_hits:
        assert orc["hit"].sum() > 0, "test selection has no hits"
    # exact rank sums and FP64 statistics of the reported hits
    assert np.array_equal(h[:, 2], orc["d"][a, b, 0]), "d0 differs"
    assert np.array_equal(h[:, 3], orc["d"][a, b, 1]), "d1 differs"
    oh, opv = orc["H"][a, b], op[a, b]
    assert np.all(np.abs(H - oh) <= H_RTOL * np.abs(oh) + H_ATOL), \
        f"H max rel err {np.max(np.abs(H - oh) / np.maximum(oh, 1e-300))}"
    assert np.all(np.abs(p - opv) <= P_RTOL * opv), \
        f"p max rel err {np.max(np.abs(p - opv) / np.maximum(opv, 1e-300))}"
    return int(band.sum())


def check_dense(dH, dp, orc):
    """Dense GPU H, p (numpy) against the oracle over the same pairs."""
    oh, op = orc["H"], orc["p"]
    errH = np.abs(dH - oh) - (H_RTOL * np.abs(oh) + H_ATOL)
    assert np.all(errH <= 0), f"dense H off at {np.argwhere(errH > 0)[:5].tolist()}"
    errp = np.abs(dp - op) - P_RTOL * op
    assert np.all(errp <= 0), f"dense p off at {np.argwhere(errp > 0)[:5].tolist()}"
