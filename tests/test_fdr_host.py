"""Host arithmetic of the empirical FDR curve (section "P-value calculation and
empirical FDR correction"): the cumulative histogram of krux_permute read as a
curve must equal the definition evaluated by the oracle at the grid thresholds."""
import numpy as np
import pytest

from paper_1307_3519_gb300.fdr import fdr_curve, hit_fdr


def _bin(p, pc, w, bins):
    b = np.floor((-np.log10(p) + np.log10(pc)) / w)
    return np.clip(b, 0, bins - 1).astype(np.int64)


def _hist(rows, pc, w, bins):
    h = np.zeros((len(rows), bins), np.int64)
    for q, p in enumerate(rows):
        p = p[p < pc]
        np.add.at(h[q], _bin(p, pc, w, bins), 1)
    return h


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_curve_equals_definition(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    pc, w, bins = 1e-3, 0.25, 12
    # log-uniform p-values below and above P_c, off the bin edges
    rows = [10.0 ** -rng.uniform(1.0, 7.0, size=rng.integers(50, 400)) for _ in range(4)]
    h = _hist(rows, pc, w, bins)
    c = fdr_curve(h, pc, w)
    n_real, pcounts, fdr = oracle_mod.fdr_from_pvalues(rows[0], rows[1:], pc, c["threshold"])
    assert np.array_equal(c["n_real"], n_real)
    assert np.allclose(c["mean_perm"], pcounts.mean(axis=0), rtol=0, atol=1e-12)
    assert np.allclose(c["fdr"], fdr, rtol=1e-12, atol=0, equal_nan=True)


def test_hit_fdr_reads_the_step():
    pc, w = 1e-2, 1.0
    h = np.array([[3, 1, 1], [1, 1, 0], [2, 0, 1]], np.int64)
    c = fdr_curve(h, pc, w)
    # tails: real 5,2,1; perms 2,1,0 and 3,1,1 -> mean 2.5,1,0.5
    assert list(c["n_real"]) == [5, 2, 1]
    assert np.allclose(c["fdr"], [0.5, 0.5, 0.5])
    assert np.allclose(hit_fdr(np.array([5e-3, 5e-4, 1e-9]), h, pc, w), [0.5, 0.5, 0.5])


def test_curve_rejects_a_histogram_without_permutations():
    with pytest.raises(ValueError):
        fdr_curve(np.zeros((1, 4), np.int64), 1e-3, 0.1)
