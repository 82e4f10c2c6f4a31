"""Checks of the seeded input generators (shapes, code ranges, the published
SplitMix64 sequence, missing-value structure)."""
import numpy as np

import synth


def test_splitmix64_known_answers():
    # SplitMix64 from state 0: the first outputs of the published generator
    assert synth.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                             0x06C45D188009454F]


def test_perms_are_permutations_and_seeded():
    a = synth.make_perms(1307, 16, 102)
    b = synth.make_perms(1307, 16, 102)
    assert a.shape == (16, 102) and a.dtype == np.int32
    assert np.array_equal(a, b)
    for p in a:
        assert np.array_equal(np.sort(p), np.arange(102))
    assert len({tuple(p) for p in a}) == 16


def test_config_shapes_and_codes():
    d = synth.config(1, T=20, S=50)
    assert d["expr"].shape == (20, 60) and d["geno"].shape == (50, 60)
    assert d["geno"].dtype == np.int8 and set(np.unique(d["geno"])) <= {0, 1, 2}
    d2 = synth.config(2, T=30, S=2500)
    assert d2["expr"].shape == (30, 102) and d2["causal_blocks"].shape == (30, 3)
    assert np.all(d2["expr"] > 0)


def test_missing_structure():
    d = synth.config(3, T=50, S=3000)
    g = d["geno"]
    miss = (g == -1)
    rows = miss.any(axis=1)
    assert rows.sum() == 300
    assert np.all(miss[rows].sum(axis=1) == 2)
    assert np.array_equal(rows, d["pattern_of_snp"] >= 0)
    assert 0.005 < np.isnan(d["expr"]).mean() < 0.015


def test_cohorts():
    d = synth.config(5, T=10, S=20)
    assert [c["N"] for c in d["cohorts"]] == list(synth.COHORT_NS)
    for c in d["cohorts"]:
        assert c["geno"].shape == (20, c["N"]) and c["expr"].shape == (10, c["N"])
