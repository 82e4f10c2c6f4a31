"""The bound behind the plain form's NaN variant (section "Handling missing
values": a trait's NaN samples leave the genotype groups, N_i' = the samples
present for both), checked by brute force on the host.

For a pair with group sizes N_i over the samples with a genotype and a trait with
c NaN samples, the kernel's coefficient set for C >= c takes 1/max(N_i - C, 1)
for every non-empty group and the threshold of df 1 whenever some group could
vanish (N_i <= C), else of df 2.  The claim: for every way the c NaN samples can
fall into the groups, and any centred sums D_i the remaining samples can have,
sum_i D_i^2 / N_i' / h_df' is at most that bound (empty groups and df 0 add
nothing).  The test enumerates small group sizes, every placement and the sets
C the kernel uses (1, 2, 3, 4, 6), with random sums."""
import itertools

import numpy as np

SETS = (1, 2, 3, 4, 6)


def _set_of(c):
    return next(C for C in SETS if C >= c)


def _bound(D, n, C, h1, h2):
    q = [1.0 / max(ni - C, 1) if ni > 0 else 0.0 for ni in n]
    groups = sum(ni > 0 for ni in n)
    if groups < 2:
        return 0.0
    sure = sum(ni > C for ni in n)
    h = h2 if sure >= 3 else h1
    return sum(d * d * qi for d, qi in zip(D, q)) / h


def _exact(D, n_present, h1, h2):
    groups = sum(ni > 0 for ni in n_present)
    if groups < 2:
        return 0.0
    h = h2 if groups == 3 else h1
    return sum(d * d / ni for d, ni in zip(D, n_present) if ni > 0) / h


def test_coefficient_sets_bound_every_placement():
    rng = np.random.default_rng(1307)
    h1, h2 = 15.137, 18.421  # chi-square thresholds of df 1 and 2 at p = 1e-4
    checked = 0
    for n in itertools.product(range(0, 7), repeat=3):
        for c in range(1, 7):
            C = _set_of(c)
            # every placement of the c NaN samples (k_i of them in group i)
            for k in itertools.product(range(c + 1), repeat=3):
                if sum(k) > c or any(ki > ni for ki, ni in zip(k, n)):
                    continue
                npres = [ni - ki for ni, ki in zip(n, k)]
                for _ in range(4):
                    # centred sums of the present samples: zero in an emptied group,
                    # summing to zero over the groups
                    D = rng.normal(size=3) * 50.0
                    D = [d if m > 0 else 0.0 for d, m in zip(D, npres)]
                    live = [i for i in range(3) if npres[i] > 0]
                    if live:
                        D[live[-1]] -= sum(D)
                    e = _exact(D, npres, h1, h2)
                    b = _bound(D, n, C, h1, h2)
                    assert e <= b * (1 + 1e-12) + 1e-12, (n, c, k, D, e, b)
                    checked += 1
    assert checked > 10000
