"""The oracle's pins must catch plausible mistakes.  Each case copies
oracle/krux_oracle.c, plants one mistake by text substitution, compiles the copy
into a temporary directory and runs a compact version of the pin suite (the
hand-worked golden examples and scipy's Kruskal-Wallis on random tied / missing
cases) against it.  The unmodified source must pass the same checks."""
import ctypes
import os
import subprocess

import numpy as np
import pytest
import scipy.stats as st

from test_oracle import _load_golden, _mp_tail

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "krux_oracle.c")

MUTANTS = {
    "no_tie_correction": ("  H /= corr;\n", "\n"),
    "wrong_offset_3K": ("- 3.0 * (Kd + 1.0);", "- 3.0 * Kd;"),
    "wrong_scale_K2": ("12.0 / (Kd * (Kd + 1.0))", "12.0 / (Kd * Kd)"),
    "rank_off_by_one": ("(int64_t)(i + j + 2)", "(int64_t)(i + j + 1)"),
    "tie_sum_t2": ("ts += t * t * t - t;", "ts += t * t - t;"),
    "df_not_minus_one": ("out->df = groups > 0 ? groups - 1 : 0;", "out->df = groups;"),
    "tails_swapped": ("if (df % 2 == 0) {", "if (df % 2 == 1) {"),
    "odd_tail_sum_dropped": ("q += exp(-x) * xp / g;", "q += 0.0 * xp / g;"),
    "even_tail_one_term": ("for (int k = 0; k < df / 2; ++k) {", "for (int k = 0; k < 1; ++k) {"),
    "groups_past_two_ignored": ("  int groups = 0;\n  for (int i = 0; i <= lmax; ++i) {",
                                "  int groups = 0;\n  for (int i = 0; i < 3 && i <= lmax; ++i) {"),
    "nan_not_dropped": ("!isnan(x[k])) ? 1 : 0;", "1) ? 1 : 0;"),
    "descending_ranks": ("if (x->v < y->v) return -1;\n  if (x->v > y->v) return 1;",
                         "if (x->v > y->v) return -1;\n  if (x->v < y->v) return 1;"),
    "group_count_doubled": ("out->n[g[k]] += 1;", "out->n[g[k]] += 2;"),
    "threshold_not_strict": ("out->p < pthresh ? 1 : 0", "out->p <= 2.0 * pthresh ? 1 : 0"),
}


class _Pair(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("H_alt", ctypes.c_double),
                ("p", ctypes.c_double), ("tie", ctypes.c_double),
                ("rank2", ctypes.c_int64 * 5), ("d", ctypes.c_int64 * 5),
                ("n", ctypes.c_int32 * 5), ("K", ctypes.c_int32),
                ("df", ctypes.c_int32), ("hit", ctypes.c_int32)]


def _compile(src_text, tmp_path, name):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"lib{name}.so"
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-o", str(so), str(c), "-lm"])
    lib = ctypes.CDLL(str(so))
    lib.oracle_pair.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                ctypes.POINTER(_Pair)]
    lib.oracle_pair.restype = ctypes.c_int
    lib.oracle_pair_l.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.POINTER(_Pair)]
    lib.oracle_pair_l.restype = ctypes.c_int
    return lib


def _pair(lib, x, g, pthresh=0.05, max_code=2):
    x = np.ascontiguousarray(x, np.float32)
    g = np.ascontiguousarray(g, np.int8)
    r = _Pair()
    lib.oracle_pair_l(x.ctypes.data, g.ctypes.data, x.size, max_code, pthresh, ctypes.byref(r))
    return r


def _pins_fail(lib):
    """Returns the name of the first failing pin, or None."""
    for i, (x, g, H, df, d) in enumerate(_load_golden()):
        r = _pair(lib, x, g)
        if r.df != df or list(r.d)[:3] != d:
            return f"golden{i}:df/d"
        if not np.isclose(r.H, float(H), rtol=1e-12, atol=1e-12):
            return f"golden{i}:H"
        if not np.isclose(r.p, _mp_tail(H, df), rtol=1e-12, atol=0):
            return f"golden{i}:p"
        hit_expected = _mp_tail(H, df) < 0.3
        if bool(_pair(lib, x, g, 0.3).hit) != hit_expected:
            return f"golden{i}:hit"
    rng = np.random.default_rng(77)
    for j in range(45):
        mc = 2 if j < 30 else 3 + (j % 2)  # the last cases: markers with 4 or 5 groups
        n = int(rng.integers(6, 80))
        x = np.round(rng.standard_normal(n), j % 3).astype(np.float32)
        g = rng.integers(0, mc + 1, n).astype(np.int8)
        if j % 2:
            x[rng.random(n) < 0.1] = np.nan
            g[rng.random(n) < 0.1] = -1
        use = (g >= 0) & ~np.isnan(x)
        groups = [x[use & (g == k)].astype(np.float64) for k in range(mc + 1)]
        groups = [a for a in groups if a.size]
        if len(groups) < 2:
            continue
        s = st.kruskal(*groups)
        r = _pair(lib, x, g, pthresh=s.pvalue * 1.5, max_code=mc)
        if not (np.isclose(r.H, s.statistic, rtol=1e-9) and np.isclose(r.p, s.pvalue, rtol=1e-9)):
            return f"scipy{j}"
        if not r.hit or _pair(lib, x, g, pthresh=s.pvalue * 0.5, max_code=mc).hit:
            return f"hit{j}"
    return None


def test_unmodified_oracle_passes(tmp_path):
    lib = _compile(open(SRC).read(), tmp_path, "orig")
    assert _pins_fail(lib) is None


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    lib = _compile(src.replace(old, new), tmp_path, name)
    assert _pins_fail(lib) is not None, f"pins did not catch mutant {name}"
