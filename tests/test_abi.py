"""The C-ABI library builds, loads and exports every function include/krux.h
declares; host-only entry points work without a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "krux.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1307_3519_gb300 import build
    build.build()
    import paper_1307_3519_gb300 as k
    return k.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(krux_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["krux_rank", "krux_scan", "krux_permute", "krux_scan_plain", "krux_scan_grouped",
                     "krux_create", "krux_destroy", "krux_make_perms"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1307_3519_gb300 as k
    names = declared_functions()
    assert sorted(k.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    for s in range(7):
        assert lib.krux_status_string(s)


def test_make_perms_matches_generator(lib):
    import paper_1307_3519_gb300 as k
    for seed, P, N in [(1307, 16, 102), (0, 3, 7), (99, 2, 500)]:
        assert np.array_equal(k.krux_make_perms(seed, P, N), synth.make_perms(seed, P, N))


def test_create_without_gpu_reports_an_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.krux_create(ctypes.byref(h), 0)
    assert st != 0 and not h.value


def test_null_arguments_are_rejected(lib):
    # validation happens before any device work
    assert lib.krux_create(None, 0) == 1
    assert lib.krux_set_profiling(None, 1) == 1


def test_every_launch_plan_is_sound(lib):
    """The shared-memory plan of every sample count (and of the tuning shapes the
    GPU tests use) passes the alignment / bounds check each launch runs, so no
    launch can get a misaligned TMA destination or vector load."""
    import paper_1307_3519_gb300 as k
    for N in range(1, 513):
        for nan in (False, True):
            for layout in (-1, 0):
                st, plan = k.krux_debug_plan(N, nan, layout)
                assert st == 0, (N, nan, layout, plan)
                assert plan["smem"] <= 232448 and plan["b_region"] % 1024 == 0
                assert plan["nc"] * plan["b_stride"] <= plan["b_region"]
    for N in (60, 102, 150):
        for layout, nc, nA, ka in [(0, 3, 3, 0), (1, 1, 2, 0), (1, 4, 2, 0), (1, 2, 4, 64),
                                   (0, 2, 3, 64), (1, 1, 4, 64), (1, 4, 3, 64)]:
            st, plan = k.krux_debug_plan(N, False, layout, nc, nA, ka)
            assert st in (0, 6)  # sound, or refused (never an unchecked plan)


def test_plain_form_plans(lib):
    """The plain form's launch plans (the whole K in one rank stage, an even number
    of resident chunks as N = 256 MMA pairs, room for the hit-event ring) and those
    of its NaN variant (the coefficient sets in place of the codes): sound wherever
    they exist, the NaN variant only where the plain form is, and both with four
    resident chunks at the benchmark's N = 102."""
    import paper_1307_3519_gb300 as k
    for N in range(1, 513):
        st2, p2 = k.krux_debug_plan(N, 2)
        st3, p3 = k.krux_debug_plan(N, 3)
        assert st2 in (0, 6) and st3 in (0, 6), (N, st2, st3)
        assert st3 != 0 or st2 == 0, N
        for st, pl in ((st2, p2), (st3, p3)):
            if st == 0:
                assert pl["smem"] <= 232448 and pl["nkb"] == 1, (N, pl)
                assert pl["nc"] >= 2 and pl["nc"] % 2 == 0, (N, pl)
    for mode in (2, 3):
        st, pl = k.krux_debug_plan(102, mode)
        assert st == 0 and pl["nc"] == 4 and pl["nA"] == 2, (mode, pl)
    assert k.krux_debug_plan(102, 2, layout=0)[0] == 6  # the plain forms need the 32-byte swizzle
    assert k.krux_debug_plan(102, 4)[0] == 1


def test_every_autotune_candidate_is_sound_or_refused(lib):
    """The shapes krux_autotune tries: each one either passes the plan check or
    is refused before any launch."""
    import paper_1307_3519_gb300 as k
    for N in (16, 48, 60, 75, 102, 150, 200, 256, 300, 400, 500, 512):
        for nan in (False, True):
            for layout in (1, 0):
                for nc in (4, 3, 2, 1):
                    for nA in (2, 3, 4):
                        for ka in (0, 64):
                            st, plan = k.krux_debug_plan(N, nan, layout, nc, nA, ka)
                            assert st in (0, 1, 6), (N, nan, layout, nc, nA, ka, st)
                            if st == 0:
                                assert plan["smem"] <= 232448 and plan["b_region"] % 1024 == 0


def test_parametric_tails_match_scipy(lib):
    """The FP64 F / t tails of the parametric finalisation (closed form for two
    numerator degrees of freedom, else the continued fraction of the incomplete
    beta function), evaluated on the host, against scipy."""
    import paper_1307_3519_gb300 as k
    import scipy.special as sps
    import scipy.stats as st
    for d1, d2 in [(1, 10), (1, 100), (2, 3), (2, 99), (1, 498), (2, 300), (3, 99)]:
        for f in [0.01, 0.5, 1.0, 3.0, 7.5, 15.0, 30.0, 80.0, 250.0]:
            want = st.f.sf(f, d1, d2)
            assert k.krux_debug_tail(0, f, d1, d2) == pytest.approx(want, rel=1e-10, abs=1e-300)
    for nu in [2, 5, 30, 100, 498]:
        for t in [0.1, 1.0, 2.5, 4.0, 6.0, 9.0, 15.0]:
            want = 2.0 * st.t.sf(t, nu)
            assert k.krux_debug_tail(1, t, nu) == pytest.approx(want, rel=1e-10, abs=1e-300)
    for a, b, x in [(0.5, 0.5, 0.3), (50.0, 0.5, 0.9), (3.0, 7.0, 0.2), (120.0, 1.0, 0.99)]:
        assert k.krux_debug_tail(2, x, a, b) == pytest.approx(sps.betainc(a, b, x), rel=1e-11)
