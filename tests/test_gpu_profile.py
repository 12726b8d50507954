"""Kernel timing (ss_profile, ss_profile_entry, ss_profile_trace): level 1
brackets the main kernels only, level 2 every bracket; the trace's brackets
lie inside the session and each ends after it starts; off records nothing."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2302_00752_gb300 import binding, pipeline
    return binding, pipeline


def run_once(gp, p):
    r = gp.run_fused(p, tol=1e-10, max_iter=1000)
    assert r.stats["status"] == "SS_OK", r.stats
    r.stamp.destroy()


def test_profile_levels_and_trace(mods):
    B, gp = mods
    p = gp.prepare(W.make_cfg1())
    run_once(gp, p)                      # plans and pools warm

    B.profile(True, level=1)
    run_once(gp, p)
    main = B.profile_totals()
    B.profile(False)
    assert any(k.startswith("k_solve") for k in main), main
    assert "k_neighbors" in main
    assert not any(k in main for k in ("k_insert", "k_finalize", "stamp_build")), main

    B.profile(True, level=2)
    run_once(gp, p)
    every = B.profile_totals()
    trace = B.profile_trace()
    B.profile(False)
    assert set(main) <= set(every)
    for k in ("k_insert", "k_finalize", "stamp_build"):
        assert k in every, every
    for name, (n, ms) in every.items():
        assert n >= 1 and ms >= 0.0, (name, n, ms)
    assert len(trace) == sum(n for n, _ in every.values())
    for name, t0, t1 in trace:
        assert t1 >= t0 >= -1e-3, (name, t0, t1)
    # a stage bracket holds the brackets launched inside it
    sb = [e for e in trace if e[0] == "stamp_build"][0]
    ins = [e for e in trace if e[0] == "k_insert"]
    assert ins and all(sb[1] <= e[1] and e[2] <= sb[2] + 1e-3 for e in ins)

    # off: nothing recorded
    run_once(gp, p)
    assert B.profile_totals() == {}
    assert B.profile_trace() == []
