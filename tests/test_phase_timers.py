"""The phase-timer build (HOUGH_PHASE_TIMERS): same results as the oracle, and cycles counted
in every phase the item runs, for both peak finders. Each case runs as a child process, since
a process loads one build of the library."""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.gpu
@pytest.mark.parametrize("mode", [0, 1])
def test_phase_timer_build_matches_oracle_and_counts(mode):
    r = subprocess.run([sys.executable, os.path.join(HERE, "phase_timer_check.py"), str(mode)], capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["enabled"] is True and "_build_phase" in res["lib"]
    c = res["cycles"]
    ran = ["clear", "stage", "vote", "fold", "scan", "sel_columns", "sel_bitmaps", "sel_a", "sel_b"]
    ran += ["it_max", "it_collect", "it_resolve", "it_order"] if mode else ["exscan", "records"]
    assert all(c[k] > 0 for k in ran), c
    if mode:
        assert c["exscan"] == 0 and c["records"] == 0
    else:
        assert c["it_max"] == 0 and c["it_resolve"] == 0
