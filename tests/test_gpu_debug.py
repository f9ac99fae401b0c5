"""The bounds-checked build (libpfreg_debug.so, -DPF_DEBUG=1).

Its kernels check every gather index of the measurement and the warp against
the buffer before loading; an index outside is counted and the load skipped,
nothing traps.  Here the element-by-element parity cases of
test_gpu_parity.py run again in a child process on that build: each must
still match the oracle and end with no out-of-bounds index (conftest checks
pf_debug_bounds after every GPU test when PFREG_DEBUG=1)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_release_build_reports_no_checks():
    import paper_2504_19930_gb300 as pk
    pk.build()
    pk.load()
    on, hits, _ = pk.pf_debug_bounds(clear=True)
    assert (on, hits) == (os.environ.get("PFREG_DEBUG") == "1", 0)


def test_parity_cases_clean_under_bounds_checks():
    import paper_2504_19930_gb300 as pk
    pk.build(debug=True)
    env = dict(os.environ, PFREG_DEBUG="1")
    sel = ("random_poses or degenerate or integer_maps or trajectory_bit_exact_small or warp or spacing "
           "or estimate_dice_trace")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_parity.py"),
                        "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider", "-k", sel],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in tail and "no tests ran" not in tail, tail
