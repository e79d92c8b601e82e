"""The debug build (NB_DEBUG: index checks on data-dependent indices that
report NB_E_INVALID instead of touching memory out of bounds) runs the same
cases as the release build without a report and with the same bits: the
checks find nothing and change no arithmetic. compute-sanitizer is closed on
this machine pool; these checks stand in for its out-of-bounds detection."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_09184_b300 import build
    build.build()
    build.build(debug=True)


def _run(tmp_path, debug):
    out = str(tmp_path / ("debug.npz" if debug else "release.npz"))
    env = dict(os.environ, NB_DEBUG="1" if debug else "0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "helpers", "debug_run.py"),
                        out], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_debug_build_reports_nothing_and_matches_release(tmp_path):
    rel, dbg = _run(tmp_path, False), _run(tmp_path, True)
    assert str(rel["lib"]) == "libnb.so" and str(dbg["lib"]) == "libnb_debug.so"
    assert rel["sys_stats"][0] > 0 and rel["sys_stats"][1] > 0  # groups and mergers happened
    for k in rel.files:
        if k == "lib":
            continue
        assert np.array_equal(rel[k], dbg[k]), k
