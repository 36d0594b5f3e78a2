"""The bounds-checking build (HPR_BOUNDS_CHECK; compute-sanitizer is not available on the GPU
pool, so the library checks its own gathers): every path -- multi-CTA, single CTA, grid,
cluster, the FP32 form, the three batch modes and the allocation-free power method -- runs
on it without one out-of-range gather index, and gives bitwise the results of the normal
build (the checks do not touch the arithmetic).  A planted out-of-range column index in a
caller's CSR (allocation-free power method) is counted and read as index 0; the context
stays usable.  Each library runs in a subprocess of its own (tests/bounds_workload.py)."""
import json
import os
import subprocess
import sys

import pytest

from paper_2408_12179_b300 import build

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib, *extra):
    out = subprocess.run([sys.executable, os.path.join(HERE, "bounds_workload.py"), lib, *extra],
                         capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-3000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_checked_build_finds_no_violation_and_matches_the_normal_build():
    build.build()
    build.build_checked()
    normal = _run(build.LIB)
    checked = _run(build.LIB_CHECKED, "--plant")
    assert normal["violations"] == -1                 # the normal build checks nothing
    assert checked["violations"] == 0, checked
    for key, val in normal["results"].items():
        assert checked["results"][key] == val, (key, val, checked["results"][key])
    assert checked["planted"] > 0                     # the planted index was caught, every step
    assert checked["results"]["after_plant"] == normal["results"]["tiny0/p0"]
    print("paths:", sorted(k for k, v in normal["results"].items() if not str(v).startswith("refused")),
          "planted violations:", checked["planted"])
