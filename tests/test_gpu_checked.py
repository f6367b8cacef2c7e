"""The bounds-checked build (libphikron_checked.so: every global access of the apply-path
kernels checks its byte range against the registered device ranges first; see
include/phikron.h) on small and uneven shapes through every apply path, in a child process
(tests/checked_cases.py) because a process loads one of the two libraries.

* every case agrees with the oracle at its gate and leaves no violation on record;
* with PHIKRON_CHECKED_SHRINK = 8 (every library allocation registered 8 bytes short, so that
  accesses to their last 8 bytes count as outside, although they are inside memory the library
  owns) a mixed apply records a violation and check_status returns PHIKRON_EBOUNDS.  Refused
  accesses are skipped, so the GPU never sees an access outside a real allocation.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = os.path.join(HERE, "checked_cases.py")


def _run(args, extra_env):
    env = dict(os.environ)
    env.update(extra_env)
    env["PHIKRON_CHECKED"] = "1"
    r = subprocess.run([sys.executable, CASES] + args, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_small_uneven_shapes_no_violation():
    res = _run([], {})
    assert res["checked"] == 1
    names = [c["name"] for c in res["cases"]]
    assert len(names) >= 20, names
    for c in res["cases"]:
        print(f"{c['name']:34s} err {c['err']:.2e} (gate {c['gate']:.0e}) violation site {c['violation']['site']}")
    for c in res["cases"]:
        assert c["violation"]["site"] == 0 and c["violation"]["count"] == 0, c
        assert c["err"] <= c["gate"], c


def test_checked_build_reports_refused_access():
    from paper_2211_00696_gb300 import phikron as B
    res = _run(["--shrink"], {"PHIKRON_CHECKED_SHRINK": "8"})
    assert res["status_code"] == B.EBOUNDS, res
    v = res["violation"]
    assert v["site"] != 0 and v["count"] >= 1 and v["bytes"] > 0, v
    print("refused:", v)
