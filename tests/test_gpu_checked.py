"""The bounds-checked build (-DFFG_CHECKED) on the GPU.

Every path of the library -- single and batched builds, FP64 and FP32
PageRank, the DAG solve, walks, minima, C_p, the batched step -- runs on a
few seeded spaces in a child process that loads the checked library
(FFG_LIB=checked): no check may fail, and every result must be bit-for-bit
the normal build's (the checks only guard accesses).  Then indices out of
range are planted in the graph's arrays on the host side of the test (an
in-neighbour past w and one below it, a minimum's raw point past the
fitness, out-neighbours past the last node): the guarded accesses are
skipped and counted with their site codes, and the process carries on
without a fault."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(checked: bool):
    env = dict(os.environ)
    if checked:
        env["FFG_LIB"] = "checked"
    else:
        env.pop("FFG_LIB", None)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_runs_clean_and_catches_planted_indices():
    normal = _run(False)
    chk = _run(True)
    assert not normal["checked"] and chk["checked"]
    assert chk["clean_failures"] == [0, 0]
    assert chk["results"] == normal["results"]
    pl = chk["planted"]
    n, code = pl["pagerank"]
    assert n > 0 and code == 101, pl
    assert pl["pagerank_finite"]
    n, code = pl["centrality"]
    assert n > 0 and code == 501, pl
    n, code = pl["walks"]
    assert n > 0 and code == 401, pl
    assert pl["walks_status"] != "ok"
    assert pl["after"] == [0, 0]
