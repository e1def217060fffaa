"""The bounds-checked build on the GPU. Every path runs with guard zones after
each workspace buffer, and no zone may change:
- FP64, FP32-refined and double-float;
- 2D on ragged, minimum and 4096-long grids, and 3D;
- graph and host-loop steps, the component calls, hc_run, the adjoint, the
  batch, and the launch-shape variants.

Planted damage, a host memset into a zone, must be reported as HC_EBOUNDS
with the right zone. tests/redzone_run.py does the work in a subprocess that
loads libhc_gb300_check.so."""
import json
import os
import subprocess
import sys

import pytest

from gpu_common import hc  # noqa: F401

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def run(hc):
    env = dict(os.environ, HC_GB300_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "redzone_run.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_the_checked_library_ran(run):
    assert run["library"] == "libhc_gb300_check.so"
    assert not run["errors"], run["errors"]
    assert len(run["results"]) > 80


def test_no_guard_zone_changes_on_any_path(run, hc):
    bad = [x for x in run["results"] if x["rc"] != hc.HC_OK or x["zone"] != -1]
    assert not bad, bad
    scanned = [x for x in run["results"] if x["zones"] >= 0]
    assert scanned and min(x["zones"] for x in scanned) >= 30


def test_planted_damage_is_reported_with_its_zone(run, hc):
    assert len(run["pokes"]) == 3
    for p in run["pokes"]:
        assert p["poke_rc"] == hc.HC_OK
        assert p["rc"] == hc.HC_EBOUNDS and p["zone"] == p["poked"] and p["owner_bytes"] > 0
