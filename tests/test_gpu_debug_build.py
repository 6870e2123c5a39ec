"""The index-checked debug build (-DMG_BOUNDS_CHECK, libmg_debug.so): the
same cycles and solves as the release library, bitwise, on DIA and SELL
levels (fused SELL steps included), the two-feature cycle and a stacked
context, with no index out of range recorded.  Each library runs in its own
child process (tests/debug_build_case.py)."""
import json
import os
import subprocess
import sys

import pytest

from paper_2608_29082_b300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_case(variant: str) -> dict:
    env = dict(os.environ, MG_LIB_VARIANT=variant)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "debug_build_case.py")],
                       capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_matches_release_and_records_nothing():
    build.build(debug=True)
    rel = run_case("release")
    dbg = run_case("debug")
    assert rel["library"] == "libmg.so" and dbg["library"] == "libmg_debug.so"
    assert rel["bounds"] == [0, 0]
    assert dbg["bounds"] == [1, 0]
    for key in rel:
        if key not in ("bounds", "library"):
            assert dbg[key] == rel[key], key
