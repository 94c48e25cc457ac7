"""Each deliberate mistake planted in a copy of the oracle (ORACLE_PLANT in
oracle/oracle.c) must make the oracle's pins fail.  The pins
(tests/test_oracle.py and tests/test_oracle_properties.py) run in a child
pytest against the planted build (ORACLE_LIBRARY); the build with no plant
must pass the same run, so a failure means the mistake was caught.

The plants cover every oracle function: Algorithm 2's start rank, the
terminator order and the length tie-break of the suffix order, Insert's tie
order, C[] without terminators, the reverse-order start rank, overlapping
pattern counts, the checkpoints of the sampled LF inversion, the row of one
suffix, rank's range, C[] for alphabets past four symbols, the direct g's
set of old reads, B_int at a terminator suffix and the full inversion's
C[]."""
import os
import subprocess
import sys

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PINS = [os.path.join(HERE, "test_oracle.py"), os.path.join(HERE, "test_oracle_properties.py")]
PLANTS = range(1, 15)


def _run_pins(lib_path: str) -> subprocess.CompletedProcess:
    env = dict(os.environ, ORACLE_LIBRARY=lib_path)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_pins_pass_on_an_unplanted_build(tmp_path):
    r = _run_pins(oracle.build_planted(0, str(tmp_path / "liboracle_plant0.so")))
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("plant", PLANTS)
def test_planted_mistake_is_caught(plant, tmp_path):
    r = _run_pins(oracle.build_planted(plant, str(tmp_path / f"liboracle_plant{plant}.so")))
    # exit code 1: tests ran and at least one failed (not a crash or a usage error)
    assert r.returncode == 1, f"planted mistake {plant} slipped through the pins:\n{r.stdout[-2000:]}"
