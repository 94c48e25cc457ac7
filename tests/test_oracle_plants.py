"""Each deliberate mistake planted in a copy of the oracle (ORACLE_PLANT in
oracle/oracle.c) must make at least one pin fail: the pins are strong enough
to catch a wrong start rank in Algorithm 2, reversed terminator order, a
wrong length tie-break, a flipped Insert tie, a C[] without terminators and
a reverse-order Algorithm 1 that starts Algorithm 2 at m_ext."""
import numpy as np
import pytest

import brute
import oracle
from test_oracle import load_golden, pack, random_set


def _pins_hold() -> bool:
    try:
        for alpha, reads, expect in load_golden():
            if bytes(oracle.bwt(*pack(reads), alpha)) != expect:
                return False
        for seed in range(30):
            rng = np.random.default_rng(seed)
            reads = random_set(rng, int(rng.integers(1, 10)), 9)
            data, off = pack(reads)
            if bytes(oracle.bwt(data, off)) != brute.bwt(reads):
                return False
            m = len(reads)
            if m > 1:
                one = oracle.bwt(data, off)
                if not np.array_equal(oracle.setbwte(data, off, list(range(m + 1))), one):
                    return False
                if not np.array_equal(oracle.setbwte(data, off, list(range(m + 1)), reverse=True), one):
                    return False
        return True
    except oracle.OracleError:
        return False


@pytest.mark.parametrize("plant", [1, 2, 3, 4, 5, 6])
def test_planted_mistake_is_caught(plant, tmp_path):
    path = oracle.build_planted(plant, str(tmp_path / f"liboracle_plant{plant}.so"))
    try:
        oracle.use_library(path)
        assert not _pins_hold(), f"planted mistake {plant} slipped through the pins"
    finally:
        oracle.use_library(None)


def test_unplanted_oracle_passes_the_same_pins():
    assert _pins_hold()
