"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
from tests import _pins


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("name", sorted(_pins.ALL_PINS))
def test_pin(lib, name):
    _pins.ALL_PINS[name](lib)


def test_rejects_empty(lib):
    with pytest.raises(ValueError):
        oracle.Machine([b"ab", b""], lib)
    with pytest.raises(ValueError):
        oracle.Machine([], lib)


def test_state_count_is_distinct_prefixes(lib):
    pats = [b"he", b"she", b"his", b"hers", b"he"]
    prefixes = {p[:j] for p in pats for j in range(1, len(p) + 1)}
    with oracle.Machine(pats, lib) as m:
        assert m.n_states == len(prefixes) + 1
        counts = m.depth_counts()
        assert counts[0] == 1 and int(counts.sum()) == m.n_states


def test_walk_steps_small(lib):
    # he/she/his/hers on "ushers": walks from each start count goto evaluations
    # u:1 (miss)  s:s,h,e then r misses -> 4  h:h,e,r,s then end -> 4
    # e:1  r:1  s:1 then end -> 1
    with oracle.Machine([b"he", b"she", b"his", b"hers"], lib) as m:
        total, longest = m.walk_steps(b"ushers")
    assert total == 1 + 4 + 4 + 1 + 1 + 1 and longest == 4


def test_duplicates_lowest_id(lib):
    # starts: 0 -> "ab" (ids 0 and 2 are equal strings: lowest wins), 1 -> none,
    # 2 -> "x", 3 -> "a" (only id 3 spells it)
    ids = oracle.pfac_ids([b"ab", b"x", b"ab", b"a"], b"abxa")
    assert ids.tolist() == [0, -1, 1, 3]
