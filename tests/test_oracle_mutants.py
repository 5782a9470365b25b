"""The pins are strong enough: each plausible mistake, planted in a copy of the
oracle's C source and compiled on the CPU, must fail at least one pin."""
import os
import shutil

import pytest

import oracle
from tests import _pins

MUTANTS = {
    "shortest_not_longest": ("len > m->klen[cur]", "len < m->klen[cur]"),
    "tie_highest_id": ("(len == m->klen[cur] && id < cur)", "(len == m->klen[cur] && id > cur)"),
    "scan_single_failure_step": (
        "while (s != 0 && oracle_goto(m, s, a) < 0) s = m->nodes[s].fail;",
        "if (s != 0 && oracle_goto(m, s, a) < 0) s = m->nodes[s].fail;",
    ),
    "failure_always_root": ("m->nodes[u].fail = f;", "m->nodes[u].fail = 0;"),
    "build_single_failure_step": (
        "while (v != 0 && oracle_goto(m, v, a) < 0) v = m->nodes[v].fail;",
        "if (v != 0 && oracle_goto(m, v, a) < 0) v = m->nodes[v].fail;",
    ),
    "no_inherited_outputs": ("v >= 0; v = m->nodes[v].dict)", "v >= 0; v = -1)"),
    "seven_bit_goto": (
        "if (m->nodes[c].byte == a) return c;",
        "if ((m->nodes[c].byte & 0x7F) == (a & 0x7F)) return c;",
    ),
    "dict_skips_failure_state": (
        "m->nodes[u].dict = (m->nodes[f].own_head >= 0) ? f : m->nodes[f].dict;",
        "m->nodes[u].dict = m->nodes[f].dict;",
    ),
    "own_list_keeps_last": ("if (m->nodes[s].own_head < 0) {", "if (1) {"),
}

ORDER = ["w1", "w2", "paper_mode", "single_keyword", "length_one", "all_grams", "invariants"]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(oracle.SOURCE).read()
    assert old in src, "mutation site vanished from the oracle source"
    path = os.path.join(str(tmp_path), "mutant.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.load(oracle.compile_source(path, os.path.join(str(tmp_path), "libmutant.so")))
    caught = []
    for pin in ORDER:
        try:
            _pins.ALL_PINS[pin](lib)
        except AssertionError:
            caught.append(pin)
            break
    if not caught:
        try:
            _pins.pin_bruteforce(lib, cases=3000)
        except AssertionError:
            caught.append("bruteforce")
    assert caught, "planted mistake %r passed every pin" % name
