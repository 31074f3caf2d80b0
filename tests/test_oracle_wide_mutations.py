"""The wide-range oracle's pins must catch plausible mistakes.  Each case plants one mistake in
a copy of oracle/wide.py's source, loaded as a separate module (the committed oracle is
untouched), and checks that the brute-force box enumeration or the binary64 rank-code pin
rejects it."""
import os
import struct
import types

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "wide.py")

MUTATIONS = {
    # the rank increment uses delta_nu's power instead of delta_rho's (transposed operand)
    "rank_delta_transposed": ("(((r << 24) | u) << rho), -(nu + 24))", "(((r << 24) | u) << nu), -(nu + 24))"),
    # the weight offset 2^nu - 1 is dropped from the dart weight
    "weight_offset_dropped": ("tw = ((((1 << nu) - 1) << (rho + 24)) + ", "tw = (0 + "),
    # top weight region skipped (off by one in the region bound)
    "region_bound_off_by_one": ("while cmp(((1 << nu) - 1, 0), y) <= 0:", "while cmp(((1 << (nu + 1)) - 1, 0), y) <= 0:"),
    # the row break compares a doubled row edge, so rows holding kept darts are skipped
    "row_edge_doubled": ("cmp(((((1 << rho) - 1) << nu) + (r << rho), -nu), theta) < 0:",
                         "cmp(((((1 << rho) - 1) << nu) + (r << rho), -nu + 1), theta) < 0:"),
    # the column break compares a doubled column edge
    "column_edge_doubled": ("cmp(((((1 << nu) - 1) << rho) + (w << nu), -rho), y) <= 0:",
                            "cmp(((((1 << nu) - 1) << rho) + (w << nu), -rho + 1), y) <= 0:"),
    # the last rank region below theta is skipped (off by one in the rank-region bound)
    "rank_region_bound": ("while cmp(((1 << rho) - 1, 0), theta) < 0:", "while cmp(((1 << (rho + 1)) - 1, 0), theta) < 0:"),
    # the code keeps one fraction bit too few
    "code_significand_short": ("top = n >> (L - 21) if L >= 21 else n << (21 - L)",
                               "top = n >> (L - 20) if L >= 20 else n << (20 - L)"),
}

CASES = [(0.3, 0.6), (1.7, 0.45), (2.9, 2.5), (0.05, 5.5), (1.1, 1.0), (3.4, 13.0)]


def _module(source: str, name: str):
    mod = types.ModuleType(name)
    exec(compile(source, f"<{name}>", "exec"), mod.__dict__)
    return mod


def _table():
    from oracle import poisson_thresholds
    return poisson_thresholds()


def _brute_force_agrees(mod) -> bool:
    T = _table()
    for x, theta in CASES:
        th = mod.dyadic(theta)
        try:
            got = {(c, q) + ids[:5] for c, q, ids in mod.element_darts(12345, x, 4, mod.seed_key(9), th, T,
                                                                       with_id=True)}
        except Exception:
            return False
        box = {b[:7] for b in mod.box_darts(12345, x, 4, 9, th, 4, 4, T)}
        if got != box:
            return False
    return True


def _rank_code_agrees(mod) -> bool:
    rng = np.random.default_rng(2)
    for _ in range(500):
        n = int(rng.integers(1, 2 ** 53))
        e = int(rng.integers(-1000, 900))
        v = n * 2.0 ** e if e > -1000 else 0.0
        if not v or v < 2.0 ** -1022 or v != v or v == float("inf"):
            continue
        bits = struct.unpack(">Q", struct.pack(">d", float(n) * 2.0 ** e))[0]
        if float(n) != n:                              # not a binary64 value: skip
            continue
        if mod.rank_code((n, e)) != bits >> 32:
            return False
    return True


def test_unmutated_copy_passes():
    mod = _module(open(SRC).read(), "wide_copy")
    assert _brute_force_agrees(mod) and _rank_code_agrees(mod)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mod = _module(src.replace(old, new), f"wide_{name}")
    assert not (_brute_force_agrees(mod) and _rank_code_agrees(mod)), f"{name} went unnoticed"
