"""The committed GB300 execution-plan table (host logic, no GPU): every line
is a well-formed key of a skeleton the library knows, naming a variant the
library offers (or -1, the built-in default) with launch fields in range,
no key appears twice, and the library loads exactly those entries."""
import os

import pytest

sk = pytest.importorskip("paper_1405_2915_gb300")

TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1405_2915_gb300",
                     "dispatch_gb300.tbl")


def entries():
    out = []
    for lineno, line in enumerate(open(TABLE), 1):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        f = line.split()
        assert len(f) == 10, f"line {lineno}: {line!r}"
        out.append((lineno, [int(v) for v in f]))
    return out


def test_table_lines_are_valid_keys_and_choices():
    seen = set()
    for lineno, (skel_id, fn, dtype, bucket, radius, residency, variant, block, ept, tile) in entries():
        assert 0 <= skel_id < len(sk.SK), lineno
        assert dtype in (sk.F32, sk.I32, sk.I64), lineno
        assert 0 <= bucket < 16 and residency in (0, 1) and radius >= 0, lineno
        assert variant == -1 or 0 <= variant < sk.skel_variant_count(skel_id), lineno
        assert block in (0, 128, 256, 512, 1024) and ept >= 0 and 0 <= tile <= 8, lineno
        key = (skel_id, fn, dtype, bucket, radius, residency)
        assert key not in seen, f"line {lineno}: key {key} appears twice"
        seen.add(key)


def test_library_loads_every_entry():
    n = len(entries())
    sk.skel_load_dispatch_table(TABLE)
    try:
        assert sk.skel_dispatch_size() == n
    finally:
        sk.skel_load_dispatch_table(None)
