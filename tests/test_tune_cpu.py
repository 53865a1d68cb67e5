"""The launch-shape table shipped with the package: every entry is keyed like
the tuner's cache and carries a valid shape (host logic, no GPU)."""
import json
import os
import re

import pytest

tune = pytest.importorskip("paper_2101_06192_gb300.tune")


def test_shipped_table_entries():
    with open(tune._SHIPPED) as f:
        table = json.load(f)
    assert table
    for key, e in table.items():
        assert re.fullmatch(r"n\d+_d\d+_w[01]_a\d+_t\d+_k[0-2]", key), key
        assert e["order"] in ("degree", "id", "auto")
        assert e["regs"] in (0, 40, 48, 64)
        assert e["walkers"] == 0 or (32 <= e["walkers"] <= 1024 and e["walkers"] % 32 == 0)


def test_key_matches_benchmark_class():
    class G:  # the benchmark graph's sizes (BA n = 2^20, m = 8)
        n, nnz, weighted, n_alpha, kernel_pref = 1 << 20, 16775658, False, 1, 0
    assert tune._key(G, 1024) in tune._load(tune._SHIPPED)
