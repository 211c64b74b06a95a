"""Regression fixtures of the oracle (written by tests/golden/make_golden.py,
which calls only the oracle).  A change to the oracle's arithmetic fails here."""
import importlib.util
import os

import numpy as np
import pytest

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
mg = importlib.util.module_from_spec(spec)
spec.loader.exec_module(mg)


@pytest.mark.parametrize("name,arr", list(mg.cases()), ids=lambda v: v if isinstance(v, str) else "")
def test_oracle_matches_frozen_fixture(name, arr):
    path = os.path.join(HERE, name + ".txt")
    ref = np.array([float(l) for l in open(path) if not l.startswith("#")])
    assert np.array_equal(np.asarray(arr, dtype=np.float64), ref)
