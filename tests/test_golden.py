"""Regression fixture: the oracle's outputs on a tiny seeded workload must not
drift (fixture written by tests/golden/make_golden.py, oracle only)."""
import json
import os

import numpy as np

from tests.golden.make_golden import tiny_case

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_golden_fixture():
    with open(os.path.join(HERE, "golden", "oracle_tiny.json")) as f:
        g = json.load(f)
    d, idx, qr, x, x0 = tiny_case()
    assert [[format(int(v), "016x") for v in r] for r in idx.keys[:20]] == g["dict_keys_hex"]
    assert [[format(int(v), "016x") for v in r] for r in qr.keys[:20]] == g["query_keys_hex"]
    assert qr.nbr.tolist() == g["nbr"]
    np.testing.assert_allclose(qr.wgt, g["wgt"], atol=1e-11)
    np.testing.assert_allclose(x0, g["hr_before_bp"], atol=1e-11)
    np.testing.assert_allclose(x, g["hr"], atol=1e-11)
