"""Writes tests/golden/oracle_tiny.json: the oracle's outputs on a tiny seeded
workload (regression fixture).  Calls only the oracle and the seeded input
generator.  Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth_inputs as S  # noqa: E402
from oracle import zoom_oracle as O  # noqa: E402


def tiny_case():
    s, P, L, k, K, w = 2, 3, 4, 3, 4, 4.0
    train = [S.make_image(900 + i, 32, 32) for i in range(2)]
    pos = S.sample_positions(5, 2, 16, 16, P, 300)
    d = O.build_dictionary(train, pos, s, P, 0.8)
    alpha, beta = S.lsh_draws(6, L, k, P * P, w)
    idx = O.build_index(d, alpha, beta, w, L, k)
    lr = S.make_image(901, 12, 12)
    x, qr, x0 = O.upscale(lr, d, idx, K, 1e-3, 2, 0.8, 1.5, 0.1, 3)
    return d, idx, qr, x, x0


def main():
    d, idx, qr, x, x0 = tiny_case()
    out = {
        "what": "oracle outputs on the tiny seeded workload of tests/golden/make_golden.py",
        "dict_keys_hex": [[format(int(v), "016x") for v in row] for row in idx.keys[:20]],
        "query_keys_hex": [[format(int(v), "016x") for v in row] for row in qr.keys[:20]],
        "nbr": qr.nbr.tolist(),
        "wgt": qr.wgt.round(12).tolist(),
        "hr_before_bp": x0.round(12).tolist(),
        "hr": x.round(12).tolist(),
    }
    with open(os.path.join(ROOT, "tests", "golden", "oracle_tiny.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
