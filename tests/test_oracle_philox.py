"""Pins the oracle's Philox4x32-10 to its published known-answer vectors and
checks the draw contract (uniform in (0, 1], index range, sign balance)."""
import json
import os

import numpy as np


def test_known_answer_vectors(orc, golden_dir):
    with open(os.path.join(golden_dir, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        out = orc.philox([int(x, 16) for x in v["ctr"]], [int(x, 16) for x in v["key"]])
        assert out == [int(x, 16) for x in v["out"]]


def test_counter_and_key_sensitivity(orc):
    base = orc.philox([1, 2, 3, 4], [5, 6])
    for i in range(4):
        c = [1, 2, 3, 4]
        c[i] ^= 1
        assert orc.philox(c, [5, 6]) != base
    assert orc.philox([1, 2, 3, 4], [5, 7]) != base


def test_uniform_words(orc):
    words = np.array([w for t in range(2000) for w in orc.philox([t, 7, 0, 4], [0, 0])], dtype=np.uint64)
    u = ((words >> 8) + 1) / 2.0 ** 24
    assert u.min() > 0.0 and u.max() <= 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs((words & 1).mean() - 0.5) < 0.02
