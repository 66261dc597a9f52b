"""The stored per-rotation oracle results of the 150^3 workload
(tests/golden/oracle_headline_150cubed.json, written by
tests/golden/make_oracle_headline.py from the oracle alone) are the oracle's:
one rotation is recomputed here, and the file's own structure is checked."""
import json
import os

import numpy as np

from paper_2110_10156_gb300 import synth
from tests.golden import make_oracle_headline as M

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_headline_150cubed.json")


def test_headline_golden_structure():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    R = d["rotations"]
    assert R == 1000 and d["pad"] == [320, 320, 320]
    for k in ("s1", "s2", "scale", "n_valid", "shift"):
        assert len(d[k]) == R
    s1 = np.array(d["s1"])
    assert d["best_rotation"] == int(np.argmax(s1))
    assert np.all(np.array(d["s2"]) <= s1) and np.all(s1 <= np.array(d["scale"]) + 1e-15)
    assert np.all((s1 >= 0) & (s1 <= 1))
    # the generator's truth is the oracle's maximum over rotations (Fig. 1)
    assert d["best_rotation"] == d["true_index"] and d["shift"][d["true_index"]] == d["t_zyx"]


def test_headline_golden_recomputes_true_rotation():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    M._PAIR = synth.config_pair(1)
    r = d["true_index"]
    _, s1, chi, s2, scale, n_valid = M.one(r)
    assert abs(s1 - d["s1"][r]) <= 1e-12 and chi == d["shift"][r]
    assert abs(s2 - d["s2"][r]) <= 1e-12 and abs(scale - d["scale"][r]) <= 1e-12
    assert n_valid == d["n_valid"][r]
