"""Writes tests/golden/oracle_regression_32cubed.json: the FP64 oracle's best
score and shift per rotation on the seeded 32^3 pair (12 ellipsoids, full
masks, 8 rotations: the true one, the identity and 6 uniform).

Calls only oracle/ (and the seeded input generator, which holds none of the
method's arithmetic).  The stored values guard the oracle against unintended
change; regenerate them only with a change to the oracle whose commit message
names the passage of the paper that justifies it.

    python tests/golden/make_oracle_regression.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_regression_32cubed.json")


def compute():
    from oracle import cs_ngf_oracle as O
    from paper_2110_10156_gb300 import synth
    p = synth.config_pair(0)
    scores, shifts = O.score_rotations(p.A, p.MA, p.B, p.MB, p.quats)
    return {
        "about": "FP64 oracle (FFT form, Eq. 6-8, full linear padding) on the seeded 32^3 pair; "
                 "written by tests/golden/make_oracle_regression.py",
        "input": "paper_2110_10156_gb300.synth.config_pair(0)",
        "eps": 1e-5, "gamma": 0.5,
        "scores": [float(s) for s in scores],
        "shifts": [[int(v) for v in c] for c in shifts],
    }


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(compute(), fh, indent=1)
        fh.write("\n")
    print(OUT)
