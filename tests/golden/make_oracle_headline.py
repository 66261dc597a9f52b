"""Writes tests/golden/oracle_headline_150cubed.json: for every one of the
1000 rotations of the seeded 150^3 pair (40 ellipsoids, thresholded masks,
320^3 full linear padding), the FP64 oracle's best score s1 and its shift,
the best score s2 outside the 3x3x3 neighbourhood of that shift, the largest
|score| over the valid shifts, and the number of valid shifts.

These are what the argmax parity rule needs (Section 3.2: argmax over the
shifts, then the maximum over rotations, Fig. 1): a rotation whose gap
s1 - s2 exceeds 2 tau s1 must come back with exactly this shift, and the
rotation with the largest s1 must be the alignment when its gap to every
other candidate exceeds 2 tau s1.

Calls only oracle/ (and the seeded input generator, which holds none of the
method's arithmetic).  Rotations run one per process in a spawn pool over
the host's cores (about 10 minutes on 8 cores).

    python tests/golden/make_oracle_headline.py [--procs N] [--limit R]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "oracle_headline_150cubed.json")
PAD = (320, 320, 320)

_PAIR = None


def _init():
    global _PAIR
    from paper_2110_10156_gb300 import synth
    _PAIR = synth.config_pair(1)


def summarise(score_map):
    """(s1, chi1, s2, scale, n_valid) of one oracle map (tie rule of best_of_map)."""
    import numpy as np
    from oracle import cs_ngf_oracle as O
    fin = np.isfinite(score_map)
    n_valid = int(fin.sum())
    if n_valid == 0:
        return float("-inf"), (0, 0, 0), float("-inf"), 0.0, 0
    s1, chi1 = O.best_of_map(score_map)
    dims = tuple((s + 1) // 2 for s in score_map.shape)
    idx = tuple(c + n - 1 for c, n in zip(chi1, dims))
    rest = score_map.copy()
    rest[~fin] = -np.inf
    rest[tuple(slice(max(0, i - 1), i + 2) for i in idx)] = -np.inf
    s2 = float(rest.max())
    scale = float(np.max(np.abs(score_map[fin])))
    return s1, chi1, s2, scale, n_valid


def one(r):
    from oracle import cs_ngf_oracle as O
    p = _PAIR
    smap, _ = O.score_map(p.A, p.MA, p.B, p.MB, p.quats[r], pad=PAD)
    s1, chi1, s2, scale, n_valid = summarise(smap)
    return r, s1, [int(v) for v in chi1], s2, scale, n_valid


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=len(os.sched_getaffinity(0)))
    ap.add_argument("--limit", type=int, default=0, help="first R rotations only (for a trial)")
    args = ap.parse_args()
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    from paper_2110_10156_gb300 import synth
    p = synth.config_pair(1)
    R = len(p.quats) if args.limit <= 0 else min(args.limit, len(p.quats))
    t0 = time.time()
    rows = [None] * R
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs, initializer=_init) as pool:
        for k, res in enumerate(pool.imap_unordered(one, range(R))):
            rows[res[0]] = res[1:]
            if (k + 1) % 50 == 0:
                print(f"{k + 1}/{R} rotations, {time.time() - t0:.0f} s", flush=True)
    s1 = [r[0] for r in rows]
    best = max(range(R), key=lambda i: (s1[i], -i))
    doc = {
        "about": "FP64 oracle (FFT form, Eq. 6-8, full linear padding 320^3) on the seeded 150^3 pair, "
                 "every rotation; s2 = best score outside the 3x3x3 neighbourhood of the best shift; "
                 "written by tests/golden/make_oracle_headline.py",
        "input": "paper_2110_10156_gb300.synth.config_pair(1)",
        "eps": 1e-5, "gamma": 0.5, "pad": list(PAD),
        "rotations": R, "true_index": int(p.true_index), "t_zyx": list(p.t_zyx),
        "best_rotation": int(best),
        "s1": [float(r[0]) for r in rows],
        "shift": [r[1] for r in rows],
        "s2": [float(r[2]) for r in rows],
        "scale": [float(r[3]) for r in rows],
        "n_valid": [int(r[4]) for r in rows],
        "host_seconds": round(time.time() - t0, 1),
        "host_procs": int(args.procs),
    }
    with open(OUT, "w") as fh:
        json.dump(doc, fh, separators=(",", ":"))
        fh.write("\n")
    print(OUT, f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
