"""Small, self-contained workload for kernel profiling (ncu) of the scoring path.

    python -m paper_2110_10156_gb300.profile_workload --size 150 --rotations 2 --batch 2

Builds a seeded synthetic pair of the given cube size (the 150^3 generator
recipe scaled), prepares the fixed spectra and scores the requested number of
rotations once, so that a profiler sees one launch of every kernel per batch
with only a few GB held on the device.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--size", type=int, default=150)
    ap.add_argument("--rotations", type=int, default=2)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args(argv)

    import torch

    from . import cs_ngf, synth
    n = args.size
    p = synth.make_pair(1001, (n, n, n), max(4, int(40 * n / 150)), max(2.0, 5 * n / 150),
                        max(3.0, 30 * n / 150), 30.0, max(1, int(20 * n / 150)),
                        args.rotations, masks="threshold")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f = cs_ngf.prepare_fixed(dev(p.A), dev(p.MA), batch=args.batch)
    B, MB = dev(p.B), dev(p.MB)
    for _ in range(args.repeat):
        sc, sh = f.score_rotations(B, MB, p.quats)
    torch.cuda.synchronize()
    print(f"dims {p.A.shape} pad {f.pad} batch {f.batch} best {float(sc.max()):.6f}")
    f.release()
    return 0


if __name__ == "__main__":
    sys.exit(main())
