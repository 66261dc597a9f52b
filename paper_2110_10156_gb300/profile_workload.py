"""Small, self-contained workload for kernel profiling (ncu) of the scoring path.

    python -m paper_2110_10156_gb300.profile_workload --size 150 --rotations 2 --batch 2
    python -m paper_2110_10156_gb300.profile_workload --headline 0 --rotations 4 --batch 4

Builds a seeded synthetic pair of the given cube size (the 150^3 generator
recipe scaled), or takes the 150^3 workload's own pair and a slice of its
rotations (--headline), prepares the fixed spectra and scores the rotations
once, so that a profiler sees one launch of every kernel per batch with only
a few GB held on the device.
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


STAGE_OF = {"k_resample": "resample", "k_fwd_x": "fwd_x", "k_fwd_y": "fwd_y", "k_zmac": "zmac",
            "k_inv_y": "inv_y", "k_inv_x": "inv_x"}


def traffic_from_csv(csv_path: str, rotations: int, out_path: str, precision: str = "fp32") -> dict:
    """DRAM bytes per rotation of each scoring stage from an ncu CSV log of one
    scored group (metrics dram__bytes_read.sum, dram__bytes_write.sum), keyed by
    the current kernel-source hash so a stale file is ignored."""
    import csv
    import json
    import os

    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}
    per = {}
    with open(csv_path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    rows = list(csv.DictReader(lines))

    def stage_of(name):
        head = name.split("(")[0].split("<")[0]
        return next((v for k, v in STAGE_OF.items() if head == k or head.endswith("::" + k)
                     or head.endswith(" " + k)), None)

    # the fixed volume's own x and y passes come before the first resample
    first = min((int(r["ID"]) for r in rows if stage_of(r.get("Kernel Name", "")) == "resample"),
                default=0)
    for r in rows:
        stage = stage_of(r.get("Kernel Name", ""))
        if stage is None or int(r["ID"]) < first:
            continue
        if r.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(r["Metric Value"].replace(",", "")) * scale.get(r.get("Metric Unit", "byte"), 1.0)
        per.setdefault(stage, {}).setdefault(r["ID"], 0.0)
        per[stage][r["ID"]] += v
    import importlib.util
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    out = {"src_hash": bench.kernel_source_hash(), "precision": precision,
           "source": f"ncu dram__bytes_read.sum + dram__bytes_write.sum, {rotations} rotations "
                     f"in one launch group ({os.path.basename(csv_path)})",
           "stages": {k: {"launches": len(v), "dram_bytes_per_rotation": sum(v.values()) / rotations}
                      for k, v in sorted(per.items())}}
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--traffic-from", help="summarise an ncu CSV log into profiles/ncu_traffic.json")
    ap.add_argument("--traffic-out", help="write the summary here instead")
    ap.add_argument("--precision", choices=("fp32", "bf16", "fp16"), default="fp32")
    ap.add_argument("--pad-mode", choices=("bound", "full"), default="bound")
    ap.add_argument("--size", type=int, default=150)
    ap.add_argument("--rotations", type=int, default=2)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--headline", type=int, default=-1, metavar="FIRST",
                    help="score the 150^3 workload's own pair, rotations FIRST .. FIRST + rotations - 1")
    ap.add_argument("--tensor-cores", choices=("on", "off"), default="on")
    args = ap.parse_args(argv)
    if args.traffic_from:
        import json
        import os
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        out = traffic_from_csv(args.traffic_from, args.rotations,
                               args.traffic_out or os.path.join(root, "profiles", "ncu_traffic.json"),
                               args.precision)
        print(json.dumps(out, indent=1))
        return 0

    import torch

    from . import cs_ngf, synth
    n = args.size
    if args.headline >= 0:
        p = synth.config_pair(1)
        quats = p.quats[args.headline:args.headline + args.rotations]
    else:
        p = synth.make_pair(1001, (n, n, n), max(4, int(40 * n / 150)), max(2.0, 5 * n / 150),
                            max(3.0, 30 * n / 150), 30.0, max(1, int(20 * n / 150)),
                            args.rotations, masks="threshold")
        quats = p.quats
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f = cs_ngf.prepare_fixed(dev(p.A), dev(p.MA), batch=args.batch, precision=args.precision,
                             pad_mode=args.pad_mode, tensor_cores=args.tensor_cores == "on")
    B, MB = dev(p.B), dev(p.MB)
    for _ in range(args.repeat):
        sc, sh = f.score_rotations(B, MB, quats)
    torch.cuda.synchronize()
    print(f"dims {p.A.shape} classes {f.length_classes()} batch {f.batch} best {float(sc.max()):.6f}")
    f.release()
    return 0


if __name__ == "__main__":
    sys.exit(main())
