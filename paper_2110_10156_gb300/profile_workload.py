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


STAGE_OF = {"k_resample": "resample", "k_mask_counts": "resample", "k_fwd_x": "fwd_x",
            "k_fwd_y": "fwd_y", "k_zmac": "zmac", "k_inv_y": "inv_y", "k_inv_x": "inv_x"}


def _stage_bytes(csv_paths) -> dict:
    """{stage: {launch id: DRAM bytes}} over ncu CSV logs (metrics
    dram__bytes_read.sum, dram__bytes_write.sum); in each log the fixed
    volume's own x and y passes, which come before its first resample, are
    left out."""
    import csv

    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "Tbyte": 1e12}

    def stage_of(name):
        head = name.split("(")[0].split("<")[0]
        return next((v for k, v in STAGE_OF.items() if head == k or head.endswith("::" + k)
                     or head.endswith(" " + k)), None)

    per = {}
    for n, path in enumerate(csv_paths):
        with open(path) as fh:
            lines = [ln for ln in fh if ln.startswith('"')]
        rows = list(csv.DictReader(lines))
        first = min((int(r["ID"]) for r in rows if r.get("Kernel Name", "").split("(")[0].split("<")[0]
                     .endswith("k_resample")), default=0)
        for r in rows:
            stage = stage_of(r.get("Kernel Name", ""))
            if stage is None or int(r["ID"]) < first:
                continue
            if r.get("Metric Name") not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
                continue
            v = float(r["Metric Value"].replace(",", "")) * scale.get(r.get("Metric Unit", "byte"), 1.0)
            key = f"{n}:{r['ID']}"
            per.setdefault(stage, {}).setdefault(key, 0.0)
            per[stage][key] += v
    return per


def traffic_from_csv(csv_paths, rotations: int, out_path: str, precision: str = "fp32",
                     base_paths=None, base_rotations: int = 0, note: str = "", fft=None) -> dict:
    """DRAM bytes of each scoring stage per rotation, from ncu CSV logs of
    launch groups of `rotations` rotations, keyed by the current kernel-source
    hash so a stale file is ignored.  With logs of the same launches at
    `base_rotations` rotations (base_paths), the bytes a launch moves whatever
    its rotation count (the z pass's fixed-spectra tile) are separated:
    per rotation = (B(R) - B(Rb)) / (R - Rb), per launch = B(R) - R * that.

    `fft` names the FFT lengths (Pz, Py, Px) of the captured launches; the file
    keeps one entry per set of lengths, and an entry for other lengths already
    in the file (same source hash and precision) is kept beside the new one."""
    import importlib.util
    import json
    import os

    paths = [csv_paths] if isinstance(csv_paths, str) else list(csv_paths)
    per = _stage_bytes(paths)
    base = _stage_bytes(base_paths) if base_paths else {}
    stages = {}
    for k, v in sorted(per.items()):
        tot = sum(v.values())
        if k in base and base_rotations and rotations != base_rotations:
            pr = (tot - sum(base[k].values())) / (rotations - base_rotations)
            fixed = tot - rotations * pr
        else:
            pr, fixed = tot / rotations, 0.0
        stages[k] = {"launches": len(v), "dram_bytes_per_rotation": pr, "dram_bytes_per_launch_fixed": fixed}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    src_hash = bench.kernel_source_hash()
    entry = {"fft": None if fft is None else [int(x) for x in fft],
             "source": f"ncu dram__bytes_read.sum + dram__bytes_write.sum, launch groups of {rotations} "
                       f"rotations ({', '.join(os.path.basename(p) for p in paths)})" +
                       (f"; per-launch bytes from {base_rotations}-rotation groups" if base else "") +
                       (f"; {note}" if note else ""),
             "stages": stages}
    classes = []
    try:
        with open(out_path) as fh:
            old = json.load(fh)
        if old.get("src_hash") == src_hash and old.get("precision") == precision:
            classes = [c for c in old.get("classes", []) if c.get("fft") != entry["fft"]]
    except (OSError, ValueError):
        pass
    out = {"src_hash": src_hash, "precision": precision, "classes": classes + [entry]}
    with open(out_path, "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")
    return out


def classify_rotations(f, B, MB, quats) -> dict:
    """{(Pz, Py, Px): [rotation indices]}: each rotation scored alone, so that
    the FFT lengths bound-limited padding gives it can be read back."""
    out = {}
    for i in range(len(quats)):
        f.score_rotations(B, MB, quats[i:i + 1])
        (cp, _), = f.length_classes()
        out.setdefault(tuple(cp), []).append(i)
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--traffic-from", nargs="+",
                    help="summarise ncu CSV logs (launch groups of --rotations) into profiles/ncu_traffic.json")
    ap.add_argument("--traffic-base", nargs="+", help="logs of the same launches with --base-rotations")
    ap.add_argument("--base-rotations", type=int, default=0)
    ap.add_argument("--traffic-note", default="", help="what the captures covered (lengths, workload)")
    ap.add_argument("--traffic-out", help="write the summary here instead")
    ap.add_argument("--traffic-fft", help="FFT lengths Pz,Py,Px of the captured launches")
    ap.add_argument("--precision", choices=("fp32", "bf16", "fp16"), default="fp32")
    ap.add_argument("--pad-mode", choices=("bound", "full"), default="bound")
    ap.add_argument("--size", type=int, default=150)
    ap.add_argument("--rotations", type=int, default=2)
    ap.add_argument("--batch", type=int, default=2)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--headline", type=int, default=-1, metavar="FIRST",
                    help="score the 150^3 workload's own pair, rotations FIRST .. FIRST + rotations - 1")
    ap.add_argument("--indices", help="with --headline: score these rotations (comma list) instead of a slice")
    ap.add_argument("--classify", type=int, default=0, metavar="N",
                    help="with --headline: print the FFT lengths of each of rotations FIRST .. FIRST + N - 1")
    ap.add_argument("--tensor-cores", choices=("on", "off"), default="on")
    args = ap.parse_args(argv)
    if args.traffic_from:
        import json
        import os
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        out = traffic_from_csv(args.traffic_from, args.rotations,
                               args.traffic_out or os.path.join(root, "profiles", "ncu_traffic.json"),
                               args.precision, args.traffic_base, args.base_rotations, args.traffic_note,
                               [int(x) for x in args.traffic_fft.split(",")] if args.traffic_fft else None)
        print(json.dumps(out, indent=1))
        return 0

    import torch

    from . import cs_ngf, synth
    n = args.size
    if args.headline >= 0:
        p = synth.config_pair(1)
        if args.indices:
            quats = p.quats[[int(i) for i in args.indices.split(",")]]
        elif args.classify:
            quats = p.quats[args.headline:args.headline + args.classify]
        else:
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
    if args.classify:
        for cp, idx in sorted(classify_rotations(f, B, MB, quats).items()):
            print(f"fft {','.join(map(str, cp))} rotations {len(idx)} indices "
                  f"{','.join(str(args.headline + i) for i in idx)}")
        f.release()
        return 0
    for _ in range(args.repeat):
        sc, sh = f.score_rotations(B, MB, quats)
    torch.cuda.synchronize()
    print(f"dims {p.A.shape} classes {f.length_classes()} batch {f.batch} best {float(sc.max()):.6f}")
    f.release()
    return 0


if __name__ == "__main__":
    sys.exit(main())
