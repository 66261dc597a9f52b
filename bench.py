#!/usr/bin/env python
"""All-shift NGF scoring benchmark (Cross-Sim-NGF hot path) on GB300.

One step = one global alignment job on the 150^3 synthetic pair: recompute the
fixed-volume spectra (cs_ngf_update_fixed) and score 1000 candidate rotations
for every shift on a 320^3 FFT grid, then take the maximum over rotations
(cs_ngf_align).  value = rotations / s over the whole job.

    python bench.py [--gpus N --steps K --warmup W] [--impl ours|reference]

Multi-GPU (torchrun): rotations are independent, so each rank scores its own
1000 rotations (weak scaling) with no collective on the data path; the
elapsed time is the max over ranks.  --impl reference times the FP64 CPU
oracle on the host cores (the only other place this script runs it).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "150³ rotations/s (all-shift s_ANGF maps) BF16 vs FP32; p50/p99 job latency"
UNIT = "rotations/s"
WORKLOAD = "150^3 float32 synthetic pair, 1000 rotations, FP32"


# ------------------------------------------------------------------ inputs
def load_pair(config: int, n_rot: int):
    """Seeded synthetic pair, cached in the temp dir (generation takes ~20 s)."""
    from paper_2110_10156_gb300 import synth
    key = f"cs_ngf_pair_c{config}_r{n_rot}_v1.npz"
    path = os.path.join(tempfile.gettempdir(), key)
    if os.path.exists(path):
        try:
            d = np.load(path)
            return {k: d[k] for k in d.files}
        except Exception:
            pass
    p = synth.config_pair(config, n_rot=n_rot)
    d = dict(A=p.A, MA=p.MA, B=p.B, MB=p.MB, quats=p.quats,
             true_index=np.array(p.true_index), t_zyx=np.array(p.t_zyx))
    try:
        np.savez(path + ".tmp.npz", **d)
        os.replace(path + ".tmp.npz", path)
    except OSError:
        pass
    return d


def rank_quats(pair, rank: int, n_rot: int):
    """Rank 0 scores the workload's own rotations; other ranks score their own
    seeded uniform rotations (weak scaling: more candidates per job)."""
    if rank == 0:
        return pair["quats"]
    from paper_2110_10156_gb300 import synth
    return synth.random_quaternions(np.random.default_rng(7000 + rank), n_rot)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ byte model
def stage_bytes(dims, pad, nb, stage, nch=3, precision="fp32"):
    """Algorithmic HBM bytes of one launch that scores nb rotations.

    nch packed channel fields per rotation (3 for the squared measure; BF16 or
    FP32 storage) plus one mask field per pair of rotations (FP32).  The z pass
    counts its field reads, the fixed-spectra tile it loads once per launch and
    its output F2, min(2n - 1, P) planes of Z = X + iY per rotation (the z
    inverse writes only the planes the slab bound admits, so this is an upper
    bound; "zmac_no_f2" leaves F2 out, a lower bound).  The inverse passes are
    counted unpruned (an upper bound)."""
    nz, ny, nx = dims
    Pz, Py, Px = pad
    vz, vy = 2 * nz - 1, 2 * ny - 1
    nvox = nz * ny * nx
    cb = 8 if precision == "fp32" else 4
    per_elem = nch * nb * cb + ((nb + 1) // 2) * 8     # bytes per element position, all fields
    F0 = per_elem * nz * ny * Px
    F1 = per_elem * nz * Px * Py
    F2 = min(vz, Pz) * Px * Py * 8
    F3 = min(vz, Pz) * min(vy, Py) * Px * 8
    UV = (2 * nch + 1) * (Px // 2 + 1) * Py * Pz * 8
    return {
        "resample": nb * nvox * 5,
        "fwd_x": nb * nvox * 5 + F0,
        "fwd_y": F0 + F1,
        "zmac": F1 + UV + nb * F2,
        "zmac_no_f2": F1 + UV,
        "inv_y": nb * (F2 + F3),
        "inv_x": nb * F3,
    }.get(stage, 0)


PADDING = {
    "bound": "bound-limited: per call the shortest FFT lengths that keep every shift the "
             "Section 3.2 overlap bound admits alias-free (same scores as the full length)",
    "full": "full linear correlation, 2n-1 per axis",
}


def zmac_flops(dims, pad, nb, nch=3):
    """Algorithmic flops of one z-pass launch over nb rotations: 5 L log2 L per
    complex length-L transform (when the forward input is zero past L/2 that
    prunes the first radix-2 stage: 5 L (log2 L - 1) + L), for nch channel
    fields plus one mask field per pair of rotations over every (kx, ky)
    column, one inverse per column, and the spectral multiply-accumulate over
    the kx <= Px/2 half (16 flops per channel field, 20 for the mask pair)."""
    Pz, Py, Px = pad
    L = Pz
    lg = math.log2(L)
    fwd = 5 * L * (lg - 1) + L if 2 * dims[0] <= L else 5 * L * lg
    inv = 5 * L * lg
    cols = Px * Py
    fields = nch * nb + (nb + 1) // 2
    mac = (Px // 2 + 1) * Py * Pz * (16 * nch + 20) * nb
    return fields * cols * fwd + nb * cols * inv + mac


FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


_SOURCE_HASH = {}


def kernel_source_hash():
    """Hash of the sources the scoring kernels and their launches are built
    from (the serving loop, search driver and allocation-free entry point are
    left out: they launch the same kernels); computed once per process."""
    if ROOT in _SOURCE_HASH:
        return _SOURCE_HASH[ROOT]
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_10156_gb300", "csrc")
    keep = ("fft_core.cuh", "kernels.cuh", "passes.cuh", "elem.cu", "cs_ngf.cu", "handle.h",
            "tc.cuh", "zmac_tc.cuh")
    for fn in sorted(os.listdir(csrc)):
        if fn in keep or (fn.startswith("passes_") and fn.endswith(".cu")):
            with open(os.path.join(csrc, fn), "rb") as fh:
                h.update(fh.read())
    _SOURCE_HASH[ROOT] = h.hexdigest()[:16]
    return _SOURCE_HASH[ROOT]


def ncu_traffic(stage: str, precision: str = "fp32", dims=None, pad=None):
    """(DRAM bytes per rotation, DRAM bytes every launch moves whatever its
    rotation count) for a stage at FFT lengths `pad`, from the committed ncu
    summary, if it was taken on the current kernel sources in the same
    precision; else None.  Lengths the summary has no capture of take the
    captured class nearest in grid points, scaled by the byte model's ratio
    between the two (per rotation: the launch's bytes at one rotation less the
    per-launch tile; per launch: the fixed-spectra tile's size)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except Exception:
        return None
    if d.get("src_hash") != kernel_source_hash() or d.get("precision", "fp32") != precision:
        return None
    classes = [c for c in d.get("classes", []) if stage in c.get("stages", {})]
    if not classes:
        return None
    exact = [c for c in classes if pad is not None and c.get("fft") == list(pad)]
    if exact or pad is None or dims is None or any(c.get("fft") is None for c in classes):
        e = (exact or classes)[0]["stages"][stage]
        return float(e["dram_bytes_per_rotation"]), float(e.get("dram_bytes_per_launch_fixed", 0.0))
    npts = lambda q: q[0] * q[1] * q[2]
    c = min(classes, key=lambda c: abs(npts(c["fft"]) - npts(pad)))
    e, cap = c["stages"][stage], tuple(c["fft"])
    one = lambda q: stage_bytes(dims, q, 1, stage, precision=precision) - stage_bytes(dims, q, 0, stage, precision=precision)
    tile = lambda q: stage_bytes(dims, q, 0, stage, precision=precision)
    pr = float(e["dram_bytes_per_rotation"]) * (one(pad) / one(cap) if one(cap) else 1.0)
    fx = float(e.get("dram_bytes_per_launch_fixed", 0.0)) * (tile(pad) / tile(cap) if tile(cap) else 1.0)
    return pr, fx


def launch_traffic(stage: str, precision: str, dims, launches_of):
    """ncu DRAM bytes of a stage summed over the launches of one step, each
    launch (lengths, rotations) at its own class's figures; None without a
    current summary."""
    tot = 0.0
    for cp, nb in launches_of:
        t = ncu_traffic(stage, precision, dims, cp)
        if t is None:
            return None
        tot += t[1] + t[0] * nb
    return tot


# ------------------------------------------------------------------ CPU oracle
def _oracle_one(args):
    A, MA, B, MB, q = args
    from oracle import cs_ngf_oracle as O
    s, _ = O.score_map(A, MA, B, MB, q)
    return O.best_of_map(s)


def _warm(_):
    from oracle import cs_ngf_oracle  # noqa: F401
    return 0


def oracle_sample(pair, n_rot: int, cores: int):
    """Time the FP64 oracle as it stands on the first n_rot rotations, one per
    process.  Returns (rotations/s, seconds, [(best score, best shift)])."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    qs = pair["quats"][:n_rot]
    args = [(pair["A"], pair["MA"], pair["B"], pair["MB"], q) for q in qs]
    with ctx.Pool(cores) as pool:
        pool.map(_warm, range(cores))                  # workers up and oracle imported
        t0 = time.perf_counter()
        best = pool.map(_oracle_one, args, chunksize=1)
        dt = time.perf_counter() - t0
    return n_rot / dt, dt, best


def compare_with_oracle(gpu_score, gpu_shift, oracle_best):
    """The GPU's per-rotation results against the oracle's on the rotations
    the CPU leg scored: the largest score difference where both found a valid
    shift, and how many rotations got the oracle's exact shift (both invalid
    counts as agreement).  Reported only; the parity tests hold the bar."""
    n = len(oracle_best)
    err, same, valid_mismatch = 0.0, 0, 0
    for i, (o_s, o_chi) in enumerate(oracle_best):
        g_s = float(gpu_score[i])
        g_ok, o_ok = math.isfinite(g_s), math.isfinite(o_s)
        if g_ok != o_ok:
            valid_mismatch += 1
            continue
        if not g_ok:
            same += 1
            continue
        err = max(err, abs(g_s - o_s))
        same += int(tuple(int(v) for v in gpu_shift[i]) == tuple(int(v) for v in o_chi))
    return {"rotations": n, "max_abs_score_err": err, "same_shift": same,
            "validity_mismatch": valid_mismatch,
            "oracle": "FP64 FFT form at the full linear length, first rotations of the workload"}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# ------------------------------------------------------------------ arms
def l2_note(roofline_step, R, batch):
    if roofline_step is not None:
        tb = roofline_step["dram_bytes_per_rotation"] * R / 1e12
        return (f"inputs larger than L2: each launch group's FFT intermediates exceed the 129 MB L2; "
                f"about {tb:.2f} TB of DRAM traffic per step (ncu bytes per rotation x {R})")
    return ("inputs larger than L2: each launch group's FFT intermediates "
            f"({batch} rotations) exceed the 129 MB L2")


def time_form(cs_ngf, A, MA, B, MB, quats, precision, args, fp32_value, tensor_cores=True):
    """One precision form on the headline workload: the same step, warm-up and
    timed steps (CUDA events on the launching stream) as the FP32 line, then
    one scoring call for the per-rotation results.  Returns (summary dict,
    (scores, shifts) as numpy)."""
    import torch
    g = cs_ngf.prepare_fixed(A, MA, batch=args.batch, precision=precision, pad_mode=args.pad_mode,
                             autotune=args.autotune == "on", tensor_cores=tensor_cores)

    def step():
        g.update_fixed(A, MA)
        return g.align(B, MB, quats)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    value = len(quats) * args.steps / (ms / 1000.0)
    sc, sh = g.score_rotations(B, MB, quats)
    out = (sc.cpu().numpy(), sh.cpu().numpy())
    summary = {"value": value, "unit": UNIT, "ms_per_step": ms / args.steps,
               "ratio_to_fp32": value / fp32_value, "steps": args.steps,
               "tensor_cores": bool(tensor_cores),
               "storage": f"{precision} channel fields of the forward x and y passes; mask / overlap "
                          "path and everything after the spectral sum FP32",
               "z_pass": ("forward z DFT of the channel fields as tcgen05 MMAs "
                          f"({precision} operands, FP32 accumulation in tensor memory)") if tensor_cores
                         else "CUDA-core FFT (FP32 arithmetic)",
               "result": {"best_rotation": res[1], "shift": list(res[2]), "score": res[0]}}
    g.release()
    return summary, out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    cores = min(host_cores(), 16)
    pair = load_pair(args.config, args.rotations)
    sample = max(1, min(cores, args.ref_sample))
    for _ in range(args.warmup):
        oracle_sample(pair, sample, cores)
    times = []
    for _ in range(args.steps):
        _, dt, _ = oracle_sample(pair, sample, cores)
        times.append(dt)
    total = sum(times)
    value = sample * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * total / args.steps,
        "ms_per_workload_extrapolated": 1000.0 * total / args.steps * (args.rotations / sample),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "volume": [150, 150, 150], "fft": [320, 320, 320],
                   "rotations": args.rotations, "sample_rotations_per_step": sample,
                   "step": f"{sample} rotations of the workload scored by the oracle (one per "
                           "process); ms_per_step is that sample's time"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the {args.rotations} rotations per step, one per "
                                   f"process, FP64 numpy FFT form at 320^3"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2110_10156_gb300 import cs_ngf

    pair = load_pair(args.config, args.rotations)
    quats = rank_quats(pair, rank, args.rotations)
    R = len(quats)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    A, MA, B, MB = dev(pair["A"]), dev(pair["MA"]), dev(pair["B"]), dev(pair["MB"])
    f = cs_ngf.prepare_fixed(A, MA, batch=args.batch, precision=args.precision,
                             pad_mode=args.pad_mode, autotune=args.autotune == "on",
                             tensor_cores=args.tensor_cores == "on")
    dims = f.dims

    def step():
        f.update_fixed(A, MA)
        local = f.align(B, MB, quats)
        if ws > 1:                                  # max over all ranks' rotations (Fig. 1)
            from paper_2110_10156_gb300 import shard
            s, r, sh = local
            return shard.all_merge_best((s, r + rank * R if r >= 0 else -1, sh))
        return local

    for _ in range(args.warmup):
        res = step()
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---------------- device-resident timed region (full launch groups replay
    # one captured CUDA graph each)
    sampler = ClockSampler(local)
    sampler.start()
    l0 = cs_ngf.launch_count()
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = cs_ngf.launch_count() - l0
    clocks = sampler.stop()
    elapsed_ms = e0.elapsed_time(e1)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    value = ws * R * args.steps / (elapsed_ms / 1000.0)

    # ---------------- per-kernel CUDA-event times: one more step with every
    # launch bracketed by events on its stream (direct launches, no graph)
    f.set_profiling(True)
    f.stage_times()
    t0p = time.perf_counter()
    step()
    torch.cuda.synchronize()
    prof_step_ms = 1000.0 * (time.perf_counter() - t0p)
    stages = f.stage_times()
    f.set_profiling(False)
    prof_steps = 1

    # ---------------- end to end through the host-buffer entry point
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hA, hMA = pin(pair["A"]), pin(pair["MA"])
    hB, hMB = pin(pair["B"]).numpy(), pin(pair["MB"]).numpy()
    out_s = torch.empty(R, dtype=torch.float32).pin_memory().numpy()
    out_c = torch.empty((R, 3), dtype=torch.int32).pin_memory().numpy()

    def e2e_step():
        A.copy_(hA, non_blocking=True)
        MA.copy_(hMA, non_blocking=True)
        f.update_fixed(A, MA)
        s, c = f.score_rotations_host(hB, hMB, quats, out_s, out_c)
        return int(np.argmax(s))

    e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    nvox = int(np.prod(dims))
    h2d = 2 * nvox * 5 + R * 36
    d2h = R * 16 + 4

    # ---------------- roofline of the dominant kernel: the model bytes (and
    # flops) of every launch of the profiled step, per class of FFT lengths
    peak, peak_kind = measured_peaks()
    stage_ms = {k: v[0] for k, v in stages.items()}
    dom = max(("resample", "fwd_x", "fwd_y", "zmac", "inv_y", "inv_x"), key=lambda k: stage_ms[k])
    classes = f.length_classes()
    launches_of = [(cp, min(f.batch, cnt - b * f.batch)) for cp, cnt in classes
                   for b in range(-(-cnt // f.batch))]
    nbatches = len(launches_of)
    total_bytes = sum(stage_bytes(dims, cp, nb, dom, precision=args.precision) for cp, nb in launches_of)
    total_bytes *= prof_steps
    achieved = total_bytes / (stage_ms[dom] / 1000.0) / 1e9 if stage_ms[dom] > 0 else 0.0
    tr = launch_traffic(dom, args.precision, dims, launches_of)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_kind": f"{peak_kind} hbm_gbs",
                "kernel": dom,
                "traffic": None if tr is None else tr / nbatches,
                "algorithmic_bytes_per_launch": total_bytes / (prof_steps * nbatches),
                "timing": "CUDA events around every launch of one profiled step after the timed region"}
    if dom == "zmac":               # the same without the F2 writes (a lower bound)
        lo = sum(stage_bytes(dims, cp, nb, "zmac_no_f2", precision=args.precision)
                 for cp, nb in launches_of) * prof_steps
        ach_lo = lo / (stage_ms[dom] / 1000.0) / 1e9 if stage_ms[dom] > 0 else 0.0
        roofline.update({"achieved_without_f2": ach_lo, "frac_without_f2": ach_lo / peak,
                         "model": "F1 read + F2 write (min(2n-1, P) planes) + fixed tile per launch"})

    # the whole step against HBM: the ncu DRAM bytes per rotation of every
    # scoring stage (same kernel sources and precision only), times the
    # rotations, over the timed step
    step_bytes = [launch_traffic(st, args.precision, dims, launches_of)
                  for st in ("resample", "fwd_x", "fwd_y", "zmac", "inv_y", "inv_x")]
    roofline_step = None
    if all(b is not None for b in step_bytes):
        per_rot = sum(step_bytes) / R
        ach = per_rot * R / (elapsed_ms / args.steps / 1000.0) / 1e9
        roofline_step = {"bound": "hbm", "dram_bytes_per_rotation": per_rot, "achieved": ach,
                         "peak": peak, "unit": "GB/s", "frac": ach / peak,
                         "note": "ncu DRAM bytes of all scoring stages per rotation x rotations / step time"}

    roofline_alu = None
    if dom == "zmac":
        fl = sum(zmac_flops(dims, cp, nb) for cp, nb in launches_of) * prof_steps
        ach = fl / (stage_ms[dom] / 1000.0) / 1e12 if stage_ms[dom] > 0 else 0.0
        roofline_alu = {"bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                        "frac": ach / FP32_ALU_PEAK_TFLOPS, "kernel": dom,
                        "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                        "flops_per_launch": fl / (prof_steps * nbatches)}

    # ---------------- the reduced-precision forms on the same workload and
    # launch configuration (ratio to the FP32 value above)
    forms, form_results = {}, {}
    if ws == 1 and args.precision == "fp32" and not args.no_forms:
        fs = ClockSampler(local)
        fs.start()
        for prec in ("bf16", "fp16"):
            forms[prec], form_results[prec] = time_form(cs_ngf, A, MA, B, MB, quats, prec, args, value)
        # the same BF16 form with the z pass on the CUDA cores, for comparison
        forms["bf16_cuda_cores"], _ = time_form(cs_ngf, A, MA, B, MB, quats, "bf16", args, value,
                                                tensor_cores=False)
        fclk = fs.stop()
        for prec in forms:
            forms[prec]["clocks"] = fclk

    cpu = None
    oracle_check = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cores = min(host_cores(), 16)
        sample = max(1, min(cores, args.ref_sample))
        v, dt, best = oracle_sample(pair, sample, cores)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{sample} of the {R} rotations, one per process, FP64 numpy FFT "
                         f"form at 320^3 ({dt:.1f} s wall)"}
        try:                      # out_s, out_c: the last host-buffer step's per-rotation results
            oracle_check = compare_with_oracle(out_s, out_c, best)
        except Exception as exc:  # reporting only: never fails the run
            oracle_check = {"error": repr(exc)}
        for prec, (fsc, fsh) in form_results.items():
            try:
                forms[prec]["oracle_check"] = compare_with_oracle(fsc, fsh, best)
            except Exception as exc:
                forms[prec]["oracle_check"] = {"error": repr(exc)}
    f.release()

    serving = None
    if rank == 0 and ws == 1 and not args.no_serving:
        serving = {prec: serving_measure(args, prec) for prec in ("fp32", "bf16")}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else f"f32 arithmetic, {args.precision} channel intermediates",
            "data": "synthetic",
            "config": {"workload": WORKLOAD if args.precision == "fp32" else WORKLOAD.replace("FP32", f"{args.precision.upper()} form"), "volume": list(dims),
                       "fft": list(max(classes, key=lambda c: c[1])[0]),
                       "padding": PADDING[args.pad_mode], "fft_full_linear": list(f.max_pad),
                       "fft_classes": [{"fft": list(cp), "rotations": n} for cp, n in classes],
                       "autotune": args.autotune == "on",
                       "splits": [{"stage": e["stage"], "length": e["length"],
                                   "split": list(e["splits"][e["variant"]]),
                                   "ms": [round(v, 3) for v in e["ms"]]} for e in cs_ngf.tuning()],
                       "rotations_per_gpu": R, "batch": f.batch, "masks": "thresholded foreground",
                       "l2": l2_note(roofline_step, R, f.batch),
                       "step": "update_fixed + score all rotations + max over rotations"},
            "roofline": roofline, "roofline_alu": roofline_alu, "roofline_step": roofline_step,
            "cpu_baseline": cpu,
            "oracle_check": oracle_check,
            "e2e": {"value": ws * R * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "stages_ms_per_step": {k: v / prof_steps for k, v in stage_ms.items()},
            "profiled_step_ms": prof_step_ms,
            "result": {"best_rotation": res[1], "shift": list(res[2]), "score": res[0]},
            "forms": forms or None,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ other workloads
def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_small_latency(args):
    """32^3 pair, 8 rotations (64^3 FFT): alignment latency, one job at a time."""
    import torch
    from paper_2110_10156_gb300 import cs_ngf
    pair = load_pair(0, 8)
    A, MA, B, MB = (_dev(pair[k]) for k in ("A", "MA", "B", "MB"))
    f = cs_ngf.prepare_fixed(A, MA)
    q = pair["quats"]
    for _ in range(max(3, args.warmup)):
        f.update_fixed(A, MA)
        f.align(B, MB, q)
    lat = []
    for _ in range(max(20, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f.update_fixed(A, MA)
        res = f.align(B, MB, q)
        lat.append(1000.0 * (time.perf_counter() - t0))
    lat = np.array(lat)
    print(json.dumps({
        "metric": "32^3 alignment latency (8 rotations, all shifts, 64^3 FFT)", "unit": "ms",
        "value": float(np.median(lat)), "p99_ms": float(np.percentile(lat, 99)),
        "rotations_per_s": float(8 / (np.median(lat) / 1000.0)), "higher_is_better": False,
        "dtype": "f32", "data": "synthetic", "config": {"workload": "32^3 pair, 8 rotations", "fft": list(f.pad)},
        "result": {"best_rotation": res[1], "shift": list(res[2]), "score": res[0]}}), flush=True)
    f.release()
    return 0


def run_large(args):
    """256^3 pair (full linear length 512 per axis; bound-limited padding takes
    400 or 320): rotations/s in the precision asked for (memory-sized
    batches)."""
    import torch
    from paper_2110_10156_gb300 import cs_ngf
    R = args.rotations if args.rotations != 1000 else 5000
    pair = load_pair(4, R)
    A, MA, B, MB = (_dev(pair[k]) for k in ("A", "MA", "B", "MB"))
    f = cs_ngf.prepare_fixed(A, MA, batch=args.batch, precision=args.precision,
                             pad_mode=args.pad_mode, tensor_cores=args.tensor_cores == "on")
    q = pair["quats"]
    f.update_fixed(A, MA)
    f.align(B, MB, q[: 2 * f.batch])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f.update_fixed(A, MA)
    res = f.align(B, MB, q)
    dt = time.perf_counter() - t0
    print(json.dumps({
        "metric": "256^3 rotations/s (all-shift maps)", "unit": UNIT, "value": R / dt,
        "higher_is_better": True, "dtype": "f32", "precision": args.precision, "data": "synthetic",
        "config": {"workload": f"256^3 pair, {R} rotations, {args.precision.upper()}",
                   "padding": PADDING[args.pad_mode],
                   "fft_classes": [{"fft": list(cp), "rotations": n} for cp, n in f.length_classes()],
                   "batch": f.batch,
                   "device_bytes": f.fixed_bytes + f.workspace_bytes},
        "seconds": dt,
        "result": {"best_rotation": res[1], "shift": list(res[2]), "score": res[0],
                   "true_rotation": int(pair["true_index"]), "true_shift": [int(v) for v in pair["t_zyx"]]}}),
          flush=True)
    f.release()
    return 0


def run_tab3(args):
    """One all-shift CSNGF evaluation on cube pairs of side 8..128 (both
    volumes' transforms, the sum in the spectrum, the inverse, the
    normalisation and the argmax): GPU path time, and the CPU direct
    algorithm (Section 5.2) timed where it finishes in seconds."""
    import torch
    from oracle import cs_ngf_oracle as O
    from paper_2110_10156_gb300 import cs_ngf, synth
    rows = []
    ident = np.array([[1.0, 0.0, 0.0, 0.0]])
    for n in (8, 16, 32, 64, 128):
        p = synth.small_pair(500 + n, (n, n, n), n_rot=1, masks="full")
        A, MA, B, MB = (_dev(getattr(p, k)) for k in ("A", "MA", "B", "MB"))
        f = cs_ngf.prepare_fixed(A, MA, batch=1)
        for _ in range(5):
            f.update_fixed(A, MA)
            f.align(B, MB, ident)
        ts = []
        for _ in range(20):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            f.update_fixed(A, MA)
            f.align(B, MB, ident)
            ts.append(time.perf_counter() - t0)
        gpu = float(np.median(ts))
        cpu = None
        if n <= args.tab3_direct_max:
            t0 = time.perf_counter()
            O.csngf_direct(p.A, p.MA, p.B, p.MB, 1e-5, 0.5)
            cpu = time.perf_counter() - t0
        rows.append({"side": n, "fft": list(f.pad), "gpu_s": gpu, "cpu_direct_s": cpu,
                     "speedup": None if cpu is None else cpu / gpu})
        f.release()
    print(json.dumps({"metric": "one all-shift CSNGF evaluation vs side (Tab. 3 workload)", "unit": "s",
                      "rows": rows, "dtype": "f32 (GPU) / f64 (CPU direct)", "data": "synthetic cubes"}),
          flush=True)
    return 0


def run_search150(args):
    """The paper's full global alignment (Section 3.2 pyramid random search with
    its schedule) on the 150^3 pair: wall time and the corner displacement of
    the result from the generator's true transform (d_E, Section 5.1)."""
    import torch
    from oracle import cs_ngf_oracle as O
    from paper_2110_10156_gb300 import cs_ngf
    pair = load_pair(1, 1000)
    A, MA, B, MB = (_dev(pair[k]) for k in ("A", "MA", "B", "MB"))
    cs_ngf.global_align(A, MA, B, MB, schedule=[(2.0, 4, 180.0, 50, 1)], seed=1)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = cs_ngf.global_align(A, MA, B, MB, seed=args.search_seed)
    dt = time.perf_counter() - t0
    qt = pair["quats"][int(pair["true_index"])]
    tt = [int(v) for v in pair["t_zyx"]]
    n = np.array(pair["A"].shape[::-1], dtype=float)
    c = (n - 1) / 2
    Rf, Rt = O.quat_to_rotmat(g["quat"]), O.quat_to_rotmat(qt)
    err = []
    for corner in np.array(np.meshgrid([0, 1], [0, 1], [0, 1])).reshape(3, -1).T:
        x = corner * (n - 1)
        err.append(np.linalg.norm((Rf @ (x + np.array(g["shift"][::-1]) - c) + c) -
                                  (Rt @ (x + np.array(tt[::-1]) - c) + c)))
    print(json.dumps({"metric": "full global alignment wall time, paper schedule (150^3 pair)", "unit": "s",
                      "value": dt, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                      "rotations_scored": g["rotations_scored"], "d_E_vx": float(np.mean(err)),
                      "found": {"euler_deg": g["euler_deg"], "shift": g["shift"], "score": g["score"]},
                      "level_best": g["level_best"],
                      "config": {"workload": "150^3 pair; sigma (5,3,2,1.5), d (4,2,2,1), u (180,30,10,0),"
                                             " a (5000,3000,300,0), p (1,20,3,1)"}}), flush=True)
    return 0


SERVE_SHAPES = ((64, 64, 64), (96, 128, 128), (150, 150, 150), (192, 192, 160))


def serve_pair(shape):
    """One seeded pair per serving shape (the 32^3 recipe, ellipsoids scaled)."""
    from paper_2110_10156_gb300 import synth
    key = "cs_ngf_serve_%dx%dx%d_v1.npz" % shape
    path = os.path.join(tempfile.gettempdir(), key)
    if os.path.exists(path):
        d = np.load(path)
        return {k: d[k] for k in d.files}
    n = max(shape)
    sc = n / 32.0
    p = synth.make_pair(3000 + n, shape, 12, 3 * sc, 10 * sc, 45.0, max(1, int(6 * sc)), 2,
                        masks="threshold", include_identity=True)
    d = dict(A=p.A, MA=p.MA, B=p.B, MB=p.MB)
    np.savez(path + ".tmp.npz", **d)
    os.replace(path + ".tmp.npz", path)
    return d


def serving_measure(args, precision="fp32"):
    """Poisson arrivals of mixed-size jobs, 200-2000 rotations each, through the
    continuous-batching server at the offered load: p50/p99 job latency (ms)
    and rotations/s."""
    from paper_2110_10156_gb300 import cs_ngf, synth
    rng = np.random.default_rng(1003)
    pairs = {s: serve_pair(s) for s in SERVE_SHAPES}
    n_jobs = args.serve_jobs
    jobs = []
    for k in range(n_jobs):
        s = SERVE_SHAPES[int(rng.integers(len(SERVE_SHAPES)))]
        R = int(rng.integers(200, 2001))
        jobs.append((s, synth.random_quaternions(rng, R)))
    srv = cs_ngf.Server(max_active_jobs=args.serve_active, max_inflight=2, batch=args.serve_batch,
                        policy=args.serve_policy)
    # capacity: each shape alone once (also warms the pooled resources)
    svc = {}
    for s in SERVE_SHAPES:
        p = pairs[s]
        q = synth.random_quaternions(rng, 128)
        t0 = time.perf_counter()
        srv.wait(srv.submit(p["A"], p["MA"], p["B"], p["MB"], q, precision=precision),
                 per_rotation=False)
        svc[s] = (time.perf_counter() - t0) / 128
    mean_service = float(np.mean([svc[s] * len(q) for s, q in jobs]))
    lam = args.serve_load / mean_service                  # jobs per second
    gaps = rng.exponential(1.0 / lam, size=n_jobs)
    t_start = time.perf_counter()
    ids = []
    for (s, q), gap in zip(jobs, gaps):
        time.sleep(float(gap))
        p = pairs[s]
        ids.append(srv.submit(p["A"], p["MA"], p["B"], p["MB"], q, precision=precision))
    res = [srv.wait(j, per_rotation=False) for j in ids]
    wall = time.perf_counter() - t_start
    srv.close()
    lat = np.array([r["latency_ms"] for r in res])
    rot = sum(len(q) for _, q in jobs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "rotations_per_s": rot / wall, "precision": precision,
            "config": {"workload": "jobs of 64^3, 96x128x128, 150^3, 192x192x160 with 200-2000 rotations",
                       "jobs": n_jobs, "offered_load": args.serve_load, "arrival_rate_per_s": lam,
                       "max_active_jobs": args.serve_active, "batch": args.serve_batch,
                       "admission": args.serve_policy},
            "service_ms_per_rotation_alone": {"x".join(map(str, s)): 1000 * v for s, v in svc.items()},
            "statuses": sorted(set(r["status"] for r in res))}


def run_serving(args):
    """--workload serve: the serving measurement as its own JSON line."""
    m = serving_measure(args, args.precision)
    print(json.dumps({
        "metric": "serving: p50/p99 job latency and rotations/s, mixed sizes, Poisson arrivals",
        "unit": "ms", "value": m["p50_ms"], "p99_ms": m["p99_ms"],
        "rotations_per_s": m["rotations_per_s"], "higher_is_better": False,
        "dtype": "f32" if args.precision == "fp32" else f"f32 arithmetic, {args.precision} channel intermediates",
        "data": "synthetic", "config": m["config"],
        "service_ms_per_rotation_alone": m["service_ms_per_rotation_alone"],
        "statuses": m["statuses"]}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--rotations", type=int, default=1000)
    ap.add_argument("--batch", type=int, default=0)
    ap.add_argument("--precision", choices=("fp32", "bf16", "fp16"), default="fp32")
    ap.add_argument("--pad-mode", choices=("bound", "full"), default="bound")
    ap.add_argument("--autotune", choices=("on", "off"), default="on",
                    help="time both radix splits of each FFT pass on the first launch group "
                         "at new lengths (warm-up) and keep the faster")
    ap.add_argument("--tensor-cores", choices=("on", "off"), default="on",
                    help="BF16 / FP16 forms: the z pass's channel DFT on the tensor cores (off: CUDA cores)")
    ap.add_argument("--ref-sample", type=int, default=16,
                    help="oracle rotations per CPU step (at most one per core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BF16 and FP16 forms' sub-results of the headline line")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving sub-result (p50/p99) of the headline line")
    ap.add_argument("--tab3-direct-max", type=int, default=16)
    ap.add_argument("--search-seed", type=int, default=2021)
    ap.add_argument("--workload", choices=("align150", "small32", "serve", "large256", "tab3", "search150"),
                    default="align150", help="align150 is the headline line; the others print "
                                              "their own metrics")
    ap.add_argument("--serve-jobs", type=int, default=24)
    ap.add_argument("--serve-load", type=float, default=0.7)
    ap.add_argument("--serve-active", type=int, default=4)
    ap.add_argument("--serve-policy", choices=("arrival", "shortest"), default="arrival")
    ap.add_argument("--serve-batch", type=int, default=16)
    args = ap.parse_args()
    if args.impl == "ours" and args.workload != "align150":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        return {"small32": run_small_latency, "serve": run_serving, "large256": run_large,
                "tab3": run_tab3, "search150": run_search150}[args.workload](args)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
