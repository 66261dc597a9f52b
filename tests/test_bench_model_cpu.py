"""The bench's roofline numerators and the ncu-summary parser, on the CPU.

The byte model is checked against the buffer sizes of the HBM layout written
out field by field; the flop model against 5 L log2 L per transform counted
column by column; the parser against a small ncu CSV whose sums are known."""
import importlib.util
import json
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    # registered under its own name so that its pool workers (spawn) can
    # import it and unpickle its functions
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    sys.modules["bench"] = mod
    spec.loader.exec_module(mod)
    return mod


def test_byte_model_at_the_headline_lengths(bench):
    dims, pad, nb = (150, 150, 150), (200, 200, 200), 32
    nvox = 150 ** 3
    # per rotation: three packed channel fields of 8 B plus half a mask field of 8 B
    field_bytes = 3 * 8 + 8 / 2
    F0 = field_bytes * 150 * 150 * 200          # [z][y][kx] after the x transform
    F1 = field_bytes * 150 * 200 * 200          # [kx][z][ky] after the y transform
    per = lambda st: bench.stage_bytes(dims, pad, nb, st) / nb
    assert per("resample") == nvox * 5          # B-hat (4 B) and M-hat (1 B) written
    assert per("fwd_x") == pytest.approx(nvox * 5 + F0)
    assert per("fwd_y") == pytest.approx(F0 + F1)
    UV = 7 * 101 * 200 * 200 * 8                 # fixed spectra, loaded once per launch
    # the z inverse's output: min(2n - 1, P) = 200 planes of Z per (kx, ky) column
    F2 = 200 * 200 * 200 * 8
    assert per("zmac") == pytest.approx(F1 + UV / nb + F2)
    assert per("zmac_no_f2") == pytest.approx(F1 + UV / nb)
    F3 = 200 * 200 * 200 * 8                     # [vz][vy][kx], again at most P planes and rows
    assert per("inv_y") == F2 + F3 and per("inv_x") == F3
    # the figures the design notes quote (MB per rotation)
    assert round(per("fwd_x") / 1e6) == 143 and round(per("fwd_y") / 1e6) == 294
    assert round(per("zmac") / 1e6) == 239 and round(per("zmac_no_f2") / 1e6) == 175
    # at full padding every one of the 2n - 1 = 299 shifts has a plane
    full = lambda st: bench.stage_bytes(dims, (320, 320, 320), nb, st) / nb
    assert full("inv_x") == 299 * 299 * 320 * 8


def test_byte_model_halves_channel_bytes_in_16_bit_forms(bench):
    dims, pad = (150, 150, 150), (200, 200, 200)
    f32 = bench.stage_bytes(dims, pad, 2, "fwd_y")
    b16 = bench.stage_bytes(dims, pad, 2, "fwd_y", precision="bf16")
    E = 150 * 150 * 200 + 150 * 200 * 200      # F0 + F1 element positions
    assert f32 - b16 == 2 * 3 * 4 * E           # 2 rotations x 3 channel fields x 4 B saved


def test_flop_model_counts_transforms_and_products(bench):
    dims, pad, nb = (150, 150, 150), (200, 200, 200), 2
    L, cols = 200, 200 * 200
    fwd = 5 * L * math.log2(L)                  # 150 > 100: no zero half to prune
    fields = 3 * nb + 1
    mac = 101 * 200 * 200 * (16 * 3 + 20) * nb
    want = fields * cols * fwd + nb * cols * 5 * L * math.log2(L) + mac
    assert bench.zmac_flops(dims, pad, nb) == pytest.approx(want)
    # full padding: the input is zero past L/2, so the first radix-2 stage is
    # pruned; a pair of rotations shares one mask field (3.5 fields each)
    L = 320
    got = bench.zmac_flops(dims, (L, L, L), 2) / 2
    fwd = 5 * L * (math.log2(L) - 1) + L
    want = 3.5 * L * L * fwd + L * L * 5 * L * math.log2(L) + 161 * L * L * 68
    assert got == pytest.approx(want)
    assert round(got / 1e9, 1) == 6.8
    assert round(bench.zmac_flops(dims, pad, 2) / 2 / 1e9, 2) == 1.65


def _csv_row(i, name, metric, unit, value):
    return f'"{i}","1","python","127.0.0.1","{name}","1","7","(1,1,1)","(1,1,1)","0","10.3",' \
           f'"Section","{metric}","{unit}","{value}"\n'


def test_traffic_summary_parser(tmp_path, bench):
    from paper_2110_10156_gb300 import profile_workload as pw
    head = '"ID","Process ID","Process Name","Host Name","Kernel Name","Context","Stream",' \
           '"Block Size","Grid Size","Device","CC","Section Name","Metric Name","Metric Unit",' \
           '"Metric Value"\n'
    rows = [
        _csv_row(0, "void csngf::k_fwd_x<200, 10, 0, 0, 1>(const float *)", "dram__bytes_read.sum", "Mbyte", "999"),
        _csv_row(1, "csngf::k_resample(const float2 *)", "dram__bytes_read.sum", "Mbyte", "1.5"),
        _csv_row(1, "csngf::k_resample(const float2 *)", "dram__bytes_write.sum", "Mbyte", "2.5"),
        _csv_row(2, "void csngf::k_zmac<200, 0, 0, 0>(const void *)", "dram__bytes_read.sum", "Gbyte", "1.25"),
        _csv_row(2, "void csngf::k_zmac<200, 0, 0, 0>(const void *)", "dram__bytes_write.sum", "byte", "1,000"),
        _csv_row(2, "void csngf::k_zmac<200, 0, 0, 0>(const void *)", "gpu__time_duration.sum", "ms", "3"),
    ]
    csv_path = tmp_path / "traffic.csv"
    csv_path.write_text("==PROF== preamble\n" + head + "".join(rows))
    out_path = tmp_path / "traffic.json"
    out = pw.traffic_from_csv(str(csv_path), 2, str(out_path), fft=(200, 200, 256))
    assert out["src_hash"] == bench.kernel_source_hash()
    (c,) = out["classes"]
    assert c["fft"] == [200, 200, 256]
    st = c["stages"]
    # the fixed volume's pass before the first resample is left out
    assert set(st) == {"resample", "zmac"}
    assert st["resample"] == {"launches": 1, "dram_bytes_per_rotation": 2.0e6,
                              "dram_bytes_per_launch_fixed": 0.0}
    assert st["zmac"]["dram_bytes_per_rotation"] == pytest.approx((1.25e9 + 1000) / 2)
    assert json.loads(out_path.read_text()) == out
    # a second capture of the same launches with one rotation separates the
    # bytes every launch moves (4 rotations: 1.25 GB; 1 rotation: 0.5 GB); at
    # other lengths it is kept beside the first class
    base_rows = [
        _csv_row(1, "csngf::k_resample(const float2 *)", "dram__bytes_read.sum", "Mbyte", "1.0"),
        _csv_row(2, "void csngf::k_zmac<200, 0, 0, 0>(const void *)", "dram__bytes_read.sum", "Gbyte", "0.5"),
    ]
    rows4 = [
        _csv_row(1, "csngf::k_mask_counts(const unsigned char *)", "dram__bytes_read.sum", "Mbyte", "4.0"),
        _csv_row(2, "void csngf::k_zmac<200, 0, 0, 0>(const void *)", "dram__bytes_read.sum", "Gbyte", "1.25"),
    ]
    p4, p1 = tmp_path / "t4.csv", tmp_path / "t1.csv"
    p4.write_text(head + "".join(rows4))
    p1.write_text(head + "".join(base_rows))
    out = pw.traffic_from_csv([str(p4)], 4, str(out_path), base_paths=[str(p1)], base_rotations=1,
                              fft=(200, 200, 200))
    assert [c["fft"] for c in out["classes"]] == [[200, 200, 256], [200, 200, 200]]
    z = out["classes"][1]["stages"]["zmac"]
    assert z["dram_bytes_per_rotation"] == pytest.approx(0.25e9)
    assert z["dram_bytes_per_launch_fixed"] == pytest.approx(0.25e9)
    r = out["classes"][1]["stages"]["resample"]   # k_mask_counts counts with the resample stage
    assert r["dram_bytes_per_rotation"] == pytest.approx(1.0e6) and r["dram_bytes_per_launch_fixed"] == pytest.approx(0.0)
    # recapturing a class replaces its entry
    out = pw.traffic_from_csv([str(p4)], 4, str(out_path), fft=(200, 200, 200))
    assert len(out["classes"]) == 2
    assert out["classes"][1]["stages"]["zmac"]["dram_bytes_per_launch_fixed"] == 0.0


def test_traffic_per_launch_by_class(bench, tmp_path, monkeypatch):
    """Each launch takes its own class's figures; lengths with no capture take
    the nearest captured class scaled by the byte model."""
    dims = (150, 150, 150)
    d = {"src_hash": bench.kernel_source_hash(), "precision": "fp32", "classes": [
        {"fft": [200, 200, 200], "stages": {"zmac": {"dram_bytes_per_rotation": 100.0,
                                                     "dram_bytes_per_launch_fixed": 1000.0}}},
        {"fft": [200, 200, 256], "stages": {"zmac": {"dram_bytes_per_rotation": 130.0,
                                                     "dram_bytes_per_launch_fixed": 1300.0}}}]}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(d))
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    L = [((200, 200, 200), 32), ((200, 200, 200), 8), ((200, 200, 256), 4)]
    assert bench.launch_traffic("zmac", "fp32", dims, L) == pytest.approx(
        2 * 1000 + 40 * 100 + 1300 + 4 * 130)
    assert bench.launch_traffic("fwd_x", "fp32", dims, L) is None
    assert bench.ncu_traffic("zmac", "bf16", dims, (200, 200, 200)) is None
    # (200, 256, 200) has as many grid points as (200, 200, 256), its nearest capture
    pr, fx = bench.ncu_traffic("zmac", "fp32", dims, (200, 256, 200))
    one = lambda q: bench.stage_bytes(dims, q, 1, "zmac") - bench.stage_bytes(dims, q, 0, "zmac")
    tile = lambda q: bench.stage_bytes(dims, q, 0, "zmac")
    assert pr == pytest.approx(130.0 * one((200, 256, 200)) / one((200, 200, 256)))
    assert fx == pytest.approx(1300.0 * tile((200, 256, 200)) / tile((200, 200, 256)))
    # the fixed-spectra tile has (Px/2 + 1) Py Pz points: 101*256 against 129*200
    assert fx == pytest.approx(1300.0 * 101 * 256 / (129 * 200))


def test_compare_with_oracle(bench):
    inf = float("inf")
    gpu_s = [0.5, 0.25, -inf, 0.7, -inf]
    gpu_c = [(1, 2, 3), (0, 0, 1), (0, 0, 0), (4, 4, 4), (0, 0, 0)]
    oracle = [(0.5 + 2e-7, (1, 2, 3)), (0.25, (0, 1, 0)), (-inf, (0, 0, 0)), (0.7, (4, 4, 4)),
              (0.1, (1, 1, 1))]
    out = bench.compare_with_oracle(gpu_s, gpu_c, oracle)
    assert out["rotations"] == 5
    assert out["max_abs_score_err"] == pytest.approx(2e-7)
    assert out["same_shift"] == 3                 # rotations 0, 2 (both invalid) and 3
    assert out["validity_mismatch"] == 1          # rotation 4


def test_reference_arm_prints_one_line(bench, monkeypatch, capsys):
    """The reference arm's JSON line, with the oracle timing stubbed out (the
    real arm runs the FP64 oracle for minutes)."""
    import argparse
    import numpy as np
    monkeypatch.setattr(bench, "load_pair", lambda config, n: {"quats": np.zeros((n, 4))})
    monkeypatch.setattr(bench, "oracle_sample",
                        lambda pair, n, cores: (n / 2.0, 2.0, [(0.5, (0, 0, 0))] * n))
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    args = argparse.Namespace(config=1, rotations=1000, ref_sample=4, warmup=3, steps=2)
    assert bench.run_reference(args) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["higher_is_better"] is True
    assert line["value"] == pytest.approx(2.0)      # 4 rotations per 2 s step
    assert line["ms_per_step"] == pytest.approx(2000.0)    # the sample actually timed
    assert line["ms_per_workload_extrapolated"] == pytest.approx(2000.0 * 1000 / 4)
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["h2d_bytes_per_step"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_oracle_sample_returns_the_oracles_best(bench):
    """The CPU leg's pool returns each sampled rotation's best (score, shift),
    the values compare_with_oracle checks the GPU's results against."""
    from oracle import cs_ngf_oracle as O
    from paper_2110_10156_gb300 import synth
    p = synth.small_pair(77, (10, 9, 11), n_rot=3, masks="full")
    pair = {"A": p.A, "MA": p.MA, "B": p.B, "MB": p.MB, "quats": p.quats}
    rate, dt, best = bench.oracle_sample(pair, 2, 2)
    assert rate > 0 and dt > 0 and len(best) == 2
    for q, (s, chi) in zip(p.quats[:2], best):
        want = O.best_of_map(O.score_map(p.A, p.MA, p.B, p.MB, q)[0])
        assert s == want[0] and tuple(chi) == tuple(want[1])
