"""The persistent autotuning cache (cs_ngf_tuning_save / cs_ngf_tuning_load):
host-only calls, so the whole round trip and every rejection runs on the CPU."""
import pytest


@pytest.fixture()
def cs():
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    cs_ngf.tuning_reset()
    yield cs_ngf
    cs_ngf.tuning_reset()


GOOD = """# written by hand
0 200 0 0 1 1.806 1.664
2 200 0 0 0 3.933 4.263
  1 256 0 1 0 0.868 1.246

4 256 0 0 0 0.214 0.477
"""


def _entries(cs):
    return sorted((e["stage"], e["length"], e["half_input"], e["storage"], e["variant"])
                  for e in cs.tuning())


def test_load_merges_entries_with_their_splits(cs, tmp_path):
    p = tmp_path / "tune.txt"
    p.write_text(GOOD)
    cs.tuning_load(p)
    got = {(e["stage"], e["length"], e["storage"]): e for e in cs.tuning()}
    assert len(got) == 4
    e = got[("fwd_x", 200, "fp32")]
    assert e["variant"] == 1 and e["splits"] == [(10, 20), (8, 25)]
    assert e["ms"] == pytest.approx([1.806, 1.664], rel=1e-6)
    assert got[("fwd_y", 256, "bf16")]["splits"] == [(16, 16), (8, 32)]
    assert got[("zmac", 200, "fp32")]["variant"] == 0
    assert got[("inv_x", 256, "fp32")]["half_input"] is False


def test_save_then_load_round_trip(cs, tmp_path):
    src = tmp_path / "a.txt"
    src.write_text(GOOD)
    cs.tuning_load(src)
    before = cs.tuning()
    out = tmp_path / "b.txt"
    cs.tuning_save(out)
    lines = [ln for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert len(lines) == 4 and all(len(ln.split()) == 7 for ln in lines)
    cs.tuning_reset()
    assert cs.tuning() == []
    cs.tuning_load(out)
    after = cs.tuning()
    assert [(e["stage"], e["length"], e["variant"], e["splits"]) for e in after] == \
           [(e["stage"], e["length"], e["variant"], e["splits"]) for e in before]
    for a, b in zip(after, before):
        assert a["ms"] == pytest.approx(b["ms"], rel=1e-5)


def test_a_loaded_entry_replaces_the_same_key(cs, tmp_path):
    p = tmp_path / "t.txt"
    p.write_text("0 200 0 0 1 2 1\n")
    cs.tuning_load(p)
    p.write_text("0 200 0 0 0 1 2\n")
    cs.tuning_load(p)
    assert _entries(cs) == [("fwd_x", 200, False, "fp32", 0)]


@pytest.mark.parametrize("line", [
    "5 200 0 0 1 1 1",          # no such pass
    "0 512 0 0 1 1 1",          # 512 has a single split
    "0 201 0 0 1 1 1",          # not a supported length
    "3 200 1 0 1 1 1",          # inverse passes have no half-input form
    "4 200 0 2 1 1 1",          # nor a storage form
    "0 200 2 0 1 1 1",          # half_input is 0 or 1
    "1 200 0 3 0 1 1",          # storage out of range
    "0 200 0 0 2 1 1",          # variant 0 or 1
    "0 200 0 0 1 -1 1",         # negative time
    "0 200 0 0 1 nan 1",        # not a number
    "0 200 0 0 1 1",            # a field missing
    "0 200 0 0 1 1 1 7",        # a field too many
    "zmac 200 0 0 1 1 1",       # names are not accepted
])
def test_bad_lines_are_refused_and_nothing_is_merged(cs, tmp_path, line):
    p = tmp_path / "bad.txt"
    p.write_text("0 256 0 0 1 1 1\n" + line + "\n")
    with pytest.raises(cs.CsNgfError) as ei:
        cs.tuning_load(p)
    assert ei.value.status == cs.EINVAL
    assert "line 2" in str(ei.value)
    assert cs.tuning() == []


def test_missing_file_and_unwritable_path(cs, tmp_path):
    with pytest.raises(cs.CsNgfError) as ei:
        cs.tuning_load(tmp_path / "absent.txt")
    assert ei.value.status == cs.EINVAL
    with pytest.raises(cs.CsNgfError):
        cs.tuning_save(tmp_path / "no_such_dir" / "t.txt")


def test_null_path_is_refused(cs):
    lib = cs.library()
    assert lib.cs_ngf_tuning_save(None) == cs.EINVAL
    assert lib.cs_ngf_tuning_load(None) == cs.EINVAL
