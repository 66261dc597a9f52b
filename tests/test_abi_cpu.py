"""The C-ABI library loads and exports every symbol include/cs_ngf.h declares;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from oracle import cs_ngf_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cs_ngf.h")


@pytest.fixture(scope="module")
def binding():
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    return cs_ngf


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_ngf_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cs_ngf_prepare_fixed", "cs_ngf_score_rotations", "cs_ngf_align"):
        assert required in names


def test_library_exports_every_declared_symbol(binding):
    lib = binding.library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(binding.EXPORTED)


def test_auto_pad_matches_oracle(binding):
    for n in range(2, 257):
        assert binding.auto_pad(n) == O.auto_pad(n)
    assert binding.auto_pad(1) == 0 and binding.auto_pad(257) == 0


def test_status_strings(binding):
    lib = binding.library()
    assert lib.cs_ngf_status_string(0) == b"ok"
    assert lib.cs_ngf_status_string(1) == b"invalid argument"
    assert lib.cs_ngf_status_string(binding.EBUSY) == b"handle busy"
    assert lib.cs_ngf_status_string(99) == b"unknown status"


def test_header_status_codes_match_the_binding(binding):
    """Every CS_NGF_E* code of the header has the same value in the binding."""
    text = open(HEADER).read()
    codes = dict((k, int(v)) for k, v in re.findall(r"\bCS_NGF_(E[A-Z]+|OK) = (\d+)", text))
    assert codes["EBUSY"] == 8
    for name, value in codes.items():
        assert getattr(binding, name) == value, name


def test_prepare_rejects_bad_arguments_before_touching_the_device(binding):
    lib = binding.library()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int32 * 3)(8, 8, 8)
    assert lib.cs_ngf_prepare_fixed(None, None, dims, None, None, ctypes.byref(h)) == binding.EINVAL
    assert b"NULL" in lib.cs_ngf_last_error()
    fake = ctypes.c_void_p(16)
    bad = (ctypes.c_int32 * 3)(8, 1, 8)
    assert lib.cs_ngf_prepare_fixed(fake, fake, bad, None, None, ctypes.byref(h)) == binding.EINVAL
    big = (ctypes.c_int32 * 3)(8, 300, 8)
    assert lib.cs_ngf_prepare_fixed(fake, fake, big, None, None, ctypes.byref(h)) == binding.EINVAL
    cfg = binding.Config()
    lib.cs_ngf_default_config(ctypes.byref(cfg))
    assert cfg.eps == pytest.approx(1e-5) and cfg.gamma == 0.5
    assert cfg.pad_mode == binding.PAD_MODES["bound"]      # bound-limited padding by default
    assert ctypes.sizeof(binding.Config) == 44 and ctypes.sizeof(binding.Info) == 80
    assert cfg.tensor_cores == 1                            # tensor-core z pass by default
    cfg.tensor_cores = 2
    assert lib.cs_ngf_prepare_fixed(fake, fake, dims, ctypes.byref(cfg), None, ctypes.byref(h)) == binding.EINVAL
    assert b"tensor_cores" in lib.cs_ngf_last_error()
    cfg.tensor_cores = 1
    cfg.pad_mode = 5
    assert lib.cs_ngf_prepare_fixed(fake, fake, dims, ctypes.byref(cfg), None, ctypes.byref(h)) == binding.EINVAL
    assert b"pad_mode" in lib.cs_ngf_last_error()
    cfg.pad_mode = binding.PAD_MODES["full"]
    assert cfg.autotune == 0
    cfg.autotune = 3
    assert lib.cs_ngf_prepare_fixed(fake, fake, dims, ctypes.byref(cfg), None, ctypes.byref(h)) == binding.EINVAL
    assert b"autotune" in lib.cs_ngf_last_error()
    cfg.autotune = 1
    assert binding.tuning() == []           # nothing timed in this process
    cfg.gamma = 1.5
    assert lib.cs_ngf_prepare_fixed(fake, fake, dims, ctypes.byref(cfg), None, ctypes.byref(h)) == binding.EINVAL
    cfg.gamma = 0.5
    cfg.pad[0] = 96                       # not a supported FFT length
    assert lib.cs_ngf_prepare_fixed(fake, fake, dims, ctypes.byref(cfg), None,
                                    ctypes.byref(h)) == binding.EUNSUPPORTED
    cfg.pad[0] = 16                       # < 2n - 1 for n = 9
    d9 = (ctypes.c_int32 * 3)(9, 8, 8)
    assert lib.cs_ngf_prepare_fixed(fake, fake, d9, ctypes.byref(cfg), None, ctypes.byref(h)) == binding.EINVAL
    assert h.value is None


def test_entry_points_reject_null_handle(binding):
    lib = binding.library()
    assert lib.cs_ngf_score_rotations(None, None, None, None, 1, None, None, None) == binding.EINVAL
    assert lib.cs_ngf_get_info(None, None) == binding.EINVAL
    lib.cs_ngf_release(None)


def test_server_config_checks_before_touching_the_device(binding):
    """The ctypes layout matches the header's defaults, and bad settings are
    refused before any device call (an unknown admission policy included)."""
    lib = binding.library()
    cfg = binding.ServerConfig()
    lib.cs_ngf_server_default_config(ctypes.byref(cfg))
    assert (cfg.max_active_jobs, cfg.max_inflight, cfg.policy) == (4, 2, 0)
    assert ctypes.sizeof(binding.ServerConfig) == 32
    h = ctypes.c_void_p()
    cfg.policy = 7
    assert lib.cs_ngf_server_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.EINVAL
    assert b"policy" in lib.cs_ngf_last_error()
    cfg.policy, cfg.max_active_jobs = 1, 0
    assert lib.cs_ngf_server_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.EINVAL
    assert h.value is None
