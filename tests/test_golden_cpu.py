"""The method's printed parameters (tests/golden/paper_parameters.json, each
value citing its section) are the defaults of the C ABI, of the Python
binding and of the oracle.  Config calls only: no device work."""
import ctypes
import inspect
import json
import os

import numpy as np
import pytest

from oracle import cs_ngf_oracle as O
from oracle import search_oracle as S

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_parameters.json")


@pytest.fixture(scope="module")
def paper():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    return {k: v["value"] for k, v in d.items() if not k.startswith("_")}


@pytest.fixture(scope="module")
def binding():
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    return cs_ngf


def test_every_value_cites_a_section():
    with open(GOLDEN) as fh:
        d = json.load(fh)
    for k, v in d.items():
        if not k.startswith("_"):
            assert v["cite"].startswith("Section "), k


def test_scoring_defaults_of_the_abi(binding, paper):
    cfg = binding.Config()
    binding.library().cs_ngf_default_config(ctypes.byref(cfg))
    assert cfg.eps == np.float32(paper["eps"])
    assert cfg.gamma == np.float32(paper["gamma"])
    assert cfg.measure == binding.MEASURES["squared"]      # Eq. 2, the squared dot product


def test_search_defaults_of_the_abi(binding, paper):
    sc = binding.SearchConfig()
    binding.library().cs_ngf_search_default_config(ctypes.byref(sc))
    m = sc.levels
    assert m == len(paper["sigma"])
    assert [sc.sigma[k] for k in range(m)] == [np.float32(v) for v in paper["sigma"]]
    assert [sc.downsample[k] for k in range(m)] == paper["downsample"]
    assert [sc.max_step_deg[k] for k in range(m)] == [np.float32(v) for v in paper["max_step_deg"]]
    assert [sc.random_rotations[k] for k in range(m)] == paper["random_rotations"]
    assert [sc.starting_points[k] for k in range(m)] == paper["starting_points"]
    assert list(sc.start_euler_deg) == paper["start_euler_deg"]
    # levels past the schedule are left zero
    assert all(sc.random_rotations[k] == 0 and sc.downsample[k] == 0 for k in range(m, 8))


def _defaults(fn, *names):
    sig = inspect.signature(fn)
    return [sig.parameters[n].default for n in names]


def test_python_defaults(binding, paper):
    want = [paper["eps"], paper["gamma"]]
    for fn in (binding.Fixed.__init__, binding.score_rotations_noalloc, binding.Server.submit,
               binding.global_align):
        assert _defaults(fn, "eps", "gamma") == want, fn.__qualname__
    assert list(_defaults(binding.global_align, "start")[0]) == paper["start_euler_deg"]


def test_oracle_defaults(paper):
    want = [paper["eps"], paper["gamma"]]
    for fn in (O.score_map, O.score_rotations, O.align, S.global_align):
        assert _defaults(fn, "eps", "gamma") == want, fn.__qualname__
    assert list(_defaults(S.global_align, "start")[0]) == paper["start_euler_deg"]
