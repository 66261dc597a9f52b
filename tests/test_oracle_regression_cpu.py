"""The oracle's results on the seeded 32^3 pair equal the stored values that
tests/golden/make_oracle_regression.py wrote from the oracle itself: a guard
against unintended change to the oracle (it pins nothing against the paper;
the pins in test_oracle_pins.py do that)."""
import json
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_stored_results():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_oracle_regression", os.path.join(HERE, "golden", "make_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(mod.OUT) as fh:
        stored = json.load(fh)
    now = mod.compute()
    assert now["shifts"] == stored["shifts"]
    assert now["scores"] == pytest.approx(stored["scores"], rel=1e-10, abs=0)
