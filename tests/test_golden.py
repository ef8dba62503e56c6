"""The oracle against its stored energies (``tests/golden/oracle_energies.json``, written by
``tests/golden/make_golden.py`` from the oracle alone): a change of the oracle's arithmetic that
moves E_c, its per-q or its per-omega parts shows up here.  The KS data come from numpy's
eigensolver, whose last bits may differ between BLAS builds, hence 1e-10 relative."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "oracle_energies.json")))


@pytest.mark.parametrize("name", sorted(GOLD["cases"]))
def test_oracle_reproduces_stored_energies(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    got = mk.compute(name)
    want = GOLD["cases"][name]
    scale = abs(want["ec"])
    assert abs(got["ec"] - want["ec"]) <= 1e-10 * scale
    assert np.abs(np.array(got["ec_q"]) - want["ec_q"]).max() <= 1e-10 * scale
    assert np.abs(np.array(got["ec_w"]) - want["ec_w"]).max() <= 1e-10 * scale
