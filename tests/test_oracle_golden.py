"""The oracle against its stored regression values (tests/golden/oracle_small.json).

These values were written by tests/golden/make_oracle_golden.py from the oracle alone; they
are not pins of the method (the paper prints no worked example of the projection) but make
any change of the oracle's arithmetic fail here until the file is regenerated, with the
change justified by the passage it follows.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def stored():
    with open(os.path.join(HERE, "golden", "oracle_small.json")) as f:
        return json.load(f)


def test_oracle_matches_stored_values(oracle, stored):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_golden",
                                                  os.path.join(HERE, "golden", "make_oracle_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    now = mod.cases()
    assert set(now) == set(stored)
    for name, case in stored.items():
        for key, val in case.items():
            if key == "cite":
                assert now[name][key] == val
                continue
            np.testing.assert_allclose(np.asarray(now[name][key]), np.asarray(val), rtol=1e-10, atol=1e-14,
                                       err_msg=f"{name}.{key}")
