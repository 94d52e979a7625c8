"""Oracle regression against fixtures written by tests/golden/make_golden.py
(which calls only the oracle).  The paper prints no worked numeric example, so
these pin the oracle against unintended changes, not against the paper."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_matches_its_recorded_outputs(oracle_mod):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    ref = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))
    now = mg.compute()
    assert set(now) == set(ref)
    for k, v in ref.items():
        a, b = np.asarray(now[k], np.float64), np.asarray(v, np.float64)
        assert a.shape == b.shape, k
        assert np.allclose(a, b, rtol=1e-9, atol=0), k  # libm may differ by an ulp across hosts
