"""The oracle reproduces its stored regression anchors (tests/golden/).

arXiv:0712.0813 prints no numerical example, so these anchors were written by
tests/golden/make_golden.py from the oracle alone; they guard the oracle
against unintended changes.  The tolerance covers last-bit differences of the
host FFT used by the input generator on another CPU architecture."""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "oracle_regression.json")))


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["config"]["name"] for c in GOLD["cases"]])
def test_oracle_matches_regression_anchor(orc, case):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    got = mg.run_case(case["config"])
    ref = case["result"]
    for key in ("E", "V", "a", "ap"):
        assert got[key] == pytest.approx(ref[key], rel=1e-10, abs=1e-14), key
    for key in ("K", "G", "mean", "var"):
        np.testing.assert_allclose(got[key], ref[key], rtol=1e-8, atol=1e-16, err_msg=key)
    for key in ("f_samples", "v_samples"):
        r = np.array(ref[key])
        np.testing.assert_allclose(np.array(got[key]), r, rtol=0, atol=1e-10 * np.abs(r).max(), err_msg=key)
