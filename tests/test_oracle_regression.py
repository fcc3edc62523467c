"""The oracle's outputs on short runs of every body kind, against the values
tests/golden/make_oracle_regression.py stored: a change to the oracle's
arithmetic fails here until the file is rewritten, in a commit that names the
passage of the paper (or the reading of it) that justifies the change."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _stored():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "oracle_regression.txt")):
        if line.startswith("#") or not line.strip():
            continue
        case, key, v = line.split()
        vals.setdefault(case, {})[key] = float(v)
    return vals


def test_oracle_outputs_match_the_stored_runs(orc):
    spec = importlib.util.spec_from_file_location("make_oracle_regression",
                                                  os.path.join(HERE, "golden", "make_oracle_regression.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    stored = _stored()
    got = gen.compute()
    assert set(got) == set(stored)
    for case, vals in got.items():
        assert set(vals) == set(stored[case]), case
        for k, v in vals.items():
            # the C arithmetic is deterministic; the population sums take
            # numpy's summation order, which may differ between builds
            assert v == pytest.approx(stored[case][k], rel=1e-12, abs=1e-15), (case, k)
