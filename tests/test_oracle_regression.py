"""Fixtures under tests/golden/:
* Table 2's default parameters (values the paper prints) against the oracle's
  and the C ABI's defaults;
* the oracle's own results on three small seeded scenes, written by
  tests/golden/make_oracle_regression.py, so that any change of the oracle's
  arithmetic shows up here and has to be made on purpose."""
import os
import sys

import pytest

import oracle

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def table2():
    vals = {}
    with open(os.path.join(HERE, "table2_parameters.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


def test_oracle_defaults_are_table_2():
    p = oracle.params()
    for k, v in table2().items():
        assert getattr(p, k) == v, k


def test_c_abi_defaults_are_table_2():
    from paper_2211_04045_gb300 import cch
    p = cch.params()
    for k, v in table2().items():
        assert getattr(p, k) == v, k


def test_oracle_matches_its_regression_record():
    sys.path.insert(0, HERE)
    import make_oracle_regression as m
    with open(os.path.join(HERE, "oracle_regression.txt")) as f:
        want = [l.strip() for l in f if l.strip() and not l.startswith("#")]
    assert m.lines() == want
