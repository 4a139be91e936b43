"""Stored fingerprints: the generated worlds and the oracle's results are the
same on every platform (x86-64 here, aarch64 on the GPU host).  The stored
values are written by tests/golden/make_golden.py, which calls only scenegen
and oracle."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def load(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def test_generator_fingerprints():
    assert make_golden.region_fingerprints() == load("scenegen_hashes.json")


def test_oracle_fingerprints():
    assert make_golden.oracle_fingerprints() == load("oracle_small.json")
