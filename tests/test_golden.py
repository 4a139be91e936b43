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


def test_rectangle_heights_equal_point_heights():
    import numpy as np
    import scenegen as sg
    rng = np.random.default_rng(4)
    for spec in (sg.SINGLE_128, sg.CITY_4096, sg.OPEN_65536):
        w = sg.World(spec)
        for _ in range(4):
            x0, y0 = (int(v) for v in rng.integers(-300, spec.wx, 2))
            nx, ny = (int(v) for v in rng.integers(1, 90, 2))
            h = w.heights(x0, y0, nx, ny)
            ref = np.array([[w.height(x0 + x, y0 + y) for x in range(nx)] for y in range(ny)], np.int32)
            assert (h == ref).all()
