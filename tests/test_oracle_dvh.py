"""Pins of the oracle's dose-volume histogram (the evaluation behind Fig. 2)
against hand counts (tests/golden/dvh.json), and invariants: every voxel is
counted once in its own structure, and a larger dose never lands in a lower
bin."""
import json
import os

import numpy as np

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "dvh.json")))


def test_dvh_hand_counts():
    for c in GOLD["cases"]:
        got = oracle.dvh(np.array(c["z"]), np.array(c["sid"]), c["n_struct"], c["dose_max"], c["n_bins"])
        np.testing.assert_array_equal(got, np.array(c["counts"]), err_msg=c["_why"])


def test_dvh_counts_every_voxel_once_and_is_monotone():
    rng = np.random.default_rng(5)
    z = rng.uniform(-0.1, 1.4, 3000)
    sid = rng.integers(0, 5, z.size).astype(np.uint8)
    c = oracle.dvh(z, sid, 5, 1.2, 37)
    np.testing.assert_array_equal(c.sum(axis=1), np.bincount(sid, minlength=5))
    # one voxel at a time: its bin never decreases as its dose grows
    last = 0
    for v in np.sort(rng.uniform(-0.2, 1.5, 400)):
        b = int(np.flatnonzero(oracle.dvh(np.array([v]), np.zeros(1, np.uint8), 1, 1.2, 37)[0])[0])
        assert b >= last
        last = b
    # bin b holds exactly the doses of [b w, (b + 1) w) for doses on a dyadic grid
    grid = np.arange(0, 1.5, 1 / 64)
    cg = oracle.dvh(grid, np.zeros(grid.size, np.uint8), 1, 1.0, 8)[0]
    np.testing.assert_array_equal(cg, [8] * 7 + [8 + 32])
