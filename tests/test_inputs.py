"""The seeded input generator: deterministic, well-formed CSR, and the
stand-in dose model at hand-worked points."""
import math

import numpy as np

from paper_1005_4396_b300 import inputs
from paper_1005_4396_b300.inputs import rng


def test_splitmix64_published_sequence():
    # SplitMix64 seeded with 0: first outputs as published with the algorithm
    # (Steele, Lea, Flood 2014; also the seeding generator of xoshiro/xorshift)
    assert [int(v) for v in rng.splitmix64(0, 3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = rng.uniform(7, 10000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.02
    n = rng.normal(7, 20000)
    assert abs(n.mean()) < 0.05 and abs(n.std() - 1) < 0.05


def test_tiny_csr_well_formed_and_deterministic(tiny_problem):
    p = tiny_problem
    cfg = p.cfg
    assert p.n_beamlets == 36 * 10 * 10 and p.n_vox == 32 * 32 * 8
    assert p.row_ptr[0] == 0 and np.all(np.diff(p.row_ptr) >= 0)
    for i in range(0, p.n_beamlets, 37):
        v = p.vox_idx[p.row_ptr[i]:p.row_ptr[i + 1]]
        assert np.all(np.diff(v) > 0)
    assert p.val.min() >= cfg.cutoff and p.val.max() <= 1.0
    q = inputs.make_problem(inputs.tiny_config())
    assert np.array_equal(q.row_ptr, p.row_ptr) and np.array_equal(q.val, p.val)


def test_tiny_geometry_hand_values(tiny_problem):
    p = tiny_problem
    R, C = 10, 10
    # beam 0 (theta = 0, travels +y), row 5 (v_r = +5 mm), column 5 (u_c = +5 mm)
    i = (0 * R + 5) * C + 5
    # voxel (ix=17, iy=16, iz=5): centre (6, 2, 6) mm; lateral offsets 1 and 1 mm;
    # the ray enters the 128 mm box at y = -64, so depth = 66 mm
    j = (5 * 32 + 16) * 32 + 17
    row = slice(p.row_ptr[i], p.row_ptr[i + 1])
    k = np.searchsorted(p.vox_idx[row], j)
    assert p.vox_idx[row][k] == j
    assert p.val[row][k] == pytest_approx(math.exp(-0.005 * 66 - 2.0 / (2 * 16)))
    # rows whose central ray lies outside the 32 mm slab are empty (v_r = +-25 .. +-45)
    for r in (0, 1, 2, 7, 8, 9):
        for k2 in (0, 17):
            i2 = (k2 * R + r) * C + 3
            assert p.row_ptr[i2 + 1] == p.row_ptr[i2]


def pytest_approx(v):
    import pytest
    return pytest.approx(v, rel=1e-14)


def test_structure_priority():
    cfg = inputs.tiny_config()
    sid, T, a, b, names = inputs.structure_map(cfg)
    assert names == ["air", "tissue", "target", "oar"]
    X, Y, Z = inputs.voxel_centres(cfg)
    both = ((X / 24) ** 2 + (Y / 20) ** 2 + (Z / 12) ** 2 <= 1) & (X ** 2 + (Y - 20) ** 2 + Z ** 2 <= 144)
    assert both.any() and np.all(sid[both] == 2)  # target wins over the OAR
    assert T[2] == 1.0 and a[3] == 0.0 and b[3] == 0.5
