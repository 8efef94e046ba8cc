"""Coarse voxels for unspecified tissue (Sec. 3): pins of the merge.  Every
fine voxel is counted once (weighted row sums of D are preserved), the
coarse dose is the mean fine dose of each block's tissue, other voxels are
untouched, and for a dose that is constant on each merged block the
volume-weighted cost of Eq. 1 equals the fine cost exactly."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs


@pytest.fixture(scope="module")
def pair():
    fine = inputs.make_problem(inputs.small_config(nx=21, ny=17, nz=7))
    return fine, inputs.coarse_tissue(fine)


def test_merge_counts_every_voxel_once(pair):
    fine, cp = pair
    c = cp.prob
    assert np.bincount(cp.fine_to, minlength=c.n_vox).tolist() == cp.weight.tolist()
    assert c.n_vox < fine.n_vox and cp.weight.max() <= 8
    # weighted row sums of D are preserved
    rs_f = np.add.reduceat(fine.val, fine.row_ptr[:-1][np.diff(fine.row_ptr) > 0])
    nzr = np.diff(c.row_ptr) > 0
    rs_c = np.add.reduceat(c.val * cp.weight[c.vox_idx], c.row_ptr[:-1][nzr])
    np.testing.assert_allclose(rs_c, rs_f, rtol=1e-12)
    # rows sorted, structures valid
    for i in range(0, c.n_beamlets, 97):
        seg = c.vox_idx[c.row_ptr[i]:c.row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)
    assert c.struct_id.max() < c.T.size


def test_coarse_dose_is_the_block_mean(pair):
    fine, cp = pair
    x = np.random.default_rng(3).uniform(size=fine.n_beamlets)
    zf = oracle.dose(fine, x)
    zc = oracle.dose(cp.prob, x)
    mean = np.bincount(cp.fine_to, weights=zf, minlength=cp.prob.n_vox) / cp.weight
    np.testing.assert_allclose(zc, mean, rtol=1e-12, atol=1e-14)
    assert np.all(cp.prob.struct_id[:np.count_nonzero(fine.struct_id != 1)] ==
                  fine.struct_id[fine.struct_id != 1])


def test_weighted_cost_equals_fine_cost_for_blockwise_constant_dose(pair):
    fine, cp = pair
    c = cp.prob
    zc = np.random.default_rng(4).uniform(0.0, 1.5, c.n_vox)
    zf = zc[cp.fine_to]  # constant on each merged block
    cf = oracle.voxel_cost(zf, fine.struct_id, fine.T, fine.alpha, fine.beta)
    cc = oracle.voxel_cost(zc, c.struct_id, c.T, c.alpha, c.beta)
    assert cc == pytest.approx(cf, rel=1e-12)
