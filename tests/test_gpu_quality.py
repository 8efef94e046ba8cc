"""GPU dose-volume histograms against the FP64 oracle's counts (the
evaluation behind Fig. 2).  The kernel takes a voxel's bin in FP32
(floor(z * s), s = n_bins / dose_max rounded to FP32), the oracle compares
the dose with the FP64 bin edges; they agree exactly except for voxels whose
dose lies within FP32 rounding of an edge, which may land on either side.
Those voxels are found from the FP64 values and reported; with them moved
to the lower (upper) bin the oracle gives the least (greatest) count at or
above every edge, and the GPU's counts must lie between."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs, quality

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import vmat  # noqa: E402


def _check_against_oracle(got, z, sid, n_struct, dose_max, n_bins):
    """GPU counts vs oracle counts; returns the number of edge voxels."""
    z64 = np.asarray(z, np.float64)
    base = oracle.dvh(z64, sid, n_struct, dose_max, n_bins)
    u = z64 * n_bins / dose_max
    k = np.rint(u)
    # FP32 product of z with n_bins / dose_max rounded to FP32: within
    # 1.5 * 2^-23 relative of u; a margin of 2^-21 covers it
    edge = (k >= 1) & (k <= n_bins - 1) & (np.abs(u - k) <= 2.0 ** -21 * k)
    lo, hi = base.copy(), base.copy()
    for j in np.flatnonzero(edge):
        s = int(sid[j])
        ob = int(np.flatnonzero(oracle.dvh(z64[j:j + 1], np.zeros(1, np.uint8), 1, dose_max, n_bins)[0])[0])
        kb = int(k[j])
        lo[s, ob] -= 1
        lo[s, kb - 1] += 1
        hi[s, ob] -= 1
        hi[s, kb] += 1
    np.testing.assert_array_equal(got.sum(axis=1), base.sum(axis=1))
    if not edge.any():
        np.testing.assert_array_equal(got, base)
        return 0
    cum = lambda c: np.cumsum(c[:, ::-1], axis=1)[:, ::-1]  # voxels at or above each lower edge
    assert np.all(cum(lo) <= cum(got)) and np.all(cum(got) <= cum(hi))
    # every bin away from an edge voxel is exact
    near = np.zeros_like(base, dtype=bool)
    for j in np.flatnonzero(edge):
        near[int(sid[j]), int(k[j]) - 1:int(k[j]) + 1] = True
    np.testing.assert_array_equal(got[~near], base[~near])
    return int(edge.sum())


@pytest.mark.parametrize("n_bins", [1, 37, 1000])
def test_dvh_counts_vs_oracle(n_bins):
    prob = inputs.make_problem(inputs.small_config())
    z = (inputs.rng.uniform(120, prob.n_vox) * 1.3).astype(np.float32)
    z[::97] = 0.0
    z[1::89] = 2.0   # above dose_max: last bin
    z[2::83] = 0.625  # on a bin edge for 8 | n_bins... and inside a bin otherwise
    with vmat.Plan(prob) as plan:
        got = plan.dvh(torch.as_tensor(z, device="cuda"), 1.25, n_bins)
    n_edge = _check_against_oracle(got, z, prob.struct_id, prob.T.size, 1.25, n_bins)
    print(f"n_bins {n_bins}: {n_edge} voxels within FP32 rounding of a bin edge")


def test_dvh_exact_edges_vs_oracle():
    """Doses exactly on bin edges (dyadic, so FP32 and FP64 agree): every
    voxel goes up into the bin the edge opens."""
    prob = inputs.make_problem(inputs.small_config())
    grid = (np.arange(prob.n_vox) % 70) / 32.0  # 0 .. 2.156 in steps of 1/32
    z = grid.astype(np.float32)
    with vmat.Plan(prob) as plan:
        got = plan.dvh(torch.as_tensor(z, device="cuda"), 2.0, 64)
    ref = oracle.dvh(grid, prob.struct_id, prob.T.size, 2.0, 64)
    np.testing.assert_array_equal(got, ref)


def test_plan_dvh_vs_oracle():
    prob = inputs.make_problem(inputs.tiny_config())
    with vmat.Plan(prob) as plan:
        plan.colgen_run(kkt_tol=1e-6)
        z = plan.plan_dose()
        c = plan.dvh(z, 1.5, 300)
    zh = z.cpu().numpy()
    _check_against_oracle(c, zh, prob.struct_id, prob.T.size, 1.5, 300)
    np.testing.assert_array_equal(c.sum(axis=1), np.bincount(prob.struct_id, minlength=prob.T.size))
    m = quality.dvh_metrics(c, 1.5, prob.struct_names, rx=float(prob.T.max()))
    t = m["target"]
    assert t["D95"] <= t["mean"] <= t["D5"] + 1.5 / 300
