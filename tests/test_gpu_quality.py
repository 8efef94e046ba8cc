"""GPU dose-volume histograms against NumPy counts with the same FP32 bin
decision (exact), and the histogram of a plan's dose covering every voxel
of every structure once."""
import numpy as np
import pytest

from paper_1005_4396_b300 import inputs, quality

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import vmat  # noqa: E402


def _counts_np(z, sid, n_struct, dose_max, n_bins):
    s = np.float32(n_bins / dose_max)
    v = z.astype(np.float32) * s                      # FP32 product, round to nearest
    b = np.where(v > 0, np.floor(v), 0).astype(np.int64)
    b = np.minimum(b, n_bins - 1)
    out = np.zeros((n_struct, n_bins), np.int64)
    np.add.at(out, (sid.astype(np.int64), b), 1)
    return out


@pytest.mark.parametrize("n_bins", [1, 37, 1000])
def test_dvh_counts_exact(n_bins):
    prob = inputs.make_problem(inputs.small_config())
    z = (inputs.rng.uniform(120, prob.n_vox) * 1.3).astype(np.float32)
    z[::97] = 0.0
    z[1::89] = 2.0   # above dose_max: last bin
    with vmat.Plan(prob) as plan:
        got = plan.dvh(torch.as_tensor(z, device="cuda"), 1.25, n_bins)
    ref = _counts_np(z, prob.struct_id, prob.T.size, 1.25, n_bins)
    np.testing.assert_array_equal(got, ref)


def test_plan_dvh_covers_every_voxel():
    prob = inputs.make_problem(inputs.tiny_config())
    with vmat.Plan(prob) as plan:
        plan.colgen_run(kkt_tol=1e-6)
        z = plan.plan_dose()
        c = plan.dvh(z, 1.5, 300)
    np.testing.assert_array_equal(c.sum(axis=1), np.bincount(prob.struct_id, minlength=prob.T.size))
    m = quality.dvh_metrics(c, 1.5, prob.struct_names, rx=float(prob.T.max()))
    t = m["target"]
    assert t["D95"] <= t["mean"] <= t["D5"] + 1.5 / 300
