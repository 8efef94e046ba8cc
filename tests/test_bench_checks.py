"""The benchmark's FP64 NumPy checks (dose, price, cost, smoothing gradient,
aperture fluence, dose-rate variation) agree with the oracle on a small
problem, so the errors it reports beside its timings mean what they say."""
import numpy as np
import pytest

import bench
import oracle
from paper_1005_4396_b300 import inputs


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.small_config())


def test_bench_fp64_checks_match_the_oracle(small):
    prob, cfg = small, small.cfg
    rng = np.random.default_rng(7)
    x = rng.uniform(size=prob.n_beamlets)
    z = bench._dose64(prob, x)
    np.testing.assert_allclose(z, oracle.dose(prob, x), rtol=1e-12, atol=1e-14)
    f = rng.normal(size=prob.n_vox)
    np.testing.assert_allclose(bench._price64(prob, f), oracle.price(prob, f), rtol=1e-12, atol=1e-12)
    c, fp = bench._cost64(prob, z)
    assert c == pytest.approx(oracle.voxel_cost(z, prob.struct_id, prob.T, prob.alpha, prob.beta), rel=1e-12)
    np.testing.assert_allclose(fp, oracle.voxel_dcost(z, prob.struct_id, prob.T, prob.alpha, prob.beta),
                               rtol=1e-12, atol=1e-15)
    l, r = inputs.random_apertures(8, cfg)
    y = rng.uniform(size=cfg.n_angles)
    np.testing.assert_array_equal(bench._fluence64(cfg, l, r, y), oracle.aperture_fluence(cfg, l, r, y))
    for cyclic in (True, False):
        np.testing.assert_allclose(bench._dG64(prob.theta_deg, y, cyclic),
                                   oracle.dG(prob.theta_deg, y, cyclic), rtol=1e-12, atol=1e-15)
        assert bench._rate64(prob.theta_deg, y, cyclic) == pytest.approx(
            oracle.rate_violation(prob.theta_deg, y, 0.0, cyclic), rel=1e-12)
