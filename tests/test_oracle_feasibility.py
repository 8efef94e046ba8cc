"""Pins of the oracle's dose-rate feasibility loop (Sec. 3): a feasible plan
is left alone; the loop ends feasible; the smoothing term never rises as
gamma grows (penalty-method property: for gamma2 > gamma1 the optima satisfy
(gamma2 - gamma1) (G(y2) - G(y1)) <= 0); and a very large gamma drives a plan
with every beam occupied to the common intensity of a 1-D problem."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs


@pytest.fixture(scope="module")
def tiny_plan():
    prob = inputs.make_problem(inputs.tiny_config())
    ref = oracle.colgen(prob, eps=1e-8)
    return prob, ref


def _rate(prob, y):
    return oracle.rate_violation(prob.theta_deg, y, 0.0, prob.cfg.cyclic)


def test_rate_violation_by_hand():
    theta = np.array([0.0, 10.0, 20.0, 350.0])
    y = np.array([1.0, 3.0, 2.0, 0.0])
    # ring pairs: |2|/10, |1|/10, |2|/330, and the wrap pair |1|/10
    assert oracle.rate_violation(theta, y, 0.0, cyclic=True) == pytest.approx(0.2)
    assert oracle.rate_violation(theta, y, 0.05, cyclic=False) == pytest.approx(0.15)
    assert oracle.rate_violation(theta[:1], y[:1], 0.3) == pytest.approx(-0.3)


def test_feasible_plan_is_left_alone(tiny_plan):
    prob, ref = tiny_plan
    out = oracle.dose_rate_feasibility(prob, ref["k"], ref["lleaf"], ref["rleaf"], ref["y"],
                                       max_rate=10 * _rate(prob, ref["y"]) + 1.0)
    assert out["rounds"] == 0 and out["gamma"] == prob.cfg.gamma
    np.testing.assert_array_equal(out["y"], ref["y"])
    assert out["cost"] == pytest.approx(ref["cost"][-1], rel=1e-9)


def test_loop_ends_feasible_and_smoothing_never_rises(tiny_plan):
    prob, ref = tiny_plan
    r0 = _rate(prob, ref["y"])
    out = oracle.dose_rate_feasibility(prob, ref["k"], ref["lleaf"], ref["rleaf"], ref["y"],
                                       max_rate=0.3 * r0, gamma_factor=2.0, eps=1e-10)
    assert out["rounds"] >= 1 and out["violation"] <= 0.0
    assert np.all(out["y"] >= 0)
    assert np.all(np.diff(out["G"]) <= 1e-7 * out["G"][0])
    assert out["gamma"] == pytest.approx(prob.cfg.gamma * 2.0 ** out["rounds"])


def test_huge_gamma_flattens_to_the_common_intensity(tiny_plan):
    """With every beam occupied, gamma -> infinity forces one common
    intensity c (Eq. 2 vanishes only at equal intensities); the deviation
    shrinks like 1/gamma, and c tends to the minimiser of the 1-D problem
    min_c sum_j F(c m_j), m = the sum of all aperture columns (Eq. 1), found
    here by bisection on its nondecreasing derivative."""
    prob, ref = tiny_plan
    cfg = prob.cfg
    assert sorted(ref["k"].tolist()) == list(range(cfg.n_angles))
    spread = {}
    for f in (1e7, 1e8):
        out = oracle.dose_rate_feasibility(prob, ref["k"], ref["lleaf"], ref["rleaf"], ref["y"],
                                           max_rate=0.0, gamma_factor=f, max_rounds=1, eps=1e-12)
        y = out["y"]
        spread[f] = (y.max() - y.min()) / y.max()
        c_mean = y.mean()
    assert 8.0 <= spread[1e7] / spread[1e8] <= 12.0
    assert spread[1e8] < 2e-3
    R = cfg.n_rows
    m = sum(oracle.aperture_dose(prob, k, ref["lleaf"][k * R:(k + 1) * R], ref["rleaf"][k * R:(k + 1) * R])
            for k in range(cfg.n_angles))
    Tv, av, bv = prob.voxel_params()

    def dphi(c):  # d/dc sum_j F(c m_j)
        e = c * m - Tv
        return float(np.sum(m * np.where(e > 0, 2 * bv * e, 2 * av * e)))

    lo, hi = 0.0, 1.0
    while dphi(hi) < 0:
        hi *= 2
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if dphi(mid) < 0 else (lo, mid)
    assert c_mean == pytest.approx(0.5 * (lo + hi), rel=2e-3)
