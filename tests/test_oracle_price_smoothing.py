"""Pins of the oracle's exact reduced-cost pricing (the smoothing derivative
entering the price of a new column, Sec. 2.2 with Eq. 2-3): the price of a
beam's aperture with the offset is the derivative of the Eq. 3 objective
along the new column, measured by finite differences of the cost functions;
the pricing picks the least such derivative over every free beam and every
feasible aperture (brute force); gamma = 0 or y = 0 reduce to the literal
pricing; the offset has the closed form -2 gamma sum_q y_q / gap."""
import dataclasses
import itertools

import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs


def _state(prob, n):
    """Occupancy, leaves, y and z after the first n column-generation
    iterations (literal pricing)."""
    cfg = prob.cfg
    rec = oracle.colgen(prob, n_iter=n, eps=1e-12)
    occ = np.zeros(cfg.n_angles, np.uint8)
    occ[rec["k"]] = 1
    return occ, rec["lleaf"], rec["rleaf"], rec["y"], rec["z"]


def _derivative(prob, y, z, k, l, r, eps):
    """d/dt of Eq. 3 at t = 0+ along the column of beam k with leaves l, r
    (dose z + t m, intensity y + t e_k), by the three-point one-sided
    difference that is exact for a quadratic (Eq. 1 is piecewise quadratic,
    Eq. 2 quadratic)."""
    cfg = prob.cfg
    m = oracle.aperture_dose(prob, k, l, r)
    e = np.zeros_like(y)
    e[k] = 1.0

    def c(t):
        return (oracle.voxel_cost(z + t * m, prob.struct_id, prob.T, prob.alpha, prob.beta) +
                cfg.gamma * oracle.G(prob.theta_deg, y + t * e, cfg.cyclic))
    c0, c1, c2 = c(0.0), c(eps), c(2 * eps)
    return (4 * c1 - c2 - 3 * c0) / (2 * eps)


def test_offset_closed_form():
    theta = np.array([0.0, 90.0, 180.0, 270.0])
    y = np.array([1.0, 0.0, 2.0, 0.0])
    g = 0.5
    ring = oracle.smoothing_offset(theta, y, g, cyclic=True)
    path = oracle.smoothing_offset(theta, y, g, cyclic=False)
    # free beams 1 and 3: -2 gamma (y_left / gap + y_right / gap)
    assert ring[1] == pytest.approx(-2 * g * (1.0 / 90 + 2.0 / 90), rel=1e-15)
    assert ring[3] == pytest.approx(-2 * g * (2.0 / 90 + 1.0 / 90), rel=1e-15)
    assert path[1] == pytest.approx(-2 * g * (1.0 / 90 + 2.0 / 90), rel=1e-15)
    assert path[3] == pytest.approx(-2 * g * (2.0 / 90), rel=1e-15)  # no wrap neighbour
    # uneven gaps
    theta = np.array([0.0, 10.0, 40.0])
    y = np.array([3.0, 0.0, 1.0])
    off = oracle.smoothing_offset(theta, y, 1.0, cyclic=True)
    assert off[1] == pytest.approx(-2 * (3.0 / 10 + 1.0 / 30), rel=1e-15)


@pytest.mark.parametrize("cyclic", [True, False])
def test_pricing_is_least_directional_derivative(cyclic):
    """Every free beam, every feasible aperture: the derivative of Eq. 3
    along its column by finite differences; the pricing with the offset picks
    the least one and reports it as p."""
    cfg = inputs.small_config(nx=10, ny=9, nz=3, n_angles=7, n_rows=2, n_cols=4, max_leaf_step=1,
                              cyclic=cyclic, gamma=5.0)
    prob = inputs.make_problem(cfg)
    N, R, C, s = cfg.n_angles, cfg.n_rows, cfg.n_cols, cfg.max_leaf_step
    occ, ll, rr, y, z = _state(prob, 3)
    assert np.all(y[occ == 1] > 0)
    fp = oracle.voxel_dcost(z, prob.struct_id, prob.T, prob.alpha, prob.beta)
    g = oracle.price(prob, fp, (occ == 0).astype(np.uint8))
    off = oracle.smoothing_offset(prob.theta_deg, y, cfg.gamma, cyclic)
    got = oracle.pricing(cfg, occ, ll, rr, g, offset=off)
    lit = oracle.pricing(cfg, occ, ll, rr, g)
    best, best_key, scale, gap = np.inf, None, 0.0, 0.0
    for k in np.flatnonzero(occ == 0):
        Llo, Lhi, Rlo, Rhi = oracle.leaf_limits(N, R, C, s, cyclic, occ, ll, rr, int(k))
        rows = [[(l, r) for l in range(Llo[q], Lhi[q] + 1) for r in range(max(l, Rlo[q]), Rhi[q] + 1)]
                for q in range(R)]
        for ap in itertools.product(*rows):
            l = np.array([a[0] for a in ap], np.int16)
            r = np.array([a[1] for a in ap], np.int16)
            d = _derivative(prob, y, z, int(k), l, r, 1e-6)
            scale = max(scale, abs(d))
            beamlet_sum = sum(g[(k * R + q) * C + c] for q in range(R) for c in range(l[q], r[q]))
            gap = max(gap, abs(d - beamlet_sum - off[k]))
            if d < best - 1e-9:
                best, best_key = d, (int(k), l, r)
    tol = 1e-7 * scale
    assert got["p"] == pytest.approx(best, abs=tol)
    d_got = _derivative(prob, y, z, got["k"], got["l"], got["r"], 1e-6)
    assert d_got == pytest.approx(got["p"], abs=tol)  # p is the derivative of its own column
    assert got["k"] == best_key[0]
    # every aperture: derivative = its summed beamlet price + the offset of
    # its beam, and the offset matters (the literal price misses it)
    assert gap <= tol
    assert np.abs(off[occ == 0]).max() > 100 * tol
    assert lit["p"] == pytest.approx(_derivative(prob, y, z, lit["k"], lit["l"], lit["r"], 1e-6)
                                     - off[lit["k"]], abs=tol)


def test_colgen_records_exact_reduced_costs():
    """The loop passes the offset of the current y: each recorded price is
    the derivative of Eq. 3 along the column chosen at that iteration."""
    cfg = inputs.small_config(gamma=5.0)
    prob = inputs.make_problem(cfg)
    R = cfg.n_rows
    rec = oracle.colgen(prob, eps=1e-12, price_smoothing=True)
    for t in (0, 2, 5, 9):
        occ, ll, rr, y, z = _state_smoothing(prob, t)
        k = int(rec["k"][t])
        l = rec["lleaf"][k * R:(k + 1) * R]
        r = rec["rleaf"][k * R:(k + 1) * R]
        d = _derivative(prob, y, z, k, l, r, 1e-6)
        assert d == pytest.approx(rec["p"][t], rel=1e-6, abs=1e-9), t


def _state_smoothing(prob, n):
    rec = oracle.colgen(prob, n_iter=n, eps=1e-12, price_smoothing=True)
    occ = np.zeros(prob.cfg.n_angles, np.uint8)
    occ[rec["k"]] = 1
    return occ, rec["lleaf"], rec["rleaf"], rec["y"], rec["z"]


def test_reduces_to_literal_pricing():
    """gamma = 0: no smoothing term, the same plan; the first iteration
    (y = 0) prices identically at any gamma."""
    cfg = inputs.small_config(gamma=0.0)
    prob = inputs.make_problem(cfg)
    a = oracle.colgen(prob)
    b = oracle.colgen(prob, price_smoothing=True)
    np.testing.assert_array_equal(a["k"], b["k"])
    np.testing.assert_array_equal(a["lleaf"], b["lleaf"])
    np.testing.assert_array_equal(a["cost"], b["cost"])
    prob5 = dataclasses.replace(prob, cfg=dataclasses.replace(cfg, gamma=5.0))
    a = oracle.colgen(prob5, n_iter=1)
    b = oracle.colgen(prob5, n_iter=1, price_smoothing=True)
    assert a["k"][0] == b["k"][0] and a["p"][0] == b["p"][0]


def test_offset_never_raises_a_price():
    """y >= 0, so the smoothing derivative at a free beam is <= 0: every
    price with the offset is at most the literal one, and strictly below it
    next to a beam with intensity."""
    cfg = inputs.small_config(gamma=5.0)
    prob = inputs.make_problem(cfg)
    occ, ll, rr, y, z = _state(prob, 4)
    off = oracle.smoothing_offset(prob.theta_deg, y, cfg.gamma, cfg.cyclic)
    free = np.flatnonzero(occ == 0)
    assert np.all(off[free] <= 0)
    N = cfg.n_angles
    for k in free:
        nb = [(k - 1) % N, (k + 1) % N]
        if any(y[q] > 0 for q in nb):
            assert off[k] < 0
        else:
            assert off[k] == 0
