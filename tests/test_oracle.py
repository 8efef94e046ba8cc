"""Pins of the FP64 oracle against things other than itself: hand-worked
values, finite differences, brute-force enumeration, dense linear algebra, an
independent bound-constrained solver and invariants of the method."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.optimize

import oracle
from paper_1005_4396_b300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "handcalc.json")))


# ------------------------------------------------------------------ Eq. 1, Eq. 2
def test_eq1_hand_values():
    L = oracle.lib()
    for c in GOLD["eq1_voxel_cost"]["cases"]:
        assert L.vo_F(c["z"], c["T"], c["alpha"], c["beta"]) == pytest.approx(c["F"], abs=1e-15)
        assert L.vo_dF(c["z"], c["T"], c["alpha"], c["beta"]) == pytest.approx(c["dF"], abs=1e-15)


def test_eq1_derivative_matches_finite_differences():
    rng = np.random.default_rng(0)
    L = oracle.lib()
    h = 1e-6
    for _ in range(500):
        T, a, b = rng.uniform(0.2, 1.5), rng.choice([0.0, rng.uniform(0.1, 3)]), rng.uniform(0.05, 5)
        z = rng.uniform(0, 2)
        if abs(z - T) < 10 * h:
            continue
        fd = (L.vo_F(z + h, T, a, b) - L.vo_F(z - h, T, a, b)) / (2 * h)
        an = L.vo_dF(z, T, a, b)
        assert abs(fd - an) <= 1e-8 * max(abs(an), 1.0)


def test_eq1_vector_forms_sum_the_scalar_form():
    rng = np.random.default_rng(1)
    sid = rng.integers(0, 4, 1000).astype(np.uint8)
    T = np.array([0.0, 0.6, 1.0, 0.5]); al = np.array([0, 0, 1, 0.0]); be = np.array([0, 0.05, 1, 0.5])
    z = rng.uniform(0, 1.5, 1000)
    L = oracle.lib()
    ref = sum(L.vo_F(z[j], T[sid[j]], al[sid[j]], be[sid[j]]) for j in range(1000))
    assert oracle.voxel_cost(z, sid, T, al, be) == pytest.approx(ref, rel=1e-13)
    fp = oracle.voxel_dcost(z, sid, T, al, be)
    assert all(fp[j] == L.vo_dF(z[j], T[sid[j]], al[sid[j]], be[sid[j]]) for j in range(1000))


def test_eq2_hand_values():
    for c in GOLD["eq2_smoothing"]["cases"]:
        assert oracle.G(c["theta"], c["y"], c["cyclic"]) == pytest.approx(c["G"], rel=1e-14)
        if "dG" in c:
            np.testing.assert_allclose(oracle.dG(c["theta"], c["y"], c["cyclic"]), c["dG"], rtol=1e-14)


@pytest.mark.parametrize("cyclic", [True, False])
def test_eq2_gradient_and_homogeneity(cyclic):
    rng = np.random.default_rng(2)
    theta = np.sort(rng.uniform(0, 360, 17))
    y = rng.uniform(0, 1, 17)
    g = oracle.dG(theta, y, cyclic)
    h = 1e-6
    for k in range(17):
        e = np.zeros(17); e[k] = h
        fd = (oracle.G(theta, y + e, cyclic) - oracle.G(theta, y - e, cyclic)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k]))
    # G is a quadratic form: G(c y) = c^2 G(y), and constant y costs nothing
    assert oracle.G(theta, 3 * y, cyclic) == pytest.approx(9 * oracle.G(theta, y, cyclic), rel=1e-13)
    assert oracle.G(theta, np.full(17, 0.7), cyclic) == pytest.approx(0.0, abs=1e-15)


# ------------------------------------------------------------------ dose / price
def _dense(prob):
    Dm = np.zeros((prob.n_beamlets, prob.n_vox))
    rows = np.repeat(np.arange(prob.n_beamlets), np.diff(prob.row_ptr))
    np.add.at(Dm, (rows, prob.vox_idx), prob.val)
    return Dm


def test_dose_and_price_match_dense_products(small_problem):
    p = small_problem
    Dm = _dense(p)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, p.n_beamlets)
    f = rng.normal(size=p.n_vox)
    np.testing.assert_allclose(oracle.dose(p, x), Dm.T @ x, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(oracle.price(p, f), Dm @ f, rtol=1e-12, atol=1e-12)
    mask = (np.arange(p.cfg.n_angles) % 3 == 0).astype(np.uint8)
    g = oracle.price(p, f, mask)
    beam = np.arange(p.n_beamlets) // (p.cfg.n_rows * p.cfg.n_cols)
    np.testing.assert_allclose(g[mask[beam] == 1], (Dm @ f)[mask[beam] == 1], rtol=1e-12, atol=1e-12)
    assert np.all(g[mask[beam] == 0] == 0)


def test_adjoint_identity(tiny_problem):
    p = tiny_problem
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = rng.uniform(0, 1, p.n_beamlets)
        w = rng.normal(size=p.n_vox)
        lhs = np.dot(oracle.dose(p, x), w)
        rhs = np.dot(x, oracle.price(p, w))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def test_aperture_dose_is_dose_of_aperture_fluence(small_problem):
    p = small_problem
    cfg = p.cfg
    l, r = inputs.random_apertures(5, cfg)
    Dm = _dense(p)
    R, C = cfg.n_rows, cfg.n_cols
    for k in [0, 3, cfg.n_angles - 1]:
        col = oracle.aperture_dose(p, k, l[k * R:(k + 1) * R], r[k * R:(k + 1) * R])
        y = np.zeros(cfg.n_angles); y[k] = 1.0
        x = oracle.aperture_fluence(cfg, l, r, y)
        np.testing.assert_allclose(col, Dm.T @ x, rtol=1e-12, atol=1e-13)
    # adjoint of the fluence map: <A y, g> = <y, A^T g>
    y = rng_y = np.random.default_rng(6).uniform(0, 1, cfg.n_angles)
    g = np.random.default_rng(7).normal(size=p.n_beamlets)
    assert np.dot(oracle.aperture_fluence(cfg, l, r, y), g) == pytest.approx(
        np.dot(rng_y, oracle.aperture_adjoint(cfg, l, r, g)), rel=1e-12)


# ------------------------------------------------------------------ pricing
def test_row_scan_hand_values():
    c = GOLD["row_scan"]
    for case in c["cases"]:
        for f32 in (False, True):
            v, l, r = oracle.row_scan(c["g"], case["Llo"], case["Lhi"], case["Rlo"], case["Rhi"], f32=f32)
            assert (v, l, r) == (case["value"], case["l"], case["r"])


def _brute_row(g, Llo, Lhi, Rlo, Rhi):
    best = None
    for l in range(Llo, Lhi + 1):
        for r in range(max(l, Rlo), Rhi + 1):
            key = (sum(g[l:r]), r - l, l)
            if best is None or key < best:
                best = key
    return None if best is None else (best[0], best[2], best[2] + best[1])


@pytest.mark.parametrize("f32", [False, True])
def test_row_scan_matches_enumeration(f32):
    # integer prices make every sum exact, so exact ties exercise the tie-break
    rng = np.random.default_rng(8)
    for _ in range(4000):
        C = int(rng.integers(1, 9))
        g = [float(v) for v in rng.integers(-3, 4, C)]
        if rng.uniform() < 0.2:
            g = [0.0] * C
        a, b = sorted(rng.integers(0, C + 1, 2)); c_, d = sorted(rng.integers(0, C + 1, 2))
        ref = _brute_row(g, a, b, c_, d)
        got = oracle.row_scan(g, a, b, c_, d, f32=f32)
        assert got == ref, (g, a, b, c_, d)


def _limits_brute(N, R, C, s, cyclic, occ, ll, rr, k):
    """Leaf limits straight from their definition: every leaf within s*d
    columns of the same leaf of the nearest beam with an aperture on each side."""
    out = []
    for row in range(R):
        cons = []
        for step in (-1, 1):
            for d in range(1, N):
                q = k + step * d
                if cyclic:
                    q %= N
                elif not 0 <= q < N:
                    break
                if occ[q]:
                    cons.append((d, ll[q * R + row], rr[q * R + row]))
                    break
        feas_l = [l for l in range(C + 1) if all(abs(l - a) <= s * d for d, a, _ in cons)]
        feas_r = [r for r in range(C + 1) if all(abs(r - b) <= s * d for d, _, b in cons)]
        out.append((min(feas_l), max(feas_l), min(feas_r), max(feas_r)))
    return out


@pytest.mark.parametrize("cyclic", [True, False])
def test_leaf_limits_definition_and_nonempty(cyclic):
    rng = np.random.default_rng(9)
    N, R, C, s = 9, 3, 7, 1
    cfg = inputs.small_config(n_angles=N, n_rows=R, n_cols=C, max_leaf_step=s, cyclic=cyclic)
    for trial in range(60):
        # build a plan one beam at a time under the limits themselves
        occ = np.zeros(N, np.uint8); ll = np.zeros(N * R, np.int16); rr = np.zeros(N * R, np.int16)
        for k in rng.permutation(N):
            lim = oracle.leaf_limits(N, R, C, s, cyclic, occ, ll, rr, k)
            ref = _limits_brute(N, R, C, s, cyclic, occ, ll, rr, k)
            assert [tuple(lim[:, row]) for row in range(R)] == ref
            for row in range(R):
                Llo, Lhi, Rlo, Rhi = lim[:, row]
                opts = [(l, r) for l in range(Llo, Lhi + 1) for r in range(max(l, Rlo), Rhi + 1)]
                assert opts, "feasible set must be non-empty"
                l, r = opts[rng.integers(len(opts))]
                ll[k * R + row], rr[k * R + row] = l, r
            occ[k] = 1
        # the final plan keeps adjacent beams within s columns
        for k in range(N if cyclic else N - 1):
            k1 = (k + 1) % N
            assert np.all(np.abs(ll[k * R:(k + 1) * R] - ll[k1 * R:(k1 + 1) * R]) <= s)
            assert np.all(np.abs(rr[k * R:(k + 1) * R] - rr[k1 * R:(k1 + 1) * R]) <= s)


def _brute_pricing(N, R, C, s, cyclic, occ, ll, rr, g):
    best = None
    for k in range(N):
        if occ[k]:
            continue
        lim = _limits_brute(N, R, C, s, cyclic, occ, ll, rr, k)
        p = 0.0
        rows = []
        for row in range(R):
            gr = list(g[(k * R + row) * C:(k * R + row + 1) * C])
            v, l, r = _brute_row(gr, *lim[row])
            p += v
            rows.append((l, r))
        if best is None or p < best[0]:
            best = (p, k, rows)
    return best


@pytest.mark.parametrize("f32", [False, True])
def test_pricing_matches_enumeration(f32):
    rng = np.random.default_rng(10)
    N, R, C, s = 7, 3, 6, 1
    for trial in range(150):
        cyclic = bool(trial % 2)
        cfg = inputs.small_config(n_angles=N, n_rows=R, n_cols=C, max_leaf_step=s, cyclic=cyclic)
        occ = np.zeros(N, np.uint8); ll = np.zeros(N * R, np.int16); rr = np.zeros(N * R, np.int16)
        nocc = int(rng.integers(0, N))
        for k in rng.permutation(N)[:nocc]:
            lim = _limits_brute(N, R, C, s, cyclic, occ, ll, rr, k)
            for row in range(R):
                Llo, Lhi, Rlo, Rhi = lim[row]
                opts = [(l, r) for l in range(Llo, Lhi + 1) for r in range(max(l, Rlo), Rhi + 1)]
                ll[k * R + row], rr[k * R + row] = opts[rng.integers(len(opts))]
            occ[k] = 1
        g = rng.integers(-4, 5, N * R * C).astype(np.float64) * 0.25  # dyadic: exact sums
        got = oracle.pricing(cfg, occ, ll, rr, g, f32=f32)
        p, k, rows = _brute_pricing(N, R, C, s, cyclic, occ, ll, rr, g)
        assert got["k"] == k and got["p"] == p
        assert [(int(a), int(b)) for a, b in zip(got["l"], got["r"])] == rows
        assert got["p2"] >= got["p"]


# ------------------------------------------------------------------ master problem
def _phi(z, w, sid, T, al, be, theta, y, d, gamma, cyclic, t):
    return oracle.voxel_cost(z + t * w, sid, T, al, be) + gamma * oracle.G(theta, y + t * d, cyclic)


def test_line_search_is_the_exact_minimiser():
    rng = np.random.default_rng(11)
    T = np.array([0.0, 0.6, 1.0, 0.5]); al = np.array([0, 0, 1, 0.0]); be = np.array([0, 0.05, 1, 0.5])
    theta = np.arange(8) * 45.0
    for trial in range(40):
        V = 300
        sid = rng.integers(1, 4, V).astype(np.uint8)
        z = rng.uniform(0, 1.5, V)
        w = rng.normal(size=V) * rng.uniform(0.1, 2)
        y = rng.uniform(0, 1, 8); d = rng.normal(size=8) * 0.3
        gamma = 0.1
        gdot = float(np.dot(oracle.dG(theta, y, True), d)); Gd = oracle.G(theta, d, True)
        t = oracle.line_search(z, w, sid, T, al, be, gdot, Gd, gamma)
        f = lambda s: _phi(z, w, sid, T, al, be, theta, y, d, gamma, True, s)
        ref = scipy.optimize.minimize_scalar(f, bounds=(0, 1), method="bounded",
                                             options=dict(xatol=1e-12))
        assert 0.0 <= t <= 1.0
        assert f(t) <= f(ref.x) + 1e-12 * max(1.0, abs(f(ref.x)))
        # optimality of t by one-sided differences
        h = 1e-7
        if t > h:
            assert f(t - h) >= f(t) - 1e-12
        if t < 1 - h:
            assert f(t + h) >= f(t) - 1e-12


def _laplacian(theta, cyclic):
    N = len(theta)
    Lp = np.zeros((N, N))
    for k in range(N if cyclic else N - 1):
        k1 = (k + 1) % N
        gap = theta[k1] - theta[k] if k1 > k else theta[0] + 360 - theta[k]
        e = np.zeros(N); e[k1] = 1; e[k] = -1
        Lp += np.outer(e, e) / gap
    return Lp


def test_master_closed_form_quadratic_instance():
    """Targets only, alpha = beta, so F is an exact quadratic; with a solution
    inside y > 0 the master's optimum is y* = (M^T A M + gamma L)^-1 M^T A T."""
    rng = np.random.default_rng(12)
    N, V = 6, 400
    theta = np.arange(N) * 60.0
    M = rng.uniform(0.0, 1.0, (N, V)) * (rng.uniform(size=(N, V)) < 0.6)
    sid = rng.integers(1, 3, V).astype(np.uint8)
    T = np.array([0.0, 1.0, 0.8]); al = np.array([0.0, 1.0, 2.5]); be = al.copy()
    gamma = 0.3
    A = np.diag(al[sid])
    H = M @ A @ M.T + gamma * _laplacian(theta, True)
    cho = np.linalg.cholesky(H)
    ystar = np.linalg.solve(cho.T, np.linalg.solve(cho, M @ A @ T[sid]))
    assert np.all(ystar > 0)
    res = oracle.master(M, np.arange(N), theta, sid, T, al, be, gamma, True, np.zeros(N), eps=1e-12)
    assert res["status"] == 0
    np.testing.assert_allclose(res["y"], ystar, rtol=1e-8, atol=1e-10)
    fstar = np.sum(al[sid] * (M.T @ ystar - T[sid]) ** 2) + gamma * ystar @ _laplacian(theta, True) @ ystar
    assert res["cost"] == pytest.approx(fstar, rel=1e-12)


@pytest.mark.parametrize("cyclic", [True, False])
def test_master_matches_lbfgsb_with_active_bounds(cyclic):
    rng = np.random.default_rng(13 + cyclic)
    N, V = 10, 800
    theta = np.sort(rng.choice(np.arange(0, 360, 5), N, replace=False)).astype(float)
    cols = [0, 1, 3, 4, 6, 7, 9]
    M = rng.uniform(0, 1, (len(cols), V)) * (rng.uniform(size=(len(cols), V)) < 0.3)
    sid = rng.integers(1, 4, V).astype(np.uint8)
    T = np.array([0.0, 0.6, 1.0, 0.5]); al = np.array([0, 0, 1, 0.0]); be = np.array([0, 0.05, 1, 3.0])
    gamma = 0.05
    res = oracle.master(M, np.array(cols), theta, sid, T, al, be, gamma, cyclic, np.zeros(N), eps=1e-12)
    assert res["status"] == 0 and np.all(res["y"] >= 0)
    free = np.zeros(N, bool); free[cols] = True
    assert np.all(res["y"][~free] == 0)

    def fg(v):
        y = np.zeros(N); y[cols] = v
        z = M.T @ v
        f = oracle.voxel_cost(z, sid, T, al, be) + gamma * oracle.G(theta, y, cyclic)
        g = M @ oracle.voxel_dcost(z, sid, T, al, be) + gamma * oracle.dG(theta, y, cyclic)[cols]
        return f, g

    ref = scipy.optimize.minimize(fg, np.full(len(cols), 0.1), jac=True, method="L-BFGS-B",
                                  bounds=[(0, None)] * len(cols),
                                  options=dict(ftol=1e-15, gtol=1e-12, maxiter=20000, maxcor=30))
    assert res["cost"] == pytest.approx(ref.fun, rel=1e-10)
    assert res["cost"] <= ref.fun * (1 + 1e-12)
    # KKT at exit: rho small relative to the start, y >= 0
    assert res["rho"] <= 1e-12 * max(res["rho0"], 1e-300) * 1.0000001


def test_colgen_invariants(tiny_problem):
    p = tiny_problem
    cfg = p.cfg
    rec = oracle.colgen(p, eps=1e-6)
    N, R = cfg.n_angles, cfg.n_rows
    assert sorted(rec["k"].tolist()) == list(range(N))           # each beam once
    assert np.all(np.diff(rec["cost"]) <= 1e-12 * rec["cost"][:-1])  # cost never rises
    assert np.all(rec["status"] == 0)
    assert np.all(rec["y"] >= 0)
    ll, rr = rec["lleaf"].astype(int), rec["rleaf"].astype(int)
    assert np.all(ll <= rr) and ll.min() >= 0 and rr.max() <= cfg.n_cols
    for k in range(N):                                            # leaf travel, ring
        k1 = (k + 1) % N
        assert np.all(np.abs(ll[k * R:(k + 1) * R] - ll[k1 * R:(k1 + 1) * R]) <= cfg.max_leaf_step)
        assert np.all(np.abs(rr[k * R:(k + 1) * R] - rr[k1 * R:(k1 + 1) * R]) <= cfg.max_leaf_step)
    # the final cost is the model's objective at the final plan (Eq. 3)
    x = oracle.aperture_fluence(cfg, rec["lleaf"], rec["rleaf"], rec["y"])
    z = oracle.dose(p, x)
    f = oracle.voxel_cost(z, p.struct_id, p.T, p.alpha, p.beta) + cfg.gamma * oracle.G(p.theta_deg, rec["y"])
    assert rec["cost"][-1] == pytest.approx(f, rel=1e-10)
    np.testing.assert_allclose(rec["z"], z, rtol=1e-9, atol=1e-12)


def test_colgen_replay_reproduces_itself(small_problem):
    p = small_problem
    rec = oracle.colgen(p, eps=1e-8)
    R = p.cfg.n_rows
    fl = np.array([rec["lleaf"][k * R:(k + 1) * R] for k in rec["k"]])
    fr = np.array([rec["rleaf"][k * R:(k + 1) * R] for k in rec["k"]])
    rep = oracle.colgen(p, eps=1e-8, forced=(rec["k"], fl, fr))
    assert np.array_equal(rep["k"], rec["k"])
    np.testing.assert_array_equal(rep["cost"], rec["cost"])


def test_pricing_single_precision_resolution_by_hand():
    """One free beam with one row g = [1, -2, -1, 3, -4] (prefix sums 1, -1,
    -2, 1, -3, largest |P| = 3): the resolution of the beam decision is one
    unit in the last place of 3 in single precision, 2^-23 * 3 (no runner-up
    beam); the row's chosen interval [4, 5) has value -4 and the least value
    strictly above it is -3 ([1, 3)), so its margin is 1, i.e.
    1 / (2^-22 * 3) units of the row's resolution."""
    cfg = inputs.small_config(n_angles=1, n_rows=1, n_cols=5, max_leaf_step=5)
    g = np.array(GOLD["row_scan"]["g"], dtype=np.float64)
    out = oracle.pricing(cfg, np.zeros(1, np.uint8), np.zeros(1, np.int16), np.zeros(1, np.int16),
                         g, f32=True)
    assert (out["k"], int(out["l"][0]), int(out["r"][0])) == (0, 4, 5)
    assert out["f32_res"] == 2.0 ** -23 * 3
    assert out["row_res"] == pytest.approx(1.0 / (2.0 ** -22 * 3), rel=1e-15)
