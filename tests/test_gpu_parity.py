"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle on
seeded inputs.  Tolerances: FP32 dose, price and cost within 1e-5 relative;
pricing decisions bit-exact when both sides take them in FP32 on the same
prices; column-generation decisions bit-exact except at near-ties (margin
<= 1e-6, tests/decisions.py); reduced-precision D within 0.5% of the
largest prescription."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs

import decisions as dec

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import vmat  # noqa: E402

@pytest.fixture(scope="module")
def tiny():
    return inputs.make_problem(inputs.tiny_config())


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.small_config())


@pytest.fixture(scope="module")
def tiny_plan(tiny):
    p = dec.precise(vmat.Plan(tiny))
    yield p
    p.close()


@pytest.fixture(scope="module")
def small_plan(small):
    p = vmat.Plan(small)
    yield p
    p.close()


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _feasible_plan(cfg, rng, n_occ):
    """Random beams with apertures built one at a time inside the leaf limits."""
    N, R, C, s = cfg.n_angles, cfg.n_rows, cfg.n_cols, cfg.max_leaf_step
    occ = np.zeros(N, np.uint8)
    ll = np.zeros(N * R, np.int16)
    rr = np.zeros(N * R, np.int16)
    order = []
    for k in rng.permutation(N)[:n_occ]:
        lim = oracle.leaf_limits(N, R, C, s, cfg.cyclic, occ, ll, rr, k)
        for row in range(R):
            Llo, Lhi, Rlo, Rhi = lim[:, row]
            opts = [(l, r) for l in range(Llo, Lhi + 1) for r in range(max(l, Rlo), Rhi + 1)]
            ll[k * R + row], rr[k * R + row] = opts[rng.integers(len(opts))]
        occ[k] = 1
        order.append(int(k))
    return occ, ll, rr, order


# ------------------------------------------------------------------ info / setup
def test_active_voxels_and_sizes(tiny_plan, tiny):
    inf = tiny_plan.info
    assert inf["n_vox"] == tiny.n_vox and inf["nnz"] == tiny.nnz
    assert inf["n_active"] == np.unique(tiny.vox_idx).size
    assert inf["n_beamlets"] == tiny.n_beamlets


# ------------------------------------------------------------------ dose
@pytest.mark.parametrize("which", ["tiny", "small"])
def test_dose_parity(which, tiny, small, tiny_plan, small_plan):
    prob, plan = (tiny, tiny_plan) if which == "tiny" else (small, small_plan)
    x = inputs.rng.uniform(21, prob.n_beamlets).astype(np.float32)
    z, fp, cost = plan.dose(_cuda(x))
    z_or = oracle.dose(prob, x.astype(np.float64))
    zmax = np.abs(z_or).max()
    np.testing.assert_allclose(z.cpu().numpy(), z_or, rtol=1e-5, atol=1e-6 * zmax)
    fp_or = oracle.voxel_dcost(z_or, prob.struct_id, prob.T, prob.alpha, prob.beta)
    wmax = 2 * max(prob.alpha.max(), prob.beta.max())
    np.testing.assert_allclose(fp.cpu().numpy(), fp_or, rtol=0,
                               atol=wmax * (1e-5 * np.abs(z_or) + 1e-6 * zmax).max())
    c_or = oracle.voxel_cost(z_or, prob.struct_id, prob.T, prob.alpha, prob.beta)
    assert cost == pytest.approx(c_or, rel=1e-5)


# ------------------------------------------------------------------ price
@pytest.mark.parametrize("masked", [False, True])
def test_price_parity(tiny, tiny_plan, masked):
    prob = tiny
    f = inputs.rng.normal(22, prob.n_vox).astype(np.float32)
    mask = None
    if masked:
        mask = (np.arange(prob.cfg.n_angles) % 4 != 1).astype(np.uint8)
    g = tiny_plan.price(_cuda(f), mask).cpu().numpy()
    g_or = oracle.price(prob, f.astype(np.float64), mask)
    scale = oracle.price(prob, np.abs(f.astype(np.float64)), mask)  # sum_j |D_ij f_j|
    assert np.all(np.abs(g - g_or) <= 1e-5 * scale + 1e-30)
    if masked:
        beam = np.arange(prob.n_beamlets) // (prob.cfg.n_rows * prob.cfg.n_cols)
        assert np.all(g[mask[beam] == 0] == 0)


def test_adjoint_identity_on_gpu(tiny, tiny_plan):
    x = inputs.rng.uniform(23, tiny.n_beamlets).astype(np.float32)
    w = inputs.rng.normal(24, tiny.n_vox).astype(np.float32)
    z, _, _ = tiny_plan.dose(_cuda(x))
    g = tiny_plan.price(_cuda(w))
    lhs = float(np.dot(z.cpu().numpy().astype(np.float64), w))
    rhs = float(np.dot(x.astype(np.float64), g.cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * np.dot(np.abs(z.cpu().numpy()), np.abs(w))


# ------------------------------------------------------------------ pricing
@pytest.mark.parametrize("cyclic", [True, False])
def test_pricing_bit_exact(small, cyclic):
    """Same FP32 prices on both sides -> identical beam, leaves and price."""
    cfg = inputs.small_config(cyclic=cyclic, max_leaf_step=1)
    prob = inputs.Problem(**{**small.__dict__, "cfg": cfg})
    rng = np.random.default_rng(30 + cyclic)
    with vmat.Plan(prob) as plan:
        for trial in range(12):
            plan.reset()
            occ, ll, rr, order = _feasible_plan(cfg, rng, int(rng.integers(0, cfg.n_angles - 1)))
            R = cfg.n_rows
            for k in order:
                plan.add_column(k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
            g = rng.normal(size=prob.n_beamlets).astype(np.float32)
            if trial % 3 == 0:  # exact zero prices: exact ties
                g[rng.uniform(size=g.size) < 0.5] = 0.0
            got = plan.pricing_select(_cuda(g))
            ref = oracle.pricing(cfg, occ, ll, rr, g.astype(np.float64), f32=True)
            assert got["k"] == ref["k"]
            np.testing.assert_array_equal(got["l"], ref["l"])
            np.testing.assert_array_equal(got["r"], ref["r"])
            assert got["p"] == ref["p"]
            assert got["p2"] == ref["p2"]


# ------------------------------------------------------------------ aperture column
def test_aperture_column_parity(tiny, tiny_plan):
    cfg = tiny.cfg
    rng = np.random.default_rng(40)
    tiny_plan.reset()
    occ, ll, rr, order = _feasible_plan(cfg, rng, 5)
    R = cfg.n_rows
    for k in order:
        tiny_plan.add_column(k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
    for k in order[:3]:
        y = np.zeros(cfg.n_angles)
        y[k] = 1.0
        tiny_plan.master_step(max_iters=0, kkt_tol=0.0, y=y)
        z = tiny_plan.plan_dose().cpu().numpy()
        col = oracle.aperture_dose(tiny, k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
        np.testing.assert_allclose(z, col, rtol=1e-5, atol=1e-6 * max(col.max(), 1e-30))
    tiny_plan.reset()


# ------------------------------------------------------------------ master problem
def test_master_parity(tiny, tiny_plan):
    cfg = tiny.cfg
    rng = np.random.default_rng(41)
    tiny_plan.reset()
    occ, ll, rr, order = _feasible_plan(cfg, rng, 12)
    R = cfg.n_rows
    for k in order:
        tiny_plan.add_column(k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
    y = np.zeros(cfg.n_angles)
    res = tiny_plan.master_step(max_iters=200000, kkt_tol=dec.GPU_KKT, y=y)
    assert res["status"] == vmat.VMAT_OK, res
    M = np.array([oracle.aperture_dose(tiny, k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
                  for k in order])
    ref = oracle.master(M, np.array(order), tiny.theta_deg, tiny.struct_id, tiny.T, tiny.alpha,
                        tiny.beta, cfg.gamma, cfg.cyclic, np.zeros(cfg.n_angles),
                        eps=dec.ORACLE_EPS)
    assert ref["status"] == 0
    assert res["cost"] == pytest.approx(ref["cost"], rel=1e-5)
    # converged to KKT 1e-12 against 1e-13: the dose within 1e-5 of its largest
    # value; y only as far as the near-collinear columns of neighbouring beams
    # determine it (the cost is flat along their differences)
    z = tiny_plan.plan_dose().cpu().numpy()
    np.testing.assert_allclose(z, ref["z"], rtol=0, atol=1e-5 * ref["z"].max())
    np.testing.assert_allclose(y, ref["y"], rtol=0, atol=1e-4 * ref["y"].max())
    assert np.all(y >= 0) and np.all(y[occ == 0] == 0)
    tiny_plan.reset()


# ------------------------------------------------------------------ column generation
def test_colgen_tiny_decisions_and_costs(tiny, tiny_plan):
    """The tiny workload as specified (D in FP64 on the oracle's side, FP32
    on the library's): decisions as in tests/decisions.py, the replayed
    oracle plan, and the plan dose of the library's own plan."""
    cfg = tiny.cfg
    R = cfg.n_rows
    ref = dec.oracle_plan(tiny)
    tiny_plan.reset()
    gpu = tiny_plan.colgen_run(kkt_tol=dec.GPU_KKT)
    first_tie = next(t for t in range(cfg.iterations) if dec.near_tie(ref, t))
    assert dec.check_unforced(gpu, ref, R) >= first_tie
    # the plan dose is the dose of the library's own plan (apertures, y) to 1e-5
    z = tiny_plan.plan_dose().cpu().numpy()
    z_own = oracle.dose(tiny, oracle.aperture_fluence(cfg, gpu["lleaf"], gpu["rleaf"], gpu["y"]))
    np.testing.assert_allclose(z, z_own, rtol=1e-5, atol=1e-6 * z_own.max())
    # replay the oracle's plan: its decisions wherever they are not near-ties
    tiny_plan.reset()
    rep = tiny_plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
    compared, ties = dec.check_replay(rep, ref, R)
    assert compared >= cfg.iterations - 3, (compared, ties)
    assert np.all(np.diff(rep["cost"]) <= 1e-6 * rep["cost"][:-1])
    # the same apertures and converged intensities: the oracle's plan dose
    z = tiny_plan.plan_dose().cpu().numpy()
    np.testing.assert_allclose(z, ref["z"], rtol=0, atol=1e-4 * ref["z"].max())
    tiny_plan.reset()


def test_colgen_small_path_neighbours(small):
    """The centred small phantom on a path of beams: mirror-image beams tie,
    so decisions agree up to the first near-tie and the replay compares the
    rest."""
    cfg = inputs.small_config(cyclic=False, max_leaf_step=2)
    prob = inputs.Problem(**{**small.__dict__, "cfg": cfg})
    ref = dec.oracle_plan(prob)
    with vmat.Plan(prob) as plan:
        dec.precise(plan)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gpu, ref, cfg.n_rows)
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, cfg.n_rows))
    dec.check_replay(rep, ref, cfg.n_rows)


@pytest.mark.parametrize("method", ["pg", "newton"])
def test_colgen_odd_beam_count(small, method):
    """An odd number of beams (13) changes the shared-memory carve-up of the
    master kernel; both master methods still match the oracle."""
    cfg = inputs.small_config(n_angles=13)
    prob = inputs.make_problem(cfg)
    ref = dec.oracle_plan(prob)
    with vmat.Plan(prob) as plan:
        plan.set_master_method(method)
        dec.precise(plan)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gpu, ref, cfg.n_rows)
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, cfg.n_rows))
    dec.check_replay(rep, ref, cfg.n_rows)


# ------------------------------------------------------------------ batched (differentiable) forms
def test_batch32_parity(small, small_plan):
    prob = small
    B, V = prob.n_beamlets, prob.n_vox
    X = inputs.fluence_batch(50, B, 32)  # [32, B]
    Z, Fp, cost = small_plan.dose_batch32(_cuda(X.T.copy()))
    Z = Z.cpu().numpy().reshape(V, 32)
    Fp = Fp.cpu().numpy().reshape(V, 32)
    for b in [0, 7, 31]:
        z_or = oracle.dose(prob, X[b].astype(np.float64))
        np.testing.assert_allclose(Z[:, b], z_or, rtol=1e-5, atol=1e-6 * z_or.max())
        c_or = oracle.voxel_cost(z_or, prob.struct_id, prob.T, prob.alpha, prob.beta)
        assert cost[b] == pytest.approx(c_or, rel=1e-5)
    F = inputs.rng.normal(51, V * 32).astype(np.float32).reshape(V, 32)
    G = small_plan.price_batch32(_cuda(F)).cpu().numpy().reshape(B, 32)
    for b in [0, 13, 31]:
        g_or = oracle.price(prob, F[:, b].astype(np.float64))
        sc = oracle.price(prob, np.abs(F[:, b].astype(np.float64)))
        assert np.all(np.abs(G[:, b] - g_or) <= 1e-5 * sc + 1e-30)


# ------------------------------------------------------------------ reduced-precision D
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_reduced_precision_dose_error(tiny, dtype):
    ref = oracle.colgen(tiny, eps=1e-6)
    x = oracle.aperture_fluence(tiny.cfg, ref["lleaf"], ref["rleaf"], ref["y"])
    z_or = oracle.dose(tiny, x)
    with vmat.Plan(tiny, dtype=dtype) as plan:
        z, _, _ = plan.dose(_cuda(x.astype(np.float32)))
    err = np.abs(z.cpu().numpy() - z_or).max() / tiny.T.max()
    assert err <= 5e-3, f"{dtype}: max dose error {err:.2e} of prescription"


# ------------------------------------------------------------------ failure handling
def test_unsorted_rows_rejected(tiny):
    bad = inputs.Problem(**tiny.__dict__)
    vox = tiny.vox_idx.copy()
    i = int(np.argmax(np.diff(tiny.row_ptr)))
    a = tiny.row_ptr[i]
    vox[a], vox[a + 1] = vox[a + 1], vox[a]
    bad.vox_idx = vox
    with pytest.raises(vmat.VmatError) as e:
        vmat.Plan(bad)
    assert e.value.status == vmat.VMAT_EINVAL


def test_bounded_wait_times_out_and_context_survives(tiny, tiny_plan):
    st = vmat.vmat_selftest_grid_wait(tiny_plan.ctx, 1, 0.05)
    assert st == vmat.VMAT_ETIMEOUT
    assert vmat.vmat_selftest_grid_wait(tiny_plan.ctx, 0, 0.5) == vmat.VMAT_OK
    x = inputs.rng.uniform(60, tiny.n_beamlets).astype(np.float32)
    z, _, _ = tiny_plan.dose(_cuda(x))
    np.testing.assert_allclose(z.cpu().numpy(), oracle.dose(tiny, x.astype(np.float64)),
                               rtol=1e-5, atol=1e-6 * float(z.max()))
