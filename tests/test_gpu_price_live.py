"""Beamlet prices g = D f (Sec. 2.2) in the live-voxel form against the FP64
oracle and against the beamlet-major row products.

The live-voxel form reads only the voxel-major rows of voxels with f_j != 0
and sums each beamlet's exact products on a fixed-point grid in 64-bit
integers, so on FP32-representable D and f its result is the exact price
rounded once to FP32 (up to ~1e-15 of max|f| x the largest row sum of D)."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import vmat  # noqa: E402


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def asym():
    # D rounded to FP32 on both sides (asym_config stores FP32-representable values)
    return inputs.make_problem(inputs.asym_config())


@pytest.fixture(scope="module")
def tiny():
    return inputs.make_problem(inputs.tiny_config())


def _sparse_f(seed, prob, frac):
    f = inputs.rng.normal(seed, prob.n_vox).astype(np.float32)
    keep = inputs.rng.uniform(seed + 1, prob.n_vox) < frac
    return np.where(keep, f, 0.0).astype(np.float32)


def _rows_sum_max(prob):
    return float(oracle.price(prob, np.ones(prob.n_vox)).max())  # largest row sum of D


@pytest.mark.parametrize("frac", [0.02, 0.3, 1.0])
def test_live_prices_are_the_exact_price_rounded_once(asym, frac):
    prob = asym
    f = _sparse_f(31, prob, frac)
    g_or = oracle.price(prob, f.astype(np.float64))
    bound = np.abs(f).max() * _rows_sum_max(prob)
    with vmat.Plan(prob) as plan:
        plan.set_price_path("live")
        g = plan.price(_cuda(f)).cpu().numpy()
        calls = vmat.vmat_get_info(plan.ctx)["price_calls"]
    assert calls == [1, 1]
    # one FP32 rounding of the exact sum (+ the fixed-point grid and the
    # oracle's own FP64 sum, both far below it)
    tol = 2.0 ** -24 * np.abs(g_or) + 1e-13 * bound
    assert np.all(np.abs(g.astype(np.float64) - g_or) <= tol)


@pytest.mark.parametrize("masked", [False, True])
def test_live_and_row_products_agree_with_the_oracle(tiny, masked):
    """Tiny workload: D in FP64 on the oracle's side, FP32 on the library's;
    both forms within the price tolerance of the parity tests, the live form
    much closer."""
    prob = tiny
    f = _sparse_f(32, prob, 0.03)
    mask = (np.arange(prob.cfg.n_angles) % 3 != 1).astype(np.uint8) if masked else None
    g_or = oracle.price(prob, f.astype(np.float64), mask)
    scale = oracle.price(prob, np.abs(f.astype(np.float64)), mask)
    out = {}
    with vmat.Plan(prob) as plan:
        for path in ("rows", "live", "auto"):
            plan.set_price_path(path)
            out[path] = plan.price(_cuda(f), mask).cpu().numpy()
        calls = vmat.vmat_get_info(plan.ctx)["price_calls"]
    assert calls == [2, 3]  # 3% of the voxels live: auto takes the live form
    for path, g in out.items():
        assert np.all(np.abs(g - g_or) <= 1e-5 * scale + 1e-30), path
    # the live form differs from the exact FP64 price only through D's FP32 rounding
    assert np.all(np.abs(out["live"] - g_or) <= 2.0 ** -24 * np.abs(g_or) + 1.2e-7 * scale + 1e-30)
    assert np.array_equal(out["live"], out["auto"])
    if masked:
        beam = np.arange(prob.n_beamlets) // (prob.cfg.n_rows * prob.cfg.n_cols)
        for g in out.values():
            assert np.all(g[mask[beam] == 0] == 0)  # masked-out beams are not written


def test_live_prices_deterministic_and_accumulators_cleared(asym):
    prob = asym
    f1 = _sparse_f(33, prob, 0.05)
    f2 = _sparse_f(35, prob, 0.05)
    with vmat.Plan(prob) as plan:
        plan.set_price_path("live")
        a = plan.price(_cuda(f1)).cpu().numpy()
        b = plan.price(_cuda(f2)).cpu().numpy()
        c = plan.price(_cuda(f1)).cpu().numpy()
        zero = plan.price(_cuda(np.zeros(prob.n_vox, np.float32))).cpu().numpy()
    assert np.array_equal(a, c)  # bit for bit, after another call in between
    assert not np.array_equal(a, b)
    assert np.all(zero == 0)


def test_auto_takes_the_row_products_on_dense_f(tiny):
    prob = tiny
    f = inputs.rng.normal(36, prob.n_vox).astype(np.float32)
    with vmat.Plan(prob) as plan:
        g = plan.price(_cuda(f)).cpu().numpy()
        plan.set_price_path("rows")
        g_rows = plan.price(_cuda(f)).cpu().numpy()
        calls = vmat.vmat_get_info(plan.ctx)["price_calls"]
    assert calls == [0, 2]
    assert np.array_equal(g, g_rows)


@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_live_prices_reduced_precision_storage(tiny, dtype):
    prob = tiny
    f = _sparse_f(37, prob, 0.03)
    with vmat.Plan(prob, dtype=dtype) as plan:
        plan.set_price_path("rows")
        g_rows = plan.price(_cuda(f)).cpu().numpy()
        plan.set_price_path("live")
        g_live = plan.price(_cuda(f)).cpu().numpy()
    scale = oracle.price(prob, np.abs(f.astype(np.float64)))
    # same stored Dhat and scale on both sides: the forms differ by FP32 sums only
    assert np.all(np.abs(g_live - g_rows) <= 1e-5 * scale + 1e-30)


def test_colgen_prices_in_the_live_form(tiny):
    """The column-generation loop with every pricing in the live-voxel form
    against the same loop with the row products: the same plan cost, and the
    same beams wherever the decisions are not near-ties of FP32 sums.  (On
    the tiny phantom the target and the tissue above its threshold are ~10%
    of the voxels, so the automatic choice takes the row products there.)"""
    prob = tiny
    n = prob.cfg.iterations
    with vmat.Plan(prob) as plan:
        auto = plan.colgen_run(kkt_tol=1e-9)
        c_auto = vmat.vmat_get_info(plan.ctx)["price_calls"]
        plan.reset()
        plan.set_price_path("live")
        live = plan.colgen_run(kkt_tol=1e-9)
        c_live = vmat.vmat_get_info(plan.ctx)["price_calls"]
    assert c_auto[1] == n and c_live[0] - c_auto[0] == n and c_live[1] == 2 * n
    assert live["cost"][-1] == pytest.approx(auto["cost"][-1], rel=1e-5)
    assert sorted(live["k"].tolist()) == list(range(prob.cfg.n_angles))
    assert np.all(np.diff(live["cost"]) <= 1e-6 * live["cost"][:-1])
