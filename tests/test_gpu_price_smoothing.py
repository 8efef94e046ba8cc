"""Smoothing-aware pricing (the exact reduced cost of a new column: summed
beamlet price + gamma dG/dy_k of Eq. 2 at the current y, Sec. 2.2 with
Eq. 3) through the C ABI against the FP64 oracle: bit-exact decisions and
prices on the same FP32 beamlet prices and y (ring and path), whole column
generation with decisions compared up to near-ties and the oracle's plan
replayed, and the batch path equal to each plan alone."""
import dataclasses

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



def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _feasible_plan(cfg, rng, n_occ):
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


@pytest.mark.parametrize("cyclic", [True, False])
def test_pricing_bit_exact_with_smoothing(cyclic):
    cfg = inputs.small_config(cyclic=cyclic, max_leaf_step=1, gamma=20.0)
    prob = inputs.make_problem(cfg)
    N, R = cfg.n_angles, cfg.n_rows
    rng = np.random.default_rng(130 + cyclic)
    flips = 0
    with vmat.Plan(prob) as plan:
        plan.set_price_smoothing(True)
        for trial in range(12):
            plan.reset()
            occ, ll, rr, order = _feasible_plan(cfg, rng, int(rng.integers(1, N - 1)))
            for k in order:
                plan.add_column(k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
            y = np.where(occ == 1, rng.uniform(0.0, 3.0, N), 0.0)
            if trial % 4 == 0:
                y[occ == 1] = np.where(rng.uniform(size=int(occ.sum())) < 0.5, 0.0, y[occ == 1])
            yd = y.copy()
            plan.master_step(max_iters=0, kkt_tol=0.0, y=yd)
            np.testing.assert_array_equal(yd, y)  # no iteration: y as given
            g = rng.normal(size=prob.n_beamlets).astype(np.float32)
            if trial % 3 == 0:  # exact zero prices: exact ties
                g[rng.uniform(size=g.size) < 0.5] = 0.0
            got = plan.pricing_select(_cuda(g))
            off = oracle.smoothing_offset(prob.theta_deg, y, cfg.gamma, cyclic)
            ref = oracle.pricing(cfg, occ, ll, rr, g.astype(np.float64), f32=True, offset=off)
            assert got["k"] == ref["k"]
            np.testing.assert_array_equal(got["l"], ref["l"])
            np.testing.assert_array_equal(got["r"], ref["r"])
            assert got["p"] == ref["p"] and got["p2"] == ref["p2"]
            lit = oracle.pricing(cfg, occ, ll, rr, g.astype(np.float64), f32=True)
            flips += lit["k"] != ref["k"]
    assert flips >= 1  # the smoothing term changed some choices


@pytest.mark.parametrize("cyclic", [True, False])
@pytest.mark.parametrize("method", ["pg", "newton"])
def test_colgen_with_smoothing(cyclic, method):
    cfg = inputs.small_config(cyclic=cyclic, gamma=20.0)
    prob = inputs.make_problem(cfg)
    R = cfg.n_rows
    ref = dec.oracle_plan(prob, price_smoothing=True)
    lit = dec.oracle_plan(prob)
    assert np.any(ref["k"] != lit["k"])  # a case where the option matters
    with vmat.Plan(prob) as plan:
        plan.set_master_method(method)
        dec.precise(plan)
        plan.set_price_smoothing(True)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        first = dec.check_unforced(gpu, ref, R)
        np.testing.assert_allclose(gpu["p"][:first], ref["p"][:first], rtol=dec.PRICE_RTOL)
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        # the replay's own decisions and recorded prices: the exact reduced
        # costs of the oracle's state
        dec.check_replay(rep, ref, R)
        # switching it off gives the literal pricing again
        plan.set_price_smoothing(False)
        plan.reset()
        gl = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gl, lit, R)


def test_tiny_plan_with_smoothing():
    """The tiny workload with gamma = 1 (there the option changes most beams'
    order): full 36-iteration plan against the oracle's.  Its box phantom is
    symmetric, so the first choice is an exact tie between mirror beams that
    FP32 prices may break either way; the replay checks every iteration."""
    cfg = inputs.tiny_config(gamma=1.0)
    prob = inputs.make_problem(cfg)
    R = cfg.n_rows
    ref = dec.oracle_plan(prob, price_smoothing=True)
    with vmat.Plan(prob) as plan:
        dec.precise(plan)
        plan.set_price_smoothing(True)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gpu, ref, R)
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        compared, ties = dec.check_replay(rep, ref, R)
        assert compared >= cfg.iterations // 2, (compared, ties)


def test_batch_with_smoothing_equals_each_plan_alone():
    probs = [inputs.make_problem(inputs.small_config(gamma=20.0)),
             inputs.make_problem(inputs.small_config(gamma=5.0, n_angles=10, cyclic=False))]
    plans = [vmat.Plan(p) for p in probs]
    try:
        plans[0].set_price_smoothing(True)
        with vmat.Batch(plans) as b:
            b.configure(1)
            outs = b.run(kkt_tol=1e-6)[0]
            for p, o in zip(plans, outs):  # alone, with the budget the batch gave it
                p.reset()
                a = p.colgen_run(kkt_tol=1e-6)
                np.testing.assert_array_equal(a["k"], o["k"])
                np.testing.assert_array_equal(a["p"], o["p"])
                np.testing.assert_array_equal(a["cost"], o["cost"])
            # a changed setting re-captures the graph
            plans[0].set_price_smoothing(False)
            lit = b.run(kkt_tol=1e-6)[0][0]
            plans[0].reset()
            a = plans[0].colgen_run(kkt_tol=1e-6)
            np.testing.assert_array_equal(a["k"], lit["k"])
            np.testing.assert_array_equal(a["cost"], lit["cost"])
            assert np.any(lit["k"] != outs[0]["k"])
    finally:
        for p in plans:
            p.close()
