"""Many plans at once: every batched plan's decisions and costs against the
FP64 oracle (tests/decisions.py), the graph-launched batch reproducing each
plan's own column generation exactly, the autotuner picking an SM share that
works, and FP16-D plans within 0.5% of the prescription of the FP64 dose."""
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
def problems():
    # five plans of uneven size (grid, beams, MLC rows), small enough for the oracle
    cfgs = [inputs.small_config(nx=20 + 3 * i, ny=18 + 2 * i, nz=6 + (i % 2), n_angles=12 + 6 * i,
                                n_rows=6 + 2 * (i % 3), n_cols=8, seed=10 + i) for i in range(5)]
    return [inputs.make_problem(c) for c in cfgs]


@pytest.fixture(scope="module")
def asym_problems():
    # four off-centre plans of uneven size whose decisions never tie
    cfgs = [inputs.asym_config(nx=20 + 3 * i, ny=18 + 2 * i, nz=6 + (i % 2), n_angles=12 + 5 * i,
                               n_rows=6 + (i % 3), n_cols=8 + (i % 2), cyclic=i != 2, seed=30 + i)
            for i in range(4)]
    return [inputs.make_problem(c) for c in cfgs]


def test_batched_plans_vs_oracle(asym_problems):
    """Each plan of a batch (side by side on disjoint SMs, one graph launch)
    takes the oracle's decisions wherever they are not near-ties, with its
    costs within 1e-5."""
    refs = [dec.oracle_plan(p) for p in asym_problems]
    plans = [dec.precise(vmat.Plan(p)) for p in asym_problems]
    try:
        with vmat.Batch(plans) as batch:
            batch.configure(2)
            outs, _, _ = batch.run(kkt_tol=dec.GPU_KKT)
        for prob, ref, out in zip(asym_problems, refs, outs):
            n = prob.cfg.iterations
            first_tie = next((t for t in range(n) if dec.near_tie(ref, t)), n)
            agree = dec.check_unforced(out, ref, prob.cfg.n_rows)
            assert agree >= first_tie and agree >= n - 2, (prob.cfg.name, agree, first_tie, n)
    finally:
        for p in plans:
            p.close()


def test_batch_matches_each_plan_run_alone(problems):
    plans = [vmat.Plan(p) for p in problems]
    try:
        with vmat.Batch(plans) as batch:
            batch.configure(2)
            outs, plan_ms, total = batch.run(kkt_tol=1e-6)
            assert total > 0 and np.all(plan_ms > 0) and np.all(plan_ms <= total * 1.0001)
            again, _, _ = batch.run(kkt_tol=1e-6)  # graph replay from reset
            for p, (plan, out) in enumerate(zip(plans, outs)):
                N = plan.cfg.n_angles
                assert sorted(out["k"].tolist()) == list(range(N))
                np.testing.assert_array_equal(again[p]["cost"], out["cost"])
                plan.reset()
                solo = plan.colgen_run(kkt_tol=1e-6)
                np.testing.assert_array_equal(solo["k"], out["k"])
                np.testing.assert_array_equal(solo["lleaf"], out["lleaf"])
                np.testing.assert_array_equal(solo["rleaf"], out["rleaf"])
                np.testing.assert_array_equal(solo["cost"], out["cost"])
                np.testing.assert_array_equal(solo["y"], out["y"])
    finally:
        for p in plans:
            p.close()


def test_autotuner_and_fp16_dose_error(problems):
    plans = [vmat.Plan(p, dtype="f16") for p in problems]
    try:
        with vmat.Batch(plans) as batch:
            share, ms = batch.tune(trial_iters=8, kkt_tol=1e-6)
            assert share in (1, 2, 3, 4) and ms[share] > 0
            assert ms[share] == min(v for v in ms.values() if v > 0)
            outs, plan_ms, total = batch.run(kkt_tol=1e-6)
        for prob, out in zip(problems, outs):  # cost never rises (FP32 noise: 1e-6 of the start)
            assert np.all(np.diff(out["cost"]) <= 1e-6 * out["cost"][0])
        for prob, plan, out in list(zip(problems, plans, outs))[:3]:
            z = plan.plan_dose().cpu().numpy()
            x = oracle.aperture_fluence(prob.cfg, out["lleaf"], out["rleaf"], out["y"])
            z64 = oracle.dose(prob, x)
            assert np.abs(z - z64).max() <= 5e-3 * prob.T.max()
    finally:
        for p in plans:
            p.close()


def test_batch_newton_matches_each_plan_alone(problems):
    """The projected-Newton master under the batch's graph launch: each plan's
    decisions, costs and intensities equal its own run with the same budget."""
    plans = [vmat.Plan(p) for p in problems[:3]]
    try:
        for p in plans:
            p.set_master_method("newton")
        with vmat.Batch(plans) as batch:
            batch.configure(2)
            outs, _, _ = batch.run(kkt_tol=1e-6)
            for plan, out in zip(plans, outs):
                N = plan.cfg.n_angles
                assert sorted(out["k"].tolist()) == list(range(N))
                plan.reset()
                solo = plan.colgen_run(kkt_tol=1e-6)
                np.testing.assert_array_equal(solo["k"], out["k"])
                np.testing.assert_array_equal(solo["cost"], out["cost"])
                np.testing.assert_array_equal(solo["y"], out["y"])
                assert np.all(out["iters"] <= 50)  # Newton: a few iterations per master
    finally:
        for p in plans:
            p.close()
