"""The projected-Newton master method (an option beyond the paper's gradient
projection): the same optimum of each master problem as the FP64 oracle, the
same column-generation decisions, in far fewer iterations."""
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


def _feasible(cfg, rng, n_occ):
    N, R, C, s = cfg.n_angles, cfg.n_rows, cfg.n_cols, cfg.max_leaf_step
    occ = np.zeros(N, np.uint8)
    ll = np.zeros(N * R, np.int16)
    rr = np.zeros(N * R, np.int16)
    order = []
    for k in rng.permutation(N)[:n_occ]:
        Llo, Lhi, Rlo, Rhi = oracle.leaf_limits(N, R, C, s, cfg.cyclic, occ, ll, rr, k)
        for row in range(R):
            l = int(rng.integers(Llo[row], min(Lhi[row], Rhi[row]) + 1))
            ll[k * R + row], rr[k * R + row] = l, int(rng.integers(max(l, Rlo[row]), Rhi[row] + 1))
        occ[k] = 1
        order.append(int(k))
    return occ, ll, rr, order


@pytest.mark.parametrize("n_cols", [1, 12, 30])
def test_newton_master_reaches_the_oracle_optimum(tiny, n_cols):
    cfg = tiny.cfg
    R = cfg.n_rows
    occ, ll, rr, order = _feasible(cfg, np.random.default_rng(140 + n_cols), n_cols)
    M = np.array([oracle.aperture_dose(tiny, k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
                  for k in order])
    ref = oracle.master(M, np.array(order), tiny.theta_deg, tiny.struct_id, tiny.T, tiny.alpha,
                        tiny.beta, cfg.gamma, cfg.cyclic, np.zeros(cfg.n_angles),
                        eps=dec.ORACLE_EPS)
    assert ref["status"] == 0
    iters = {}
    for method in ("pg", "newton"):
        with vmat.Plan(tiny) as plan:
            plan.set_master_method(method)
            dec.precise(plan)
            for k in order:
                plan.add_column(k, ll[k * R:(k + 1) * R], rr[k * R:(k + 1) * R])
            y = np.zeros(cfg.n_angles)
            res = plan.master_step(max_iters=200000, kkt_tol=dec.GPU_KKT, y=y)
            assert res["status"] == vmat.VMAT_OK, (method, res)
            assert res["cost"] == pytest.approx(ref["cost"], rel=1e-5)
            z = plan.plan_dose().cpu().numpy()
            np.testing.assert_allclose(z, ref["z"], rtol=0, atol=1e-5 * ref["z"].max())
            assert np.all(y >= 0) and np.all(y[occ == 0] == 0)
            iters[method] = res["iters"]
    if n_cols >= 12:
        assert iters["newton"] * 10 <= iters["pg"], iters


def test_newton_column_generation_tiny(tiny):
    cfg = tiny.cfg
    R = cfg.n_rows
    ref = dec.oracle_plan(tiny)
    with vmat.Plan(tiny) as plan:
        plan.set_master_method("newton")
        dec.precise(plan)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gpu, ref, R)
        # the oracle's plan replayed: decisions where they are not near-ties,
        # every master cost within 1e-5
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        dec.check_replay(rep, ref, R)
        assert np.all(np.diff(rep["cost"]) <= 1e-6 * rep["cost"][0])
        newton_iters = int(rep["iters"].sum())
        plan.set_master_method("pg")
        plan.reset()
        pg = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        np.testing.assert_allclose(pg["cost"], rep["cost"], rtol=1e-5)
        assert newton_iters * 10 <= int(pg["iters"].sum()), (newton_iters, int(pg["iters"].sum()))


def test_newton_prostate_first_iterations():
    prob = inputs.make_problem(inputs.prostate_config())
    cfg = prob.cfg
    R, n = cfg.n_rows, 8
    ref = oracle.colgen(prob, n_iter=n, eps=1e-8)
    fl = np.array([ref["lleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    fr = np.array([ref["rleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    with vmat.Plan(prob, val_f32=True) as plan:
        plan.set_master_method("newton")
        rep = plan.colgen_run(n_iters=n, kkt_tol=1e-6, forced=(ref["k"], fl, fr))
    np.testing.assert_allclose(rep["cost"], ref["cost"], rtol=1e-5)
