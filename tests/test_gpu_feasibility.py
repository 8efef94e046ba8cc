"""Dose-rate feasibility of the final plan (Sec. 3) through the C ABI against
the oracle's loop on the same apertures: the same number of gamma rounds,
the same final gamma, cost within 1e-5, dose within 1e-5 of its largest
value and intensities within 1e-4 of the largest (both sides solved tightly:
the library's extended-precision master at KKT 1e-12, the oracle at 1e-13);
a feasible plan is only checked; the context keeps its own gamma."""
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
    prob = inputs.make_problem(inputs.tiny_config())
    return prob, dec.oracle_plan(prob)


def _replay(plan, prob, ref):
    R = prob.cfg.n_rows
    fl = np.array([ref["lleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    fr = np.array([ref["rleaf"][k * R:(k + 1) * R] for k in ref["k"]])
    plan.reset()
    return plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=(ref["k"], fl, fr))


def _rho_plan(prob, ref):
    """Starting KKT residual of the plan's first master problem (one column, y = 0)."""
    cfg = prob.cfg
    R = cfg.n_rows
    k0 = int(ref["k"][0])
    col = oracle.aperture_dose(prob, k0, ref["lleaf"][k0 * R:(k0 + 1) * R], ref["rleaf"][k0 * R:(k0 + 1) * R])
    r = oracle.master(col[None, :], np.array([k0]), prob.theta_deg, prob.struct_id, prob.T, prob.alpha,
                      prob.beta, cfg.gamma, cfg.cyclic, np.zeros(cfg.n_angles), max_iter=0)
    return r["rho0"]


@pytest.mark.parametrize("method", ["pg", "newton"])
def test_feasibility_matches_the_oracle(tiny, method):
    prob, ref = tiny
    cfg = prob.cfg
    max_rate = 0.3 * oracle.rate_violation(prob.theta_deg, ref["y"], 0.0, cfg.cyclic)
    with vmat.Plan(prob) as plan:
        plan.set_master_method(method)
        dec.precise(plan)
        _replay(plan, prob, ref)
        gpu = plan.dose_rate_feasibility(max_rate, gamma_factor=2.0, max_rounds=20, kkt_tol=dec.GPU_KKT)
        # the context keeps its gamma: a zero-iteration master evaluates Eq. 3 with it
        y = gpu["y"].copy()
        c0 = plan.master_step(max_iters=0, kkt_tol=0.0, y=y)["cost"]
    orc = oracle.dose_rate_feasibility(prob, ref["k"], ref["lleaf"], ref["rleaf"], ref["y"], max_rate,
                                       gamma_factor=2.0, max_rounds=20, eps=dec.ORACLE_EPS,
                                       rho_ref=_rho_plan(prob, ref))
    assert gpu["status"] == vmat.VMAT_OK and gpu["violation"] <= 0.0
    assert orc["rounds"] >= 1
    assert gpu["rounds"] == orc["rounds"] and gpu["gamma"] == pytest.approx(orc["gamma"])
    np.testing.assert_allclose(gpu["y"], orc["y"], rtol=0, atol=1e-4 * orc["y"].max())
    assert gpu["cost"] == pytest.approx(orc["cost"], rel=1e-5)
    R = cfg.n_rows
    cols = {k: oracle.aperture_dose(prob, k, ref["lleaf"][k * R:(k + 1) * R], ref["rleaf"][k * R:(k + 1) * R])
            for k in ref["k"]}
    z = sum(y[k] * cols[k] for k in ref["k"])
    z_orc = sum(orc["y"][k] * cols[k] for k in ref["k"])
    np.testing.assert_allclose(z, z_orc, rtol=0, atol=1e-5 * z_orc.max())
    c_eq3 = oracle.voxel_cost(z, prob.struct_id, prob.T, prob.alpha, prob.beta) + \
        cfg.gamma * oracle.G(prob.theta_deg, y, cfg.cyclic)
    assert c0 == pytest.approx(c_eq3, rel=1e-5)


def test_feasible_plan_is_only_checked(tiny):
    prob, ref = tiny
    cfg = prob.cfg
    with vmat.Plan(prob) as plan:
        dec.precise(plan)
        _replay(plan, prob, ref)
        loose = 2.0 * oracle.rate_violation(prob.theta_deg, ref["y"], 0.0, cfg.cyclic) + 1.0
        out = plan.dose_rate_feasibility(loose, max_rounds=20)
        assert out["rounds"] == 0 and out["gamma"] == cfg.gamma and out["violation"] < 0
        tight = plan.dose_rate_feasibility(0.0, max_rounds=0, allow_infeasible=True)
        assert tight["status"] == vmat.VMAT_ENOTCONV and tight["rounds"] == 0 and tight["violation"] > 0
        np.testing.assert_array_equal(tight["y"], out["y"])
    with pytest.raises(vmat.VmatError):
        with vmat.Plan(prob) as plan:
            plan.dose_rate_feasibility(-1.0)
