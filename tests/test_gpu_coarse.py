"""Coarse tissue voxels (Sec. 3) through the C ABI: the merged problem (with
its volume-weighted tissue structures) matches the oracle like any problem,
and a plan optimised on it, evaluated at full resolution on the fine
problem, costs within a few percent of a plan optimised at full resolution."""
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


def test_coarse_plan_parity_and_full_resolution_quality():
    cfg = inputs.small_config(nx=21, ny=17, nz=7)
    fine = inputs.make_problem(cfg)
    cp = inputs.coarse_tissue(fine)
    R = cfg.n_rows
    ref = dec.oracle_plan(cp.prob)
    with vmat.Plan(cp.prob) as plan:
        # the merged problem's decisions under the rule of tests/decisions.py
        dec.precise(plan)
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        dec.check_replay(rep, ref, R)
        plan.reset()
        dec.check_unforced(plan.colgen_run(kkt_tol=dec.GPU_KKT), ref, R)
        # the default master's own plan, evaluated at full resolution below
        plan.reset()
        plan.set_master_precision(False)
        gpu = plan.colgen_run(kkt_tol=1e-6)
    with vmat.Plan(fine) as fplan:
        x = oracle.aperture_fluence(cfg, gpu["lleaf"], gpu["rleaf"], gpu["y"])
        z, _, cost = fplan.dose(torch.as_tensor(x.astype(np.float32), device="cuda"))
        z_or = oracle.dose(fine, x)
        np.testing.assert_allclose(z.cpu().numpy(), z_or, rtol=1e-5, atol=1e-6 * z_or.max())
        c_or = oracle.voxel_cost(z_or, fine.struct_id, fine.T, fine.alpha, fine.beta)
        assert cost == pytest.approx(c_or, rel=1e-5)
        full_c = cost + cfg.gamma * oracle.G(fine.theta_deg, gpu["y"], cfg.cyclic)
        fine_plan = fplan.colgen_run(kkt_tol=1e-6)
    assert full_c <= 1.05 * fine_plan["cost"][-1], (full_c, fine_plan["cost"][-1])
