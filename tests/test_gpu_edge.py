"""Degenerate shapes and inputs through the C ABI against the FP64 oracle:
one beam, two beams, one leaf row, one leaf column, the largest row and
column counts, the largest beam count, no smoothing, no leaf travel between
neighbours, and all-zero fluence and voxel vectors."""
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


CASES = {
    "one_beam": dict(n_angles=1),
    "two_beams": dict(n_angles=2),
    "one_row": dict(n_rows=1),
    "one_col": dict(n_cols=1),
    "no_smoothing": dict(gamma=0.0),
    "frozen_leaves": dict(max_leaf_step=0),
    "path_neighbours": dict(cyclic=False, n_angles=7),
    "max_rows": dict(n_rows=128, n_cols=3, nz=16),
    "max_cols": dict(n_rows=3, n_cols=128, nx=40),
}


def _cfg(**kw):
    base = dict(nx=14, ny=12, nz=5, n_angles=8, n_rows=4, n_cols=6)
    base.update(kw)
    return inputs.small_config(**base)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("method", ["pg", "newton"])
def test_degenerate_plans(case, method):
    prob = inputs.make_problem(_cfg(**CASES[case]))
    cfg = prob.cfg
    R = cfg.n_rows
    ref = dec.oracle_plan(prob)
    with vmat.Plan(prob) as plan:
        plan.set_master_method(method)
        dec.precise(plan)
        gpu = plan.colgen_run(kkt_tol=dec.GPU_KKT)
        assert sorted(gpu["k"].tolist()) == list(range(cfg.n_angles))
        assert np.all(gpu["y"] >= 0)
        dec.check_unforced(gpu, ref, R)
        plan.reset()
        rep = plan.colgen_run(kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, R))
        dec.check_replay(rep, ref, R)


def test_largest_beam_count():
    """360 beams (the ABI's limit): the gradient-projection path matches the
    oracle; the projected-Newton variant's factor does not fit in shared
    memory at this size and is refused with VMAT_EINVAL."""
    prob = inputs.make_problem(_cfg(nx=10, ny=10, nz=3, n_angles=360, n_rows=2, n_cols=3))
    ref = dec.oracle_plan(prob, n_iter=24)
    with vmat.Plan(prob) as plan:
        with pytest.raises(vmat.VmatError) as e:
            plan.set_master_method("newton")
        assert e.value.status == vmat.VMAT_EINVAL
        dec.precise(plan)
        gpu = plan.colgen_run(n_iters=24, kkt_tol=dec.GPU_KKT)
        dec.check_unforced(gpu, ref, prob.cfg.n_rows)
        plan.reset()
        rep = plan.colgen_run(n_iters=24, kkt_tol=dec.GPU_KKT, forced=dec.forced(ref, prob.cfg.n_rows))
        dec.check_replay(rep, ref, prob.cfg.n_rows)


def test_zero_vectors():
    prob = inputs.make_problem(_cfg())
    with vmat.Plan(prob) as plan:
        z, fp, cost = plan.dose(torch.zeros(prob.n_beamlets, device="cuda"))
        assert torch.count_nonzero(z).item() == 0
        z0 = np.zeros(prob.n_vox)
        assert cost == pytest.approx(oracle.voxel_cost(z0, prob.struct_id, prob.T, prob.alpha, prob.beta),
                                     rel=1e-12)
        np.testing.assert_allclose(fp.cpu().numpy(),
                                   oracle.voxel_dcost(z0, prob.struct_id, prob.T, prob.alpha, prob.beta),
                                   rtol=1e-6)
        g = plan.price(torch.zeros(prob.n_vox, device="cuda"))
        assert torch.count_nonzero(g).item() == 0
