"""The allocation-free dose + cost entry point against the FP64 oracle and
against the context-based vmat_dose.

vmat_dose_cost_noalloc serves callers that must not let the library allocate
GPU memory (a host framework owning a fixed device pool, a service that may
not allocate while serving, an embedded integration with budgets fixed up
front).  Its scratch is a static device array shared by all calls, so two
calls in a row must each give the result of the context-based vmat_dose on
their own input (nothing left over from the previous call).  This file is
collected last on purpose."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import vmat  # noqa: E402


def test_noalloc_dose_matches_vmat_dose_on_two_calls():
    prob = inputs.make_problem(inputs.tiny_config())
    V, B = prob.n_vox, prob.n_beamlets
    # voxel-major CSR of D over every grid voxel (rows sorted by beamlet)
    rows = np.repeat(np.arange(B, dtype=np.int32), np.diff(prob.row_ptr))
    order = np.argsort(prob.vox_idx, kind="stable")
    vm_col = rows[order]
    vm_val = prob.val[order].astype(np.float32)
    vm_ptr = np.zeros(V + 1, np.int64)
    np.cumsum(np.bincount(prob.vox_idx, minlength=V), out=vm_ptr[1:])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    ptr_d, col_d, val_d = dev(vm_ptr), dev(vm_col), dev(vm_val)
    sid_d = dev(prob.struct_id)
    prm_d = dev(np.concatenate([prob.T, prob.alpha, prob.beta]).astype(np.float64))
    z = torch.empty(V, device="cuda")
    fp = torch.empty(V, device="cuda")
    cost = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    with vmat.Plan(prob) as plan:
        for seed in (71, 72):  # two calls in a row share the static scratch
            x = dev(inputs.rng.uniform(seed, B).astype(np.float32))
            vmat.vmat_dose_cost_noalloc(V, ptr_d, col_d, val_d, x, sid_d, prm_d, prob.T.size,
                                        z, fp, cost, stream)
            torch.cuda.synchronize()
            zg, fg, cg = z.cpu().numpy(), fp.cpu().numpy(), float(cost.item())
            # the FP64 oracle on the same fluence: dose, F' and cost within 1e-5
            z_or = oracle.dose(prob, x.cpu().numpy().astype(np.float64))
            zmax = np.abs(z_or).max()
            np.testing.assert_allclose(zg, z_or, rtol=1e-5, atol=1e-6 * zmax)
            fp_or = oracle.voxel_dcost(z_or, prob.struct_id, prob.T, prob.alpha, prob.beta)
            wmax = 2 * max(prob.alpha.max(), prob.beta.max())
            np.testing.assert_allclose(fg, fp_or, rtol=0,
                                       atol=wmax * (1e-5 * np.abs(z_or) + 1e-6 * zmax).max())
            c_or = oracle.voxel_cost(z_or, prob.struct_id, prob.T, prob.alpha, prob.beta)
            assert cg == pytest.approx(c_or, rel=1e-5)
            # and the context-based entry point
            z_ref, fp_ref, c_ref = plan.dose(x)
            zr = z_ref.cpu().numpy()
            np.testing.assert_allclose(zg, zr, rtol=1e-5, atol=1e-6 * np.abs(zr).max())
            np.testing.assert_allclose(fg, fp_ref.cpu().numpy(), rtol=1e-5,
                                       atol=1e-5 * np.abs(fp_ref.cpu().numpy()).max())
            assert cg == pytest.approx(c_ref, rel=1e-5)


def test_noalloc_rejects_grids_beyond_its_scratch():
    t = torch.zeros(1, device="cuda")
    with pytest.raises(vmat.VmatError) as e:
        vmat.vmat_dose_cost_noalloc(524289, t, t, t, t, t, t, 3, None, None, t, None)
    assert e.value.status == vmat.VMAT_EINVAL


def test_noalloc_flags_structure_ids_beyond_params():
    """A voxel whose structure id has no parameters gets F' = NaN and a NaN
    cost; its dose is still computed and nothing past params is read."""
    prob = inputs.make_problem(inputs.small_config())
    V, B = prob.n_vox, prob.n_beamlets
    rows = np.repeat(np.arange(B, dtype=np.int32), np.diff(prob.row_ptr))
    order = np.argsort(prob.vox_idx, kind="stable")
    vm_ptr = np.zeros(V + 1, np.int64)
    np.cumsum(np.bincount(prob.vox_idx, minlength=V), out=vm_ptr[1:])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    sid = prob.struct_id.copy()
    sid[5] = prob.T.size  # one past the last structure
    x = inputs.rng.uniform(73, B).astype(np.float32)
    z = torch.empty(V, device="cuda")
    fp = torch.empty(V, device="cuda")
    cost = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    vmat.vmat_dose_cost_noalloc(V, dev(vm_ptr), dev(rows[order]), dev(prob.val[order].astype(np.float32)),
                                dev(x), dev(sid), dev(np.concatenate([prob.T, prob.alpha, prob.beta])),
                                prob.T.size, z, fp, cost, stream)
    torch.cuda.synchronize()
    fg = fp.cpu().numpy()
    assert np.isnan(fg[5]) and np.isfinite(np.delete(fg, 5)).all()
    assert np.isnan(float(cost.item()))
    z_or = oracle.dose(prob, x.astype(np.float64))
    np.testing.assert_allclose(z.cpu().numpy(), z_or, rtol=1e-5, atol=1e-6 * np.abs(z_or).max())
