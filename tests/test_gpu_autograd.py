"""The differentiable dose + cost (torch.autograd over the C-ABI) against the
FP64 oracle's gradient and against central finite differences of the
oracle's cost (h = 1e-3, 64 random directions normalised to |d|_inf = 1,
relative error <= 1e-4)."""
import numpy as np
import pytest

import oracle
from paper_1005_4396_b300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1005_4396_b300 import autograd, vmat  # noqa: E402


@pytest.fixture(scope="module")
def small():
    return inputs.make_problem(inputs.small_config())


@pytest.fixture(scope="module")
def small_plan(small):
    p = vmat.Plan(small)
    yield p
    p.close()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_cost(prob, x):
    return oracle.voxel_cost(oracle.dose(prob, x), prob.struct_id, prob.T, prob.alpha, prob.beta)


def _oracle_grad_x(prob, x):
    z = oracle.dose(prob, x)
    return oracle.price(prob, oracle.voxel_dcost(z, prob.struct_id, prob.T, prob.alpha, prob.beta))


def test_fluence_cost_and_gradient_match_oracle(small, small_plan):
    prob = small
    Xh = inputs.fluence_batch(81, prob.n_beamlets, 32).T.copy()  # [B, 32]
    X = torch.tensor(Xh, device="cuda", requires_grad=True)
    w = inputs.rng.uniform(82, 32) + 0.5
    cost = autograd.dose_cost(small_plan, X)
    (cost * torch.tensor(w, device="cuda")).sum().backward()
    g = X.grad.cpu().numpy()
    for b in (0, 9, 31):
        x = Xh[:, b].astype(np.float64)
        assert float(cost[b].detach()) == pytest.approx(_oracle_cost(prob, x), rel=1e-5)
        assert _rel(g[:, b], w[b] * _oracle_grad_x(prob, x)) <= 1e-4


def test_fluence_gradient_finite_differences(small, small_plan):
    prob = small
    Xh = inputs.fluence_batch(83, prob.n_beamlets, 32).T.copy()
    X = torch.tensor(Xh, device="cuda", requires_grad=True)
    autograd.dose_cost(small_plan, X)[0].backward()
    g = X.grad.cpu().numpy()[:, 0].astype(np.float64)
    x = Xh[:, 0].astype(np.float64)
    h = 1e-3
    D = inputs.rng.normal(84, 64 * prob.n_beamlets).reshape(64, prob.n_beamlets)
    D /= np.abs(D).max(axis=1, keepdims=True)
    fd = np.array([(_oracle_cost(prob, x + h * d) - _oracle_cost(prob, x - h * d)) / (2 * h) for d in D])
    an = D @ g
    assert _rel(an, fd) <= 1e-4


def test_intensity_cost_and_gradient_match_oracle(small, small_plan):
    prob = small
    cfg = prob.cfg
    l, r = inputs.random_apertures(85, cfg)
    ld = torch.tensor(l, device="cuda")
    rd = torch.tensor(r, device="cuda")
    Yh = inputs.rng.uniform(86, cfg.n_angles * 32).astype(np.float32).reshape(cfg.n_angles, 32)
    Y = torch.tensor(Yh, device="cuda", requires_grad=True)
    w = inputs.rng.uniform(87, 32) + 0.5
    cost = autograd.aperture_dose_cost(small_plan, Y, ld, rd)
    (cost * torch.tensor(w, device="cuda")).sum().backward()
    gy = Y.grad.cpu().numpy()
    for b in (0, 17, 31):
        y = Yh[:, b].astype(np.float64)
        x = oracle.aperture_fluence(cfg, l, r, y)
        c_or = _oracle_cost(prob, x) + cfg.gamma * oracle.G(prob.theta_deg, y, cfg.cyclic)
        assert float(cost[b]) == pytest.approx(c_or, rel=1e-5)
        g_or = oracle.aperture_adjoint(cfg, l, r, _oracle_grad_x(prob, x)) + \
            cfg.gamma * oracle.dG(prob.theta_deg, y, cfg.cyclic)
        assert _rel(gy[:, b], w[b] * g_or) <= 1e-4


def test_intensity_gradient_finite_differences(small, small_plan):
    prob = small
    cfg = prob.cfg
    l, r = inputs.random_apertures(88, cfg)
    Yh = inputs.rng.uniform(89, cfg.n_angles * 32).astype(np.float32).reshape(cfg.n_angles, 32)
    Y = torch.tensor(Yh, device="cuda", requires_grad=True)
    autograd.aperture_dose_cost(small_plan, Y, torch.tensor(l, device="cuda"),
                                torch.tensor(r, device="cuda"))[3].backward()
    g = Y.grad.cpu().numpy()[:, 3].astype(np.float64)
    y = Yh[:, 3].astype(np.float64)

    def c(v):
        return (_oracle_cost(prob, oracle.aperture_fluence(cfg, l, r, v)) +
                cfg.gamma * oracle.G(prob.theta_deg, v, cfg.cyclic))

    h = 1e-3
    D = inputs.rng.normal(90, 64 * cfg.n_angles).reshape(64, cfg.n_angles)
    D /= np.abs(D).max(axis=1, keepdims=True)
    fd = np.array([(c(y + h * d) - c(y - h * d)) / (2 * h) for d in D])
    assert _rel(D @ g, fd) <= 1e-4


def test_prostate_scale_gradients():
    """The differentiable forward on the prostate-scale phantom (288,000
    beamlets, 4.5e8 non-zeros, 180 beams): gradients of sampled vectors
    against the FP64 oracle."""
    prob = inputs.make_problem(inputs.prostate_config())
    cfg = prob.cfg
    with vmat.Plan(prob, val_f32=True) as plan:
        Xh = inputs.fluence_batch(91, prob.n_beamlets, 32).T.copy()
        X = torch.tensor(Xh, device="cuda", requires_grad=True)
        cost = autograd.dose_cost(plan, X)
        cost.sum().backward()
        x = Xh[:, 5].astype(np.float64)
        assert float(cost[5]) == pytest.approx(_oracle_cost(prob, x), rel=1e-5)
        assert _rel(X.grad.cpu().numpy()[:, 5], _oracle_grad_x(prob, x)) <= 1e-4
        l, r = inputs.random_apertures(92, cfg)
        Yh = inputs.rng.uniform(93, cfg.n_angles * 32).astype(np.float32).reshape(cfg.n_angles, 32)
        Y = torch.tensor(Yh, device="cuda", requires_grad=True)
        cy = autograd.aperture_dose_cost(plan, Y, torch.tensor(l, device="cuda"),
                                         torch.tensor(r, device="cuda"))
        cy.sum().backward()
        y = Yh[:, 2].astype(np.float64)
        xf = oracle.aperture_fluence(cfg, l, r, y)
        g_or = oracle.aperture_adjoint(cfg, l, r, _oracle_grad_x(prob, xf)) + \
            cfg.gamma * oracle.dG(prob.theta_deg, y, cfg.cyclic)
        assert _rel(Y.grad.cpu().numpy()[:, 2], g_or) <= 1e-4
