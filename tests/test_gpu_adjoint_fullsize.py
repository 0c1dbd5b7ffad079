"""Adjoint gradient at full size: the 32^3-hex cube (196,608 tets) with
log-normal per-element mu_e, kappa_e (sigma 0.3, seed 1), objective the mean
top-face u_z after 20 generalized-alpha steps, checkpoints every 5 steps.

* directional derivative along a random direction (seed 2) vs central
  differences with h = 1e-6 relative: <= 1e-6 relative;
* 50 random elements (seed 2; 25 for mu, 25 for kappa) vs central
  differences with h = 1e-5 relative: |g - fd| <= 1e-6 max|g|. One element
  moves J by ~1e-11 relative, so at h = 1e-6 the forward runs' 1e-12
  Newton tolerance already puts the difference quotient at the 1e-6 max|g|
  noise floor; h = 1e-5 keeps the check clear of it;
* the same element-wise check on 10 of those elements with FP64 levels;
* a perturbed forward run between a forward and its backward leaves the
  gradient unchanged (to 1e-12 of its largest entry);
* FP32 preconditioner levels give the FP64 gradient to 1e-6.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as Ad
from paper_1809_06350_gb300 import hyel as H, inputs
from paper_1809_06350_gb300.adjoint import AdjointProblem, HyelObjective

pytestmark = pytest.mark.gpu

DT = 1e-3


def test_config5_adjoint_vs_finite_differences():
    from gpu_support import ensure_built
    ensure_built()
    m = inputs.cube_mesh(32)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    E = m["tets"].shape[0]
    f = inputs.element_fields(E, mat, seed=1, sigma=0.3)
    mu, ka = f["mu_e"], f["kappa_e"]
    w = Ad.top_uz_weights(m)
    load = {"p_max": 2e4, "t_ramp": 20 * DT}
    grads = {}
    for prec in (H.HYEL_PREC_FP64, H.HYEL_PREC_FP32):
        P = AdjointProblem(m, mat, load, DT, 20, w, checkpoint_every=5,
                           solver=H.solver_params(outer_rtol=1e-14, precision=prec), tol_r=1e-12)
        mu_t = torch.tensor(mu, requires_grad=True)
        ka_t = torch.tensor(ka, requires_grad=True)
        J = HyelObjective.apply(mu_t, ka_t, P)
        J.backward()
        grads[prec] = (mu_t.grad.numpy().copy(), ka_t.grad.numpy().copy())
        gm, gk = grads[prec]
        rng = np.random.default_rng(2)
        dmu, dka = rng.standard_normal(E), rng.standard_normal(E)
        els = rng.choice(E, 50, replace=False)

        def J_of(a, b):
            with torch.no_grad():
                return float(HyelObjective.apply(torch.tensor(a), torch.tensor(b), P))

        if prec == H.HYEL_PREC_FP64:
            # a perturbed forward between forward and backward must not change
            # the gradient (the backward restores the moduli of its forward)
            mu_t2 = torch.tensor(mu, requires_grad=True)
            ka_t2 = torch.tensor(ka, requires_grad=True)
            J2 = HyelObjective.apply(mu_t2, ka_t2, P)
            J_of(mu * 1.01, ka * 0.99)
            J2.backward()
            # (the perturbation moves the gradient by ~1e-2 relative; rerunning the
            # same forward and backward reproduces it to rounding)
            for g2, g1 in ((mu_t2.grad.numpy(), gm), (ka_t2.grad.numpy(), gk)):
                assert np.max(np.abs(g2 - g1)) <= 1e-12 * np.abs(g1).max()
            # element-wise central differences on the first 10 of the 50 elements
            h = 1e-5
            for which, sel in ((0, els[:5]), (1, els[25:30])):
                base, g = (mu, gm) if which == 0 else (ka, gk)
                for e in sel:
                    p, q = base.copy(), base.copy()
                    p[e] *= 1 + h
                    q[e] *= 1 - h
                    if which == 0:
                        d = (J_of(p, ka) - J_of(q, ka)) / (2 * h * base[e])
                    else:
                        d = (J_of(mu, p) - J_of(mu, q)) / (2 * h * base[e])
                    assert abs(g[e] - d) <= 1e-6 * np.abs(g).max(), (which, e, g[e], d)
        if prec == H.HYEL_PREC_FP32:
            h = 1e-6
            fd = (J_of(mu * (1 + h * dmu), ka * (1 + h * dka)) - J_of(mu * (1 - h * dmu), ka * (1 - h * dka))) / (2 * h)
            ad = np.sum(gm * mu * dmu) + np.sum(gk * ka * dka)
            assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad)
            h = 1e-5
            for which, sel in ((0, els[:25]), (1, els[25:])):
                base, g = (mu, gm) if which == 0 else (ka, gk)
                for e in sel:
                    p, q = base.copy(), base.copy()
                    p[e] *= 1 + h
                    q[e] *= 1 - h
                    if which == 0:
                        d = (J_of(p, ka) - J_of(q, ka)) / (2 * h * base[e])
                    else:
                        d = (J_of(mu, p) - J_of(mu, q)) / (2 * h * base[e])
                    assert abs(g[e] - d) <= 1e-6 * np.abs(g).max(), (which, e, g[e], d)
        P.close()
    for k in range(2):
        a, b = grads[H.HYEL_PREC_FP64][k], grads[H.HYEL_PREC_FP32][k]
        assert np.max(np.abs(a - b)) <= 1e-6 * np.abs(a).max()
