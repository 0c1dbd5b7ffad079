"""GPU parity of the adjoint path (pattern 3) against the oracle.

* transposed operator and transposed nested solve vs the oracle matrix
  (A^T x, direct solve of A^T x = r at 1e-9);
* parameter sensitivities -lam^T dR_e/dtheta_e (mu, kappa; mu, k1, k2 for HGO)
  vs complex-step derivatives of the oracle's element residual;
* dJ/d(mu_e, kappa_e) through three generalized-alpha steps vs the oracle's
  dense discrete adjoint (1e-8) and vs central finite differences of GPU
  forward runs (1e-6), with FP64 and FP32 preconditioner levels.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import adjoint as Ad
from oracle import element as el
from oracle import system as S
from paper_1809_06350_gb300 import hyel as H, inputs
from paper_1809_06350_gb300.adjoint import AdjointProblem, HyelObjective

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def test_transposed_spmv_and_solve():
    m = inputs.cube_mesh(6)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), load={"p_max": 2e4, "t_ramp": DT})
    prob, N = gp.prob, gp.N
    st = inputs.random_state(N, seed=2, u_scale=3e-3, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    am, af, gam = S.gen_alpha(0.5)
    K = S.assemble_matrix(prob, st, (am, af, gam, DT))
    Kd, _ = S.apply_dirichlet(K, np.zeros(4 * N), S.dirichlet_dofs(prob))
    x = inputs.random_vector(4 * N, seed=5)
    y = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_FULL, H.HYEL_MAT_TRANSPOSED, _dev(x).data_ptr(), y.data_ptr())
    KT = Kd.T.tocsr()
    assert np.all(np.abs(y.cpu().numpy() - KT @ x) <= 1e-13 * (abs(KT) @ np.abs(x)) + 1e-300)
    r = inputs.random_vector(4 * N, seed=6) * np.concatenate([~prob.dir_mask.ravel(), np.ones(N, bool)])
    xo = S.direct_solve(KT, r)
    for prec in (H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S):
        xg = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        stt, rc = H.hyel_solve_nested_transpose(gp.ctx, H.solver_params(outer_rtol=1e-13, precision=prec),
                                                _dev(r).data_ptr(), xg.data_ptr())
        assert np.linalg.norm(xg.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-9
    # the forward operator is intact after the transposed solve
    xf = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_solve_nested(gp.ctx, H.solver_params(outer_rtol=1e-13), rhs.data_ptr(), xf.data_ptr())
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * DT, (am, af, gam, DT))
    _, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    xo2 = S.direct_solve(Kd, rhs_o)
    assert np.linalg.norm(xf.cpu().numpy() - xo2) / np.linalg.norm(xo2) <= 1e-9
    gp.close()


@pytest.mark.parametrize("kind", ["gibbs", "hgo"])
def test_param_sensitivity_matches_complex_step(kind):
    if kind == "hgo":
        m = inputs.tube_mesh(2, 12, 3)
        mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.1)
        fields = inputs.element_fields(m["tets"].shape[0], mat, seed=3, with_fibres=True)
    else:
        m = inputs.cube_mesh(4)
        mat = inputs.material_nh(1e5, 1e6, 1e3, body=(0.0, 0.0, -9.81))
        fields = inputs.element_fields(m["tets"].shape[0], mat, seed=3)
    gp = GpuProblem(m, mat, fields)
    prob, N, E = gp.prob, gp.N, gp.info["E"]
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(N, seed=8, u_scale=0.03 * h, v_scale=0.05, p_scale=2e3, rate_scale=3.0)
    lam = inputs.random_vector(7 * N, seed=9)
    lam_free = lam * Ad.free_mask(prob)
    dev, sst = gp.stage(st)
    grad = torch.zeros((E, 4), dtype=torch.float64, device="cuda")
    H.hyel_param_sensitivity(gp.ctx, sst, _dev(lam).data_ptr(), grad.data_ptr())
    g = grad.cpu().numpy()
    es = el.gather(prob.tets, st)
    lm = lam_free[4 * N:].reshape(N, 3)[prob.tets]
    lp = lam_free[3 * N:4 * N][prob.tets]
    hcs = 1e-30
    names = ["mu", "kappa", "k1", "k2"]
    active = [0, 2, 3] if kind == "hgo" else [0, 1]
    for k in active:
        me = dict(prob.me)
        me["mu"] = prob.me["mu"].astype(np.complex128)
        me["kappa"] = prob.me["kappa"].astype(np.complex128)
        if k == 0:
            me["mu"] = me["mu"] + 1j * hcs * prob.me["mu"]
            scale = prob.me["mu"]
        elif k == 1:
            me["kappa"] = me["kappa"] + 1j * hcs * prob.me["kappa"]
            scale = prob.me["kappa"]
        else:
            k1, k2, H1, H2 = prob.me["fib"]
            k1c, k2c = k1.astype(np.complex128), k2.astype(np.complex128)
            if k == 2:
                k1c = k1c + 1j * hcs * k1
                scale = k1
            else:
                k2c = k2c + 1j * hcs * k2
                scale = k2
            me["fib"] = (k1c, k2c, H1, H2)
        tau = el.tau_m(prob.geo, me)
        Rm_e, Rp_e = el.element_residual(prob.geo, me, tau, es)
        dRm = Rm_e.imag / (hcs * scale)[:, None, None]
        dRp = Rp_e.imag / (hcs * scale)[:, None]
        ref = -(np.einsum("eai,eai->e", lm, dRm) + np.einsum("ea,ea->e", lp, dRp))
        assert np.max(np.abs(g[:, k] - ref)) <= 1e-11 * np.max(np.abs(ref)), names[k]
    gp.close()


def _adjoint_case():
    m = inputs.cube_mesh(2, jitter=0.05, seed=0)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    f = inputs.element_fields(48, mat, seed=4)
    return m, mat, f["mu_e"], f["kappa_e"], {"p_max": 2e4, "t_ramp": 3 * DT}


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32])
def test_adjoint_gradient_matches_dense_adjoint_and_fd(precision):
    m, mat, mu, ka, load = _adjoint_case()
    w = Ad.top_uz_weights(m)
    solver = H.solver_params(outer_rtol=1e-13, precision=precision)
    P = AdjointProblem(m, mat, load, DT, 3, w, checkpoint_every=2, solver=solver, tol_r=1e-12)
    mu_t = torch.tensor(mu, requires_grad=True)
    ka_t = torch.tensor(ka, requires_grad=True)
    J = HyelObjective.apply(mu_t, ka_t, P)
    J.backward()
    gm, gk = mu_t.grad.numpy(), ka_t.grad.numpy()
    # oracle dense adjoint
    prob = S.Problem(m, mat, fields={"mu_e": mu, "kappa_e": ka}, load=load)
    states = Ad.forward(prob, 3, DT, tol=1e-12)
    Jo = w @ states[-1][0]
    assert float(J.detach()) == pytest.approx(Jo, rel=1e-9)
    go = Ad.gradient(prob, states, w, DT)
    assert np.max(np.abs(gm - go[:, 0])) <= 1e-8 * np.max(np.abs(go[:, 0]))
    assert np.max(np.abs(gk - go[:, 1])) <= 1e-8 * np.max(np.abs(go[:, 1]))
    # central differences of GPU forward runs
    for e in (3, 29):
        for base, gg, which in ((mu, gm, 0), (ka, gk, 1)):
            hh = 1e-4 * base[e]
            vals = []
            for s in (1, -1):
                b = base.copy()
                b[e] += s * hh
                args = (torch.tensor(b), torch.tensor(ka)) if which == 0 else (torch.tensor(mu), torch.tensor(b))
                with torch.no_grad():
                    vals.append(float(HyelObjective.apply(*args, P)))
            fd = (vals[0] - vals[1]) / (2 * hh)
            assert abs(gg[e] - fd) <= 1e-6 * np.max(np.abs(gg)) + 1e-6 * abs(fd), (e, which, gg[e], fd)
    P.close()
