"""GPU parity of the Chebyshev preconditioner of the A-solves
(HYEL_APREC_CHEB: z = p(M^-1 A) M^-1 v with the 3x3 block-Jacobi M, interval
from Ritz values of M^-1 A in the M-inner product) against the oracle, on the
8^3-hex cube (729 nodes):

* the interval against the oracle's FP64 Arnoldi (the GPU runs it in FP32);
* the polynomial (degrees 1, 4, 8) against the oracle's block Chebyshev
  iteration with A's entries rounded to FP32 (FP32 directions and products
  on the GPU, FP64 residual and result);
* nested solves (FP64, FP32, BF16S levels; with the Chebyshev S-preconditioner)
  and a Newton step reach the oracle's direct results; graph and host-driven
  runs give the same bits;
* on a stiffness-dominated A (dt = 0.1) the A-solves need fewer iterations than
  with block-Jacobi alone; bad degrees fail.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import newton as Nw
from oracle import schur_hat as SH
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

CHEB = H.HYEL_APREC_CHEB


def _setup(dt):
    m = inputs.cube_mesh(8)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    gp = GpuProblem(m, mat, load={"p_max": 2e4, "t_ramp": dt})
    prob = gp.prob
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=37, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    N = gp.N
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=dt), sst, 0, rhs.data_ptr())
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, dt)
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * dt, ga)
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    wo = S.diag_scaling(Kd)
    Ks = (sp.diags(wo) @ Kd @ sp.diags(wo)).tocsr()
    As = S.split_blocks(Ks, N)[0].tocsr()
    return {"gp": gp, "Kd": Kd, "As": As, "rhs": rhs, "rhs_o": rhs_o, "N": N}


@pytest.fixture(scope="module")
def cube():
    c = _setup(1e-3)
    yield c
    c["gp"].close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _f32(M):
    out = M.copy()
    out.data = out.data.astype(np.float32).astype(np.float64)
    return out


def test_interval_matches_oracle(cube):
    gp, As, N = cube["gp"], cube["As"], cube["N"]
    lmin, lmax = H.hyel_a_cheb_setup(gp.ctx)
    rmin, rmax = SH.ritz_bounds_m(As, N)
    assert lmax == pytest.approx(rmax, rel=1e-4) and lmin == pytest.approx(rmin, rel=1e-3), ((lmin, lmax), (rmin, rmax))
    Mb, Mi = SH.block_diag_inverse(As, N)
    Minv = sp.block_diag([sp.coo_matrix(b) for b in Mi]).tocsr()
    ev = np.linalg.eigvals((Minv @ As).toarray()).real
    assert lmax >= 0.97 * ev.max() and lmin * SH.RITZ_LOW >= ev.min() * (1 - 1e-4)


@pytest.mark.parametrize("degree", [1, 4, 8])
def test_polynomial_matches_oracle(cube, degree):
    gp, As, N = cube["gp"], cube["As"], cube["N"]
    bounds = H.hyel_a_cheb_setup(gp.ctx)
    x = inputs.random_vector(3 * N, seed=80 + degree)
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    H.hyel_a_cheb_apply(gp.ctx, degree, _dev(x).data_ptr(), y.data_ptr())
    lmin, lmax = SH.cheb_interval(bounds)
    ref = SH.chebyshev_apply_block(As, N, lmin, lmax, degree, x, Av=_f32(As))
    err = np.max(np.abs(y.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err <= 5e-5, (degree, err)


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_nested_solve_matches_direct(cube, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, a_precond=CHEB,
                             s_precond=H.HYEL_SPREC_CHEB)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (precision, err, st.as_dict())


def test_nested_solve_with_restarts(cube):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-6, a=(3000, 2), inner=(3000, 2), a_precond=CHEB,
                             a_cheb_degree=3)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-9, st.as_dict()
    assert st.a_its > 2 * st.a_solves


def test_graph_and_host_loop_bitwise(cube):
    gp, N = cube["gp"], cube["N"]
    out = []
    for graph in (1, 0):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, graph=graph, a_precond=CHEB,
                                 s_precond=H.HYEL_SPREC_CHEB)
        st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
        out.append((x.cpu().numpy(), st.outer_its, st.a_its, st.inner_its))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:]


def test_newton_step_matches_oracle():
    dt = 1e-3
    m = inputs.cube_mesh(6)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, 0.45), 1e3)
    load = {"p_max": 2e4, "t_ramp": 10 * dt}
    gp = GpuProblem(m, mat, load=load)
    prob, N = gp.prob, gp.N
    z = inputs.zero_state(N)
    y1, yd1, info = Nw.newton_step(prob, {k: z[k] for k in ("u", "p", "v")}, {k: z[k] for k in ("udot", "pdot", "vdot")},
                                   0.0, dt, tol_r=1e-10, tol_a=1e-12)
    dev = {k: gp.dev(z[k]) for k in z}
    state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
    sp_ = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, a_precond=CHEB, s_precond=H.HYEL_SPREC_CHEB)
    st, rc = H.hyel_newton_step(gp.ctx, H.time_params(dt=dt, tol_r=1e-10, tol_a=1e-12), sp_, state)
    assert st.converged and st.iterations == info["iterations"]
    for k in ("u", "p", "v"):
        got = dev[k].cpu().numpy().reshape(y1[k].shape)
        assert np.linalg.norm(got - y1[k]) / max(np.linalg.norm(y1[k]), 1e-300) <= 1e-9, k
    gp.close()


def test_fewer_a_iterations_when_stiffness_dominated():
    c = _setup(0.1)
    gp, Kd, N = c["gp"], c["Kd"], c["N"]
    xo = S.direct_solve(Kd, c["rhs_o"])
    per = {}
    for ap in (H.HYEL_APREC_BJACOBI, CHEB):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-12, sub_rtol=1e-2, a_precond=ap)
        st, rc = H.hyel_solve_nested(gp.ctx, params, c["rhs"].data_ptr(), x.data_ptr())
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8
        per[ap] = (st.a_its / st.a_solves, st.inner_its / st.inner_solves)
    assert per[CHEB][0] < per[H.HYEL_APREC_BJACOBI][0] and per[CHEB][1] < per[H.HYEL_APREC_BJACOBI][1], per
    gp.close()


def test_bad_degree(cube):
    gp, N = cube["gp"], cube["N"]
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    for kw in ({"a_precond": CHEB, "a_cheb_degree": 0}, {"a_precond": CHEB, "a_cheb_degree": 17},
               {"a_precond": CHEB, "inner_solver": H.HYEL_INNER_CG_SYM}):
        _, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(**kw), cube["rhs"].data_ptr(), x.data_ptr(),
                                    raise_on_error=False)
        assert rc == H.HYEL_EINVAL, kw
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    y2 = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    H.hyel_a_cheb_setup(gp.ctx)
    assert H.lib().hyel_a_cheb_apply(gp.ctx, 0, y.data_ptr(), y2.data_ptr()) == H.HYEL_EINVAL
    assert H.lib().hyel_a_cheb_apply(gp.ctx, 4, y.data_ptr(), y.data_ptr()) == H.HYEL_EINVAL
