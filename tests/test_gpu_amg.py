"""Aggregation multigrid as the preconditioner of the A-solves
(HYEL_APREC_AMG): it changes iteration counts, never the solution.

* nested solve with the multigrid A-levels vs the oracle's direct solve
  (1e-9 at outer tolerance 1e-13), FP64 and FP32 levels, cube and tube;
* the transposed nested solve with multigrid A-levels vs the oracle;
* graph and host-driven runs agree bit for bit;
* two Newton steps of the small HGO tube match the oracle;
* on a stiffness-dominated tube (5 x 50 x 25 hexes) the multigrid A-levels
  need at most a third of the block-Jacobi A-iterations for the same Newton
  step (measured on GB300: 2,251 against 17,400).
"""
import numpy as np
import pytest
import torch

from oracle import newton as Nw
from oracle import system as S
from paper_1809_06350_gb300 import hyel as H, inputs

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3
AMG = H.HYEL_APREC_AMG


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _system(mesh, mat, fields=None, load=None, seed=17):
    gp = GpuProblem(mesh, mat, fields, load or {"p_max": 2e4, "t_ramp": DT})
    prob = gp.prob
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=seed, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    rhs = torch.zeros(4 * gp.N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * DT, ga)
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    return gp, Kd, rhs, rhs_o, dev


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32])
@pytest.mark.parametrize("case", ["cube", "tube"])
def test_amg_nested_solve_matches_direct(case, precision):
    if case == "cube":
        gp, Kd, rhs, rhs_o, _ = _system(inputs.cube_mesh(8), inputs.material_nh(1e5, 1e6, 1e3))
    else:
        m = inputs.tube_mesh(3, 24, 6)
        mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.0)
        gp, Kd, rhs, rhs_o, _ = _system(m, mat, load={"p_max": 0.0, "t_ramp": 10 * DT})
    N = gp.N
    xo = S.direct_solve(Kd, rhs_o)
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    p = H.solver_params(outer_rtol=1e-13, precision=precision, a_precond=AMG)
    st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
    assert _rel(x.cpu().numpy(), xo) <= 1e-9, st.as_dict()
    # the transposed system on the same blocks
    r = inputs.random_vector(4 * N, seed=6) * np.concatenate([~gp.prob.dir_mask.ravel(), np.ones(N, bool)])
    xt = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_solve_nested_transpose(gp.ctx, p, _dev(r).data_ptr(), xt.data_ptr())
    assert _rel(xt.cpu().numpy(), S.direct_solve(Kd.T.tocsr(), r)) <= 1e-9
    gp.close()


def test_amg_graph_and_host_driven_loops_agree_bitwise():
    gp, Kd, rhs, rhs_o, _ = _system(inputs.cube_mesh(8), inputs.material_nh(1e5, 1e6, 1e3))
    out = []
    for graph in (1, 0):
        x = torch.zeros(4 * gp.N, dtype=torch.float64, device="cuda")
        p = H.solver_params(outer_rtol=1e-12, a_precond=AMG, graph=graph)
        st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
        out.append((x.cpu().numpy(), st.outer_its, st.a_its, st.inner_its))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:]
    gp.close()


def test_amg_small_tube_newton_steps_match_oracle():
    m = inputs.tube_mesh(3, 24, 6)
    mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.0)
    gp = GpuProblem(m, mat, load={"p_max": 0.0, "t_ramp": 10 * DT})
    prob, N = gp.prob, gp.N
    z = inputs.zero_state(N)
    dev = {k: gp.dev(z[k]) for k in z}
    state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
    sp_ = H.solver_params(outer_rtol=1e-13, a_precond=AMG)
    yn = {k: z[k] for k in ("u", "p", "v")}
    ydn = {k: z[k] for k in ("udot", "pdot", "vdot")}
    for step in range(2):
        tp = H.time_params(dt=DT, t_n=step * DT, tol_r=1e-10, tol_a=1e-12)
        st, rc = H.hyel_newton_step(gp.ctx, tp, sp_, state)
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, step * DT, DT, tol_r=1e-10, tol_a=1e-12)
        assert st.converged and st.iterations == info["iterations"]
        for k in ("u", "p", "v"):
            assert _rel(dev[k].cpu().numpy().reshape(y1[k].shape), y1[k]) <= 1e-9, (step, k)
        yn = {k: y1[k] for k in ("u", "p", "v")}
        ydn = {k: yd1[k] for k in ("udot", "pdot", "vdot")}
    gp.close()


def test_amg_cuts_a_iterations_on_a_stiff_tube():
    m = inputs.tube_mesh(5, 50, 25)
    mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.0)
    gp = GpuProblem(m, mat, load={"p_max": 0.0, "t_ramp": 10 * DT}, with_oracle=False)
    N = gp.N
    its = {}
    for aprec in (H.HYEL_APREC_BJACOBI, AMG):
        z = inputs.zero_state(N)
        dev = {k: gp.dev(z[k]) for k in z}
        state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
        sp_ = H.solver_params(outer_rtol=1e-10, precision=H.HYEL_PREC_FP32, outer=(200, 200), a=(2000, 500),
                              s=(400, 200), inner=(2000, 500), a_precond=aprec)
        st, rc = H.hyel_newton_step(gp.ctx, H.time_params(dt=DT, l_max=8), sp_, state)
        assert st.converged
        its[aprec] = st.a_its
    assert its[AMG] * 3 <= its[H.HYEL_APREC_BJACOBI], its
    gp.close()
