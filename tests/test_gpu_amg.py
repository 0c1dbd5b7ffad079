"""Smoothed-aggregation multigrid with rigid-body modes as the preconditioner
of the A-solves (HYEL_APREC_AMG): it changes iteration counts, never the
solution.

* nested solve with the multigrid A-levels vs the oracle's direct solve
  (1e-9 at outer tolerance 1e-13), FP64 and FP32 levels, cube and tube;
* the transposed nested solve with multigrid A-levels vs the oracle;
* graph and host-driven runs agree bit for bit;
* two Newton steps of the small HGO tube match the oracle, and so does one
  Newton step of the cube at the paper's large time step dt = 0.1 (nu = 0.3
  and the incompressible 0.5);
* a mesh of at most 96 nodes is a single level solved by its dense
  Gauss-Jordan inverse (applied in FP32): every A-solve then reaches 1e-10
  in at most two iterations (the inverse, then one refinement step);
* the hierarchy: two coarse block-nodes (translation, rotation) per
  aggregate, sizes falling to a dense coarsest level;
* on a stiffness-dominated tube (5 x 50 x 25 hexes) the multigrid A-levels
  need at most a third of the block-Jacobi A-iterations for the same Newton
  step;
* mesh independence on the stiff tube at rest (dt = 1e-3): the A-iterations
  per A-solve stay at most 12 from 7,800 to 56,100 nodes (measured on GB300:
  9.5 and 8.1) and at the full size of 222,200 nodes (6.6), where the
  solution's residual is recomputed through hyel_spmv.
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


def test_amg_single_dense_level_is_exact():
    """cube 3^3 (64 nodes <= 96): level 0 is the coarsest and the V-cycle is
    its dense inverse, applied in FP32, so each A-solve reaches 1e-10 in at
    most two iterations."""
    gp, Kd, rhs, rhs_o, _ = _system(inputs.cube_mesh(3), inputs.material_nh(1e5, 1e6, 1e3))
    N = gp.N
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    p = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-10, a_precond=AMG)
    st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
    assert H.hyel_amg_info(gp.ctx) == [(N, H.hyel_mesh_info(gp.ctx)["nnzb"])]
    assert st.a_solves > 0 and st.a_its <= 2 * st.a_solves, st.as_dict()
    assert _rel(x.cpu().numpy(), S.direct_solve(Kd, rhs_o)) <= 1e-9
    gp.close()


def _tube_at_rest(shape):
    m = inputs.tube_mesh(*shape)
    mat = inputs.material_hgo(3e4, 2e5, 5.0, 0.0)
    gp = GpuProblem(m, mat, load={"p_max": 0.0, "t_ramp": 10 * DT}, with_oracle=False)
    z = inputs.zero_state(gp.N)
    dev, sst = gp.stage(z)
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, 0)
    rhs = torch.as_tensor(inputs.random_vector(4 * gp.N, seed=1), device="cuda")
    return gp, rhs


def test_amg_hierarchy_shape():
    gp, rhs = _tube_at_rest((5, 50, 25))
    assert H.hyel_amg_info(gp.ctx) == []
    x = torch.zeros(4 * gp.N, dtype=torch.float64, device="cuda")
    H.hyel_solve_nested(gp.ctx, H.solver_params(a_precond=AMG), rhs.data_ptr(), x.data_ptr())
    lv = H.hyel_amg_info(gp.ctx)
    assert len(lv) >= 3 and lv[0] == (gp.N, H.hyel_mesh_info(gp.ctx)["nnzb"])
    for (n0, _), (n1, b1) in zip(lv, lv[1:]):
        assert n1 % 2 == 0 and n1 < n0 and n1 <= b1 <= n1 * n1
    assert lv[-1][0] <= 96
    gp.close()


def test_amg_a_iterations_are_mesh_independent_on_the_stiff_tube():
    per = []
    for shape in ((5, 50, 25), (10, 100, 50)):
        gp, rhs = _tube_at_rest(shape)
        x = torch.zeros(4 * gp.N, dtype=torch.float64, device="cuda")
        p = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=H.HYEL_PREC_FP32, a_precond=AMG)
        st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
        assert rc == H.HYEL_OK and st.rel_residual <= 1e-9  # the true residual of FP32 levels
        per.append(st.a_its / st.a_solves)
        gp.close()
    assert max(per) <= 12.0, per


def test_amg_fullsize_stiff_tube_solve():
    """The full-size tube (10 x 200 x 100 hexes, 222,200 nodes, 1.2M tets) at
    dt = 1e-3, tangent at rest: one nested solve with the multigrid A-solves
    and FP32 levels converges with at most 12 A-iterations per A-solve
    (measured on GB300: 6.6, as on meshes 28 times smaller), and the
    residual of its solution, recomputed through hyel_spmv on the assembled
    system, meets the outer tolerance up to the FP32 levels' gap (1e-9)."""
    gp, rhs = _tube_at_rest((10, 200, 100))
    N = gp.N
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    p = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=H.HYEL_PREC_FP32, a_precond=AMG)
    st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
    assert rc == H.HYEL_OK, st.as_dict()
    lv = H.hyel_amg_info(gp.ctx)
    assert lv[0][0] == N == 222200 and len(lv) >= 3 and lv[-1][0] <= 96
    assert st.a_its / st.a_solves <= 12.0, st.as_dict()
    y = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_FULL, H.HYEL_MAT_ASSEMBLED, x.data_ptr(), y.data_ptr())
    rel = (torch.linalg.norm(rhs - y) / torch.linalg.norm(rhs)).item()
    assert rel <= 1e-9, rel
    gp.close()


@pytest.mark.parametrize("nu", [0.3, 0.5])
def test_amg_large_dt_newton_step_matches_oracle(nu):
    """The paper's large time step (dt = 0.1: A dominated by the stiffness)
    on the 6^3 cube (343 nodes, so the hierarchy has coarse levels), nu = 0.3
    and the incompressible nu = 0.5: one Newton step with the multigrid
    A-solves, FP64 and FP32 levels, matches the oracle's direct-solve Newton
    step at 1e-9 relative with the same number of corrections."""
    dt = 0.1
    m = inputs.cube_mesh(6)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, nu), 1e3)
    gp = GpuProblem(m, mat, load={"p_max": 2e4, "t_ramp": 10 * dt})
    prob, N = gp.prob, gp.N
    z = inputs.zero_state(N)
    yz = {k: z[k] for k in ("u", "p", "v")}
    ydz = {k: z[k] for k in ("udot", "pdot", "vdot")}
    y1, yd1, info = Nw.newton_step(prob, yz, ydz, 0.0, dt, tol_r=1e-10, tol_a=1e-12)
    assert info["converged"]
    for precision in (H.HYEL_PREC_FP64, H.HYEL_PREC_FP32):
        dev = {k: gp.dev(z[k]) for k in z}
        state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
        sp_ = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, a_precond=AMG)
        st, rc = H.hyel_newton_step(gp.ctx, H.time_params(dt=dt, tol_r=1e-10, tol_a=1e-12), sp_, state)
        assert st.converged and st.iterations == info["iterations"], (nu, precision, st.as_dict(), info)
        assert len(H.hyel_amg_info(gp.ctx)) >= 2
        for k in ("u", "p", "v"):
            assert _rel(dev[k].cpu().numpy().reshape(y1[k].shape), y1[k]) <= 1e-9, (nu, precision, k)
    gp.close()
