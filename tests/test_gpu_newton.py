"""GPU parity of the generalized-alpha Newton step (§3.3) against the oracle
(direct solves): config-1 cube, one step from rest and a second step from the
first (which exercises the K_{.,udot} R_k right-hand-side terms), FP64 and
FP32 preconditioner levels. Bar: y_{n+1}, ydot_{n+1} within 1e-9 relative,
same number of Newton corrections."""
import numpy as np
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import newton as Nw
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_two_newton_steps_match_oracle(precision):
    m = inputs.cube_mesh(8)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    load = {"p_max": 2e4, "t_ramp": 2 * DT}
    gp = GpuProblem(m, mat, load=load)
    prob = gp.prob
    N = gp.N
    z = inputs.zero_state(N)
    dev = {k: gp.dev(z[k]) for k in z}
    state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
    sp_ = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision)
    yn = {k: z[k] for k in ("u", "p", "v")}
    ydn = {k: z[k] for k in ("udot", "pdot", "vdot")}
    for step in range(2):
        t_n = step * DT
        tp = H.time_params(dt=DT, t_n=t_n, tol_r=1e-10, tol_a=1e-12)
        st, rc = H.hyel_newton_step(gp.ctx, tp, sp_, state)
        y1, yd1, info = Nw.newton_step(prob, yn, ydn, t_n, DT, tol_r=1e-10, tol_a=1e-12)
        assert st.converged and info["converged"]
        assert st.iterations == info["iterations"], (st.as_dict(), info)
        for k in ("u", "p", "v"):
            assert _rel(dev[k].cpu().numpy().reshape(y1[k].shape), y1[k]) <= 1e-9, (step, k)
        for k in ("udot", "pdot", "vdot"):
            assert _rel(dev[k].cpu().numpy().reshape(yd1[k].shape), yd1[k]) <= 1e-9, (step, k)
        yn = {k: y1[k] for k in ("u", "p", "v")}
        ydn = {k: yd1[k] for k in ("udot", "pdot", "vdot")}
    gp.close()


@pytest.mark.parametrize("nu", [0.45, 0.499, 0.5])
def test_poisson_sweep_newton_step_matches_oracle(nu):
    """The Poisson-ratio sweep of the cube workload (kappa from nu; nu = 0.5
    is the incompressible model): one Newton step under the ramped dead load
    matches the oracle's direct-solve Newton step: FP64 and FP32 levels with
    the diag(S^) S-preconditioner, FP64 and BF16S levels with the Chebyshev
    polynomial in the explicit S^."""
    m = inputs.cube_mesh(6)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, nu), 1e3)
    load = {"p_max": 2e4, "t_ramp": 10 * DT}
    gp = GpuProblem(m, mat, load=load)
    prob, N = gp.prob, gp.N
    z = inputs.zero_state(N)
    yz = {k: z[k] for k in ("u", "p", "v")}
    ydz = {k: z[k] for k in ("udot", "pdot", "vdot")}
    y1, yd1, info = Nw.newton_step(prob, yz, ydz, 0.0, DT, tol_r=1e-10, tol_a=1e-12)
    assert info["converged"]
    for precision, sprec in ((H.HYEL_PREC_FP64, H.HYEL_SPREC_JACOBI), (H.HYEL_PREC_FP32, H.HYEL_SPREC_JACOBI),
                             (H.HYEL_PREC_FP64, H.HYEL_SPREC_CHEB), (H.HYEL_PREC_BF16S, H.HYEL_SPREC_CHEB)):
        dev = {k: gp.dev(z[k]) for k in z}
        state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
        sp_ = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, s_precond=sprec)
        st, rc = H.hyel_newton_step(gp.ctx, H.time_params(dt=DT, tol_r=1e-10, tol_a=1e-12), sp_, state)
        assert st.converged and st.iterations == info["iterations"], (nu, precision, sprec, st.as_dict(), info)
        for k in ("u", "p", "v"):
            assert _rel(dev[k].cpu().numpy().reshape(y1[k].shape), y1[k]) <= 1e-9, (nu, precision, sprec, k)
    gp.close()


def test_newton_iteration_cap_reports_noconv():
    m = inputs.cube_mesh(4)
    gp = GpuProblem(m, inputs.material_nh(), load={"p_max": 2e4, "t_ramp": DT}, with_oracle=False)
    z = inputs.zero_state(gp.N)
    dev = {k: gp.dev(z[k]) for k in z}
    state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
    tp = H.time_params(dt=DT, tol_r=1e-30, tol_a=0.0, l_max=1)
    st, rc = H.hyel_newton_step(gp.ctx, tp, H.solver_params(), state, raise_on_error=False)
    assert rc == H.HYEL_ENOCONV and st.iterations == 1 and not st.converged
    gp.close()


def test_degenerate_meshes():
    """A single tetrahedron with no Dirichlet data (one ragged 4-row slice;
    A and S stay regular through the mass terms) takes a Newton step under a
    traction load equal to the oracle's; with no load and a state at rest the
    predictor is already converged (no correction)."""
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    m = {"X": X, "tets": np.array([[0, 1, 2, 3]], dtype=np.int32),
         "traction_tris": np.array([[1, 2, 3]], dtype=np.int32), "traction_dir": np.array([1.0, 1.0, 1.0]),
         "dirichlet": np.zeros((0, 2), dtype=np.int32), "dirichlet_values": np.zeros(0)}
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    for p_max, expect_its in ((2e4, None), (0.0, 0)):
        gp = GpuProblem(m, mat, load={"p_max": p_max, "t_ramp": DT})
        prob, N = gp.prob, gp.N
        z = inputs.zero_state(N)
        dev = {k: gp.dev(z[k]) for k in z}
        state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
        tp = H.time_params(dt=DT, tol_r=1e-10, tol_a=1e-12)
        st, rc = H.hyel_newton_step(gp.ctx, tp, H.solver_params(outer_rtol=1e-13), state)
        y1, yd1, info = Nw.newton_step(prob, {k: z[k] for k in ("u", "p", "v")},
                                       {k: z[k] for k in ("udot", "pdot", "vdot")}, 0.0, DT, tol_r=1e-10, tol_a=1e-12)
        assert st.converged and info["converged"] and st.iterations == info["iterations"]
        if expect_its is not None:
            assert st.iterations == expect_its
        else:
            assert st.iterations >= 1
        for k in ("u", "p", "v"):
            assert _rel(dev[k].cpu().numpy().reshape(y1[k].shape), y1[k]) <= 1e-9, (p_max, k)
        gp.close()
