"""GPU parity of the block preconditioners of §4.2–4.4 (Algorithm 1 = LDU, and
the DU, D and SIMPLE variants) against the oracle, on the 8^3-hex cube (729
nodes, nu = 0.3):

* one application z = P^-1 r with tight sub-solver tolerances against the
  oracle's block steps with exact (LAPACK) sub-solves;
* nested FGMRES solves with each variant reach the direct solution (FP64 and
  FP32 levels; SIMPLE also with the Chebyshev preconditioner on its S^-solve);
* with tight sub-solves LDU converges in at most 2 outer iterations, DU in at
  most 3 (its preconditioned operator has a single eigenvalue and a
  nilpotent part of degree 2), and SIMPLE takes the outer iteration count
  that GMRES with the exact SIMPLE matrix takes in the oracle (within 1);
* the graph and the host-driven loop give the same bits; bad values fail.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3
KINDS = {"LDU": H.HYEL_BLOCK_LDU, "DU": H.HYEL_BLOCK_DU, "D": H.HYEL_BLOCK_D, "SIMPLE": H.HYEL_BLOCK_SIMPLE}


@pytest.fixture(scope="module")
def cube():
    m = inputs.cube_mesh(8)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    gp = GpuProblem(m, mat, load={"p_max": 2e4, "t_ramp": DT})
    prob = gp.prob
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=29, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    N = gp.N
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * DT, ga)
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    wo = S.diag_scaling(Kd)
    Ks = (sp.diags(wo) @ Kd @ sp.diags(wo)).tocsr()
    yield {"gp": gp, "Kd": Kd, "Ks": Ks, "w": wo, "rhs": rhs, "rhs_o": rhs_o, "dev": dev, "N": N}
    gp.close()


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _tight(kind, **kw):
    return H.solver_params(outer_rtol=1e-13, sub_rtol=1e-12, inner_rtol=1e-13, block_precond=KINDS[kind],
                           a=(3000, 500), s=(2000, 200), inner=(3000, 500), **kw)


@pytest.mark.parametrize("kind", list(KINDS))
def test_apply_matches_oracle(cube, kind):
    gp, Ks, N = cube["gp"], cube["Ks"], cube["N"]
    r = inputs.random_vector(4 * N, seed=50 + KINDS[kind])
    z = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    st = H.hyel_block_precond_apply(gp.ctx, _tight(kind), _dev(r).data_ptr(), z.data_ptr())
    ref = S.block_precond_apply(Ks, N, kind, r)
    err = np.linalg.norm(z.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, (kind, err, st.as_dict())
    # the sub-solves the variant runs
    n_a = {"LDU": 2, "DU": 1, "D": 1, "SIMPLE": 1}[kind]
    assert st.a_solves == n_a and st.s_solves == 1
    assert (st.inner_solves > 0) == (kind != "SIMPLE")


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32])
def test_nested_solve_matches_direct(cube, kind, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, block_precond=KINDS[kind])
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (kind, precision, err, st.as_dict())
    assert st.rel_residual <= 1e-12


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_BF16S])
def test_simple_with_chebyshev_s_hat_solve(cube, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, block_precond=H.HYEL_BLOCK_SIMPLE,
                             s_precond=H.HYEL_SPREC_CHEB)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())


def _gmres_count(Aop, b, tol, m=400):
    """Iterations right-preconditioned GMRES (operator Aop = K P^-1, zero
    start) needs for ||r|| <= tol ||b||, by the least-squares residual."""
    n = b.size
    beta = np.linalg.norm(b)
    V = np.zeros((m + 1, n))
    Hh = np.zeros((m + 1, m))
    V[0] = b / beta
    for j in range(m):
        w = Aop(V[j])
        for _ in range(2):
            h = V[:j + 1] @ w
            w = w - V[:j + 1].T @ h
            Hh[:j + 1, j] += h
        Hh[j + 1, j] = np.linalg.norm(w)
        e = np.zeros(j + 2)
        e[0] = beta
        y = np.linalg.lstsq(Hh[:j + 2, :j + 1], e, rcond=None)[0]
        if np.linalg.norm(e - Hh[:j + 2, :j + 1] @ y) <= tol * beta or Hh[j + 1, j] == 0.0:
            return j + 1
        V[j + 1] = w / Hh[j + 1, j]
    return m


def test_outer_iterations_with_tight_sub_solves(cube):
    gp, Ks, N, w = cube["gp"], cube["Ks"], cube["N"], cube["w"]
    its = {}
    for kind in ("LDU", "DU", "SIMPLE"):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        p = _tight(kind)
        p.outer.rtol = 1e-10
        st, rc = H.hyel_solve_nested(gp.ctx, p, cube["rhs"].data_ptr(), x.data_ptr())
        its[kind] = st.outer_its
    assert its["LDU"] <= 2 and its["DU"] <= 3, its
    # GMRES with the exact SIMPLE matrix on the oracle's scaled system
    P = S.block_precond_matrix(Ks, N, "SIMPLE")
    Pinv = np.linalg.inv(P)
    b = w * cube["rhs_o"]
    ref = _gmres_count(lambda v: Ks @ (Pinv @ v), b, 1e-10)
    assert abs(its["SIMPLE"] - ref) <= 1, (its, ref)
    assert ref > its["DU"]


@pytest.mark.parametrize("kind", ["DU", "SIMPLE"])
def test_graph_and_host_loop_bitwise(cube, kind):
    gp, N = cube["gp"], cube["N"]
    out = []
    for graph in (1, 0):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, graph=graph, block_precond=KINDS[kind])
        st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
        out.append((x.cpu().numpy(), st.outer_its, st.s_its, st.a_its))
    assert np.array_equal(out[0][0], out[1][0]) and out[0][1:] == out[1][1:]


def test_bad_block_precond(cube):
    gp, N = cube["gp"], cube["N"]
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    for bad in (-1, 4):
        _, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(block_precond=bad), cube["rhs"].data_ptr(), x.data_ptr(),
                                    raise_on_error=False)
        assert rc == H.HYEL_EINVAL
    rc = H.lib().hyel_block_precond_apply(gp.ctx, H.solver_params(block_precond=7), cube["rhs"].data_ptr(),
                                          x.data_ptr(), None)
    assert rc == H.HYEL_EINVAL
    rc = H.lib().hyel_block_precond_apply(gp.ctx, H.solver_params(), x.data_ptr(), x.data_ptr(), None)
    assert rc == H.HYEL_EINVAL
