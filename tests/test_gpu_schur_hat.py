"""GPU parity of the explicit S^ = D - C diag(A)^-1 B and the Chebyshev
S-preconditioner built on it, against the oracle (oracle/schur_hat.py), on an
8^3-hex cube (729 nodes: 22 full 32-row slices and a ragged one), compressible
(nu = 0.3) and incompressible (nu = 0.5):

* S^ x (the FP64 copy, and the solver's FP32 copy summed in FP32) against
  the oracle's sparse S^ of the scaled system, within a rounding bound of
  the entries' magnitudes; the stored pattern is the distance-2 node graph;
* the Ritz-value interval against the oracle's (same SplitMix64 start vector,
  same number of Arnoldi steps);
* the Chebyshev polynomial (degrees 1, 2, 4, 7; estimated and fixed-ratio
  intervals) against the oracle's;
* nested solves with the Chebyshev S-preconditioner reach the direct
  solution (FP64, FP32 and BF16S levels; S GMRES(2) restarts; transposed
  system), the graph and the host-driven loop give the same bits, and at
  nu = 0.5 the S-solves need fewer iterations than with diag(S^);
* argument checks.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import schur_hat as SH
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


def _setup(nu):
    m = inputs.cube_mesh(8)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, nu), 1e3)
    gp = GpuProblem(m, mat, load={"p_max": 2e4, "t_ramp": DT})
    prob = gp.prob
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=23, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
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
    A, B, C, D = S.split_blocks(Ks, N)
    Sh = SH.schur_hat(Ks, N)
    Sbound = (abs(D) + abs(C) @ sp.diags(1.0 / np.abs(A.diagonal())) @ abs(B)).tocsr()
    return {"gp": gp, "m": m, "Kd": Kd, "Ks": Ks, "Sh": Sh, "Sbound": Sbound, "rhs": rhs, "rhs_o": rhs_o,
            "dev": dev, "N": N}


@pytest.fixture(scope="module", params=[0.3, 0.5])
def cube(request):
    c = _setup(request.param)
    c["nu"] = request.param
    yield c
    c["gp"].close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_shat_spmv_and_pattern(cube):
    gp, N, Sh, Sb = cube["gp"], cube["N"], cube["Sh"], cube["Sbound"]
    _, info = H.hyel_schur_hat_setup(gp.ctx)
    # pattern: the distance-2 node graph
    tets = np.asarray(cube["m"]["tets"])
    adj = sp.csr_matrix((np.ones(16 * len(tets)), (np.repeat(tets, 4, axis=1).ravel(), np.tile(tets, (1, 4)).ravel())),
                        shape=(N, N))
    adj.data[:] = 1.0
    d2 = adj @ adj
    assert info["nnz"] == d2.nnz
    assert info["max_row"] == np.diff(d2.indptr).max()
    assert info["slots"] % 32 == 0 and info["slots"] >= info["nnz"]
    x = inputs.random_vector(N, seed=31)
    ref = Sh @ x
    bound = Sb @ np.abs(x)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED64, _dev(x).data_ptr(), y.data_ptr())
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-13 * bound + 1e-300)
    y32 = torch.zeros(N, dtype=torch.float32, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED32, _dev(x, torch.float32).data_ptr(), y32.data_ptr())
    # the FP32 copy is summed in FP32 (a dozen terms per entry), the product
    # accumulated in FP32 (about 60 terms per row)
    x32 = x.astype(np.float32).astype(np.float64)
    assert np.all(np.abs(y32.cpu().numpy() - Sh @ x32) <= 1e-5 * (Sb @ np.abs(x32)))


def test_ritz_bounds_match_oracle(cube):
    gp, Sh = cube["gp"], cube["Sh"]
    (lmin, lmax), _ = H.hyel_schur_hat_setup(gp.ctx)
    # the GPU runs the estimate in FP32 (on the FP32 copy of S^), the oracle
    # in FP64: 12 steps of rounding at 6e-8 move the extreme Ritz values by
    # far less than these bars
    rmin, rmax = SH.ritz_bounds(Sh)
    assert lmax == pytest.approx(rmax, rel=1e-4)
    assert lmin == pytest.approx(rmin, rel=1e-3)
    # the Ritz values interlace the spectrum of the symmetric part of the
    # scaled operator, which is nearly symmetric here: the largest lies
    # below the largest eigenvalue, the smallest above the smallest
    ev = np.linalg.eigvals(np.diag(1.0 / Sh.diagonal()) @ Sh.toarray()).real
    assert lmax / SH.RITZ_SAFETY <= ev.max() * (1 + 1e-6) and lmax >= ev.max() * 0.97
    assert lmin * SH.RITZ_LOW >= ev.min() * (1 - 1e-6)


@pytest.mark.parametrize("degree,ratio,matrix", [(1, 0.0, H.HYEL_MAT_SCALED64), (2, 0.0, H.HYEL_MAT_SCALED64),
                                                 (4, 0.0, H.HYEL_MAT_SCALED64), (7, 0.0, H.HYEL_MAT_SCALED64),
                                                 (4, 20.0, H.HYEL_MAT_SCALED64), (4, 0.0, H.HYEL_MAT_SCALED32),
                                                 (7, 0.0, H.HYEL_MAT_SCALED32)])
def test_chebyshev_matches_oracle(cube, degree, ratio, matrix):
    """S^ read in FP64 with FP64 vectors (bar 1e-12), or as inside the
    S-solve: FP32 values (summed in FP32), directions and S^ d products,
    FP64 residual and result (the oracle rounds S^'s entries to FP32, keeping
    M = diag(S^) in FP64, and computes in FP64; bar 5e-5: a few FP32
    roundings per entry and step, amplified by at most the polynomial's
    norm)."""
    gp, N, Sh = cube["gp"], cube["N"], cube["Sh"]
    bounds, _ = H.hyel_schur_hat_setup(gp.ctx)
    x = inputs.random_vector(N, seed=40 + degree)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    H.hyel_schur_hat_cheb(gp.ctx, degree, ratio, _dev(x).data_ptr(), y.data_ptr(), matrix=matrix)
    lmin, lmax = SH.cheb_interval(bounds, ratio)
    Sv = SH.float32_values(Sh) if matrix == H.HYEL_MAT_SCALED32 else None
    ref = SH.chebyshev_apply(Sh, lmin, lmax, degree, x, Sv=Sv)
    err = np.abs(y.cpu().numpy() - ref)
    bar = 1e-12 if matrix == H.HYEL_MAT_SCALED64 else 5e-5
    assert np.max(err) <= bar * np.max(np.abs(ref)), (degree, np.max(err) / np.max(np.abs(ref)))


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_nested_solve_chebyshev_matches_direct(cube, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision, s_precond=H.HYEL_SPREC_CHEB)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())
    assert st.rel_residual <= 1e-12


def test_chebyshev_with_s_restarts(cube):
    """S GMRES(2) at sub-tolerance 1e-6: the end-of-cycle polynomial update
    and the restart run many times; the solve still reaches the direct one."""
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-6, s=(2000, 2), s_precond=H.HYEL_SPREC_CHEB,
                             s_cheb_degree=3)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())
    assert st.s_its > 2 * st.s_solves


def test_graph_and_host_loop_bitwise(cube):
    gp, N = cube["gp"], cube["N"]
    out = []
    for graph in (1, 0):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, graph=graph, s_precond=H.HYEL_SPREC_CHEB)
        st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
        out.append((x.cpu().numpy(), st.outer_its, st.s_its, st.inner_its))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


def test_transposed_solve_chebyshev(cube):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    b = inputs.random_vector(4 * N, seed=77)
    for d in S.dirichlet_dofs(gp.prob):
        b[d] = 0.0
    xo = S.direct_solve(Kd.T.tocsr(), b)
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, s_precond=H.HYEL_SPREC_CHEB)
    st, rc = H.hyel_solve_nested_transpose(gp.ctx, params, _dev(b).data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())


def test_fewer_s_iterations_when_incompressible(cube):
    if cube["nu"] != 0.5:
        pytest.skip("the comparison is made on the incompressible case")
    gp, N = cube["gp"], cube["N"]
    per = {}
    for sprec in (H.HYEL_SPREC_JACOBI, H.HYEL_SPREC_CHEB):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, s_precond=sprec)
        st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
        per[sprec] = st.s_its / st.s_solves
    assert per[H.HYEL_SPREC_CHEB] < per[H.HYEL_SPREC_JACOBI], per


def test_argument_checks():
    m = inputs.cube_mesh(3)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), with_oracle=False)
    N = gp.N
    st = inputs.zero_state(N)
    dev, sst = gp.stage(st)
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, 0)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    L = H.lib()
    assert L.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED64, x.data_ptr(), y.data_ptr()) in (H.HYEL_ESTATE,)
    assert L.hyel_schur_hat_cheb(gp.ctx, H.HYEL_MAT_SCALED64, 4, 20.0, x.data_ptr(), y.data_ptr()) == H.HYEL_ESTATE
    H.hyel_schur_hat_setup(gp.ctx)
    assert L.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_ASSEMBLED, x.data_ptr(), y.data_ptr()) == H.HYEL_EINVAL
    for deg, ratio in ((0, 20.0), (17, 20.0), (4, 1.0), (4, -2.0), (4, float("nan"))):
        assert L.hyel_schur_hat_cheb(gp.ctx, H.HYEL_MAT_SCALED64, deg, ratio, x.data_ptr(), y.data_ptr()) == H.HYEL_EINVAL
    assert L.hyel_schur_hat_cheb(gp.ctx, H.HYEL_MAT_ASSEMBLED, 4, 0.0, x.data_ptr(), y.data_ptr()) == H.HYEL_EINVAL
    assert L.hyel_schur_hat_cheb(gp.ctx, H.HYEL_MAT_SCALED64, 4, 0.0, x.data_ptr(), x.data_ptr()) == H.HYEL_EINVAL
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    xs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    for kw in ({"s_precond": 2}, {"s_precond": 1, "s_cheb_degree": 0}, {"s_precond": 1, "s_cheb_ratio": 0.5}, {"s_precond": 1, "s_cheb_ratio": -1.0},
               {"s_precond": 1, "a_precond": H.HYEL_APREC_AMG}):
        _, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(**kw), rhs.data_ptr(), xs.data_ptr(), raise_on_error=False)
        assert rc == H.HYEL_EINVAL, kw
    gp.close()


def test_mesh_reupload_rebuilds_pattern_and_interval():
    """A second mesh in the same context gets a new S^ pattern, values and
    interval (the first mesh's are freed with it); the products match the
    oracle on the new mesh, and a solve with both Chebyshev preconditioners
    reaches the direct solution."""
    dt = 1e-3
    gp = GpuProblem(inputs.cube_mesh(4), inputs.material_nh(1e5, 1e6, 1e3), with_oracle=False)
    st0 = inputs.zero_state(gp.N)
    _, sst0 = gp.stage(st0)
    H.hyel_assemble(gp.ctx, H.time_params(dt=dt), sst0, 0, 0)
    H.hyel_schur_hat_setup(gp.ctx)
    H.hyel_a_cheb_setup(gp.ctx)
    # second mesh, different size, same context
    m = inputs.cube_mesh(6)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, 0.45), 1e3)
    load = {"p_max": 2e4, "t_ramp": dt}
    inp = H.MeshInputs(m, mat, None, load)
    H.hyel_mesh_upload(gp.ctx, inp.X, inp.tets, inp.bc, inp.mat)
    N = m["X"].shape[0]
    prob = S.Problem(m, mat, load=load)
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(N, seed=44, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev = {k: torch.as_tensor(np.ascontiguousarray(st[k]).ravel(), dtype=torch.float64, device="cuda")
           for k in ("u", "p", "v", "udot", "pdot", "vdot")}
    sst = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=dt), sst, 0, rhs.data_ptr())
    _, info = H.hyel_schur_hat_setup(gp.ctx)
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, dt)
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * dt, ga)
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    wo = S.diag_scaling(Kd)
    Ks = (sp.diags(wo) @ Kd @ sp.diags(wo)).tocsr()
    Sh = SH.schur_hat(Ks, N)
    x = inputs.random_vector(N, seed=45)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED64, _dev(x).data_ptr(), y.data_ptr())
    A, B, C, D = S.split_blocks(Ks, N)
    Sb = (abs(D) + abs(C) @ sp.diags(1.0 / np.abs(A.diagonal())) @ abs(B)).tocsr()
    assert np.all(np.abs(y.cpu().numpy() - Sh @ x) <= 1e-13 * (Sb @ np.abs(x)) + 1e-300)
    xo = S.direct_solve(Kd, rhs_o)
    xs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, s_precond=H.HYEL_SPREC_CHEB,
                             a_precond=H.HYEL_APREC_CHEB)
    H.hyel_solve_nested(gp.ctx, params, rhs.data_ptr(), xs.data_ptr())
    assert np.linalg.norm(xs.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-9
    gp.close()
