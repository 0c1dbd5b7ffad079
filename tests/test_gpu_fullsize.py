"""Full-size parity on the benchmark workload (48^3-hex cube: 663,552 tets,
470,596 unknowns), in the launch configuration bench.py times (CUDA-graph
solver, FP64 and FP32 preconditioner levels).

* Tangent: 64 sampled block rows (seeded, boundary nodes included) against
  the oracle's complex-step tangent assembled from the elements touching them;
  bar |a_gpu - a_orc| <= 1e-12 max|same block row|.
* Residual: the whole R_m, R_p vector against the oracle (real arithmetic).
* Newton step: the oracle's residual at the GPU's converged state satisfies
  the stopping test ||R||/||R_(0)|| <= tol_R (a property any correct step has,
  at any size); FP32 preconditioner levels, and FP32 levels with the BF16 A,
  reach the FP64 state to 1e-9; so do FP64 and BF16S levels with the
  Chebyshev S-preconditioner on the explicit S^.
* Explicit S^: 8 sampled columns (boundary nodes included) against the
  oracle's S^ built from the tangent rows of their distance-2 neighbourhoods.
"""
import numpy as np
import scipy.sparse as sp
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import schur_hat as SH
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


@pytest.fixture(scope="module")
def big():
    mesh = inputs.cube_mesh(48)
    mat = inputs.material_nh(1e5, inputs.kappa_from_nu(1e5, 0.3), 1e3)
    gp = GpuProblem(mesh, mat, load={"p_max": 2e4, "t_ramp": 10 * DT})
    yield gp
    gp.close()


def _blocks_sparse(K, N, rows, cols):
    K = K.tocsr()
    r3 = (3 * rows[:, None] + np.arange(3)).astype(np.int64)
    c3 = (3 * cols[:, None] + np.arange(3)).astype(np.int64)
    A = np.asarray(K[np.repeat(r3, 3, axis=1).ravel(), np.tile(c3, (1, 3)).ravel()]).reshape(-1, 3, 3)
    B = np.asarray(K[r3.ravel(), np.repeat(3 * N + cols, 3)]).reshape(-1, 3)
    C = np.asarray(K[np.repeat(3 * N + rows, 3), c3.ravel()]).reshape(-1, 3)
    D = np.asarray(K[3 * N + rows, 3 * N + cols]).ravel()
    return A, B, C, D


def test_fullsize_assembly_sampled_rows_and_residual(big):
    gp = big
    prob, N = gp.prob, gp.N
    h = 1.0 / 48
    st = inputs.random_state(N, seed=5, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    res = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT, t_n=2 * DT), sst, res.data_ptr(), 0)
    rp, col, A, B, Cb, D = gp.download()
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    rng = np.random.default_rng(11)
    nodes = np.unique(np.concatenate([rng.choice(N, 60, replace=False), [0, 48, N - 1, N - 49]]))
    K = S.assemble_rows(prob, st, ga, nodes)
    Kd, _ = S.apply_dirichlet(K, np.zeros(4 * N), S.dirichlet_dofs(prob))
    for i in nodes:
        sl = slice(rp[i], rp[i + 1])
        cols = col[sl]
        Ao, Bo, Co, Do = _blocks_sparse(Kd, N, np.full(len(cols), i), cols)
        for name, g, o in (("A", A[sl], Ao), ("B", B[sl], Bo), ("C", Cb[sl], Co), ("D", D[sl], Do)):
            scale = max(np.abs(o).max(), 1e-300)
            assert np.max(np.abs(g - o)) <= 1e-12 * scale, (i, name)
    Rm, Rp = S.assemble_residual(prob, st, 2 * DT + af * DT)
    Rm = np.where(prob.dir_mask, 0.0, Rm)
    r = res.cpu().numpy()
    assert np.max(np.abs(r[:3 * N] - Rm.ravel())) <= 1e-12 * np.abs(Rm).max()
    assert np.max(np.abs(r[3 * N:] - Rp)) <= 1e-12 * np.abs(Rp).max()


def _oracle_norm(prob, yn, ydn, y1, yd1, t_n):
    am, af, gam = S.gen_alpha(0.5)
    stg = S.stage_values(yn, ydn, y1, yd1, am, af)
    Rm, Rp = S.assemble_residual(prob, stg, t_n + af * DT)
    Rk = S.kinematic_residual(stg)
    free = ~prob.dir_mask
    return np.sqrt(np.sum(Rk[free] ** 2) + np.sum(Rp ** 2) + np.sum(Rm[free] ** 2))


def test_fullsize_newton_step_fp64_and_fp32(big):
    gp = big
    prob, N = gp.prob, gp.N
    z = inputs.zero_state(N)
    yz = {k: z[k] for k in ("u", "p", "v")}
    ydz = {k: z[k] for k in ("udot", "pdot", "vdot")}
    norm0 = _oracle_norm(prob, yz, ydz, yz, ydz, 0.0)  # predictor from rest: y1 = 0, ydot1 = 0
    finals = {}
    runs = ((H.HYEL_PREC_FP64, 0), (H.HYEL_PREC_FP32, 0), (H.HYEL_PREC_BF16S, 0),
            (H.HYEL_PREC_FP64, H.HYEL_SPREC_CHEB), (H.HYEL_PREC_BF16S, H.HYEL_SPREC_CHEB))
    for prec, sprec in runs:
        dev = {k: gp.dev(z[k]) for k in z}
        state = H.state_struct(dev["u"], dev["p"], dev["v"], dev["udot"], dev["pdot"], dev["vdot"])
        sp_ = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=prec, graph=1, s_precond=sprec)
        st, rc = H.hyel_newton_step(gp.ctx, H.time_params(dt=DT, t_n=0.0), sp_, state)
        assert st.converged
        y1 = {k: dev[k].cpu().numpy().reshape(z[k].shape) for k in ("u", "p", "v")}
        yd1 = {k: dev[k].cpu().numpy().reshape(z[k].shape) for k in ("udot", "pdot", "vdot")}
        nrm = _oracle_norm(prob, yz, ydz, y1, yd1, 0.0)
        assert st.res_norm0 == pytest.approx(norm0, rel=1e-12)
        assert nrm / norm0 <= 1e-6
        assert abs(nrm - st.res_norm) <= 1e-12 * norm0
        finals[(prec, sprec)] = np.concatenate([y1[k].ravel() for k in ("u", "p", "v")] +
                                               [yd1[k].ravel() for k in ("udot", "pdot", "vdot")])
    f64 = finals[(H.HYEL_PREC_FP64, 0)]
    for key in runs[1:]:
        assert np.linalg.norm(finals[key] - f64) / np.linalg.norm(f64) <= 1e-9, key


def test_fullsize_schur_hat_sampled_columns(big):
    gp = big
    prob, N = gp.prob, gp.N
    h = 1.0 / 48
    st = inputs.random_state(N, seed=5, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT, t_n=2 * DT), sst, 0, 0)
    (lmin, lmax), info = H.hyel_schur_hat_setup(gp.ctx)
    assert 0 < lmin < lmax and np.isfinite(lmax)
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    tets = prob.tets
    adj = sp.csr_matrix((np.ones(16 * len(tets)), (np.repeat(tets, 4, axis=1).ravel(), np.tile(tets, (1, 4)).ravel())),
                        shape=(N, N))
    adj.data[:] = 1.0
    assert info["nnz"] == (adj @ adj).nnz
    rng = np.random.default_rng(13)
    cols = np.unique(np.concatenate([rng.choice(N, 4, replace=False), [0, 48, N - 1, N // 2]]))
    for j in cols:
        n1 = adj[j].indices
        n2 = np.unique(adj[n1].indices)
        K = S.assemble_rows(prob, st, ga, n2)
        Kd, _ = S.apply_dirichlet(K, np.zeros(4 * N), S.dirichlet_dofs(prob))
        wo = S.diag_scaling(Kd)
        Ks = (sp.diags(wo) @ Kd @ sp.diags(wo)).tocsr()
        with np.errstate(divide="ignore"):
            Sh = SH.schur_hat(Ks, N)
        A, B, C, D = S.split_blocks(Ks, N)
        dA = np.abs(A.diagonal())
        dA[dA == 0] = 1.0
        Sb = (abs(D) + abs(C) @ sp.diags(1.0 / dA) @ abs(B)).tocsr()
        e = torch.zeros(N, dtype=torch.float64, device="cuda")
        e[int(j)] = 1.0
        y = torch.zeros(N, dtype=torch.float64, device="cuda")
        H.hyel_spmv(gp.ctx, H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED64, e.data_ptr(), y.data_ptr())
        yg = y.cpu().numpy()
        ref = Sh[:, [j]].toarray().ravel()[n2]
        bound = Sb[:, [j]].toarray().ravel()[n2]
        assert np.all(np.abs(yg[n2] - ref) <= 1e-12 * bound.max()), j
        outside = np.setdiff1d(np.arange(N), n2)
        assert np.all(yg[outside] == 0.0), j
