"""GPU parity of the linear-algebra path against the oracle (config-1 cube).

* block SpMVs (FP64 assembled/scaled, FP32 scaled) vs the oracle matrix;
* the BF16-with-block-scale A-SpMV vs the same quantization applied to the
  oracle's scaled A, and within the quantization bound of the exact product;
* the symmetric diagonal scaling W (§4.1) vs its definition;
* the matrix-free Schur product (Algorithm 2) with a tight inner solve vs the
  explicit dense S = D - C A^-1 B of the scaled system;
* the nested FGMRES solve vs the oracle's direct solve: relative error <= 1e-9
  at outer tolerance 1e-13, in FP64, with FP32 preconditioner levels and with
  the BF16 A in the FP32 levels;
* the same with GMRES restarts forced at every level;
* A M^-1 (block-Jacobi folded into the operator of the A-solves) in FP64,
  FP32 and BF16 with block scale;
* tight intermediate/inner tolerances give convergence in <= 2 outer
  iterations (exact LDU preconditioner, §4.4);
* status codes: iteration cap, NaN right-hand side.
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


@pytest.fixture(scope="module")
def cube():
    m = inputs.cube_mesh(8)
    mat = inputs.material_nh(1e5, 1e6, 1e3)
    gp = GpuProblem(m, mat, load={"p_max": 2e4, "t_ramp": DT})
    prob = gp.prob
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=17, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    N = gp.N
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    am, af, gam = S.gen_alpha(0.5)
    ga = (am, af, gam, DT)
    rhs_o, _, _, _ = S.newton_rhs(prob, st, af * DT, ga)
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    yield {"gp": gp, "Kd": Kd, "rhs": rhs, "rhs_o": rhs_o, "dev": dev, "N": N}
    gp.close()


def _dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def test_spmv_full_and_blocks(cube):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    x = inputs.random_vector(4 * N, seed=1)
    y = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_FULL, H.HYEL_MAT_ASSEMBLED, _dev(x).data_ptr(), y.data_ptr())
    ref = Kd @ x
    bound = abs(Kd) @ np.abs(x)
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-13 * bound + 1e-300)
    A, B, C, D = S.split_blocks(Kd, N)
    for op, M, nin in ((H.HYEL_OP_A, A, 3 * N), (H.HYEL_OP_B, B, N), (H.HYEL_OP_C, C, 3 * N), (H.HYEL_OP_D, D, N)):
        xi = inputs.random_vector(nin, seed=op)
        yo = torch.zeros(M.shape[0], dtype=torch.float64, device="cuda")
        H.hyel_spmv(gp.ctx, op, H.HYEL_MAT_ASSEMBLED, _dev(xi).data_ptr(), yo.data_ptr())
        assert np.all(np.abs(yo.cpu().numpy() - M @ xi) <= 1e-13 * (abs(M) @ np.abs(xi)) + 1e-300)


def test_scaling_and_fp32_spmv(cube):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    w = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_solve_setup(gp.ctx, w.data_ptr())
    wo = S.diag_scaling(Kd)
    assert np.max(np.abs(w.cpu().numpy() - wo) / wo) <= 1e-13
    Ks = sp.diags(wo) @ Kd @ sp.diags(wo)
    As = S.split_blocks(Ks, N)[0]
    x = inputs.random_vector(3 * N, seed=9)
    y = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_A, H.HYEL_MAT_SCALED32, _dev(x, torch.float32).data_ptr(), y.data_ptr())
    assert np.all(np.abs(y.cpu().numpy() - As @ x) <= 2e-6 * (abs(As) @ np.abs(x)))
    y64 = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_A, H.HYEL_MAT_SCALED64, _dev(x).data_ptr(), y64.data_ptr())
    assert np.all(np.abs(y64.cpu().numpy() - As @ x) <= 1e-13 * (abs(As) @ np.abs(x)))


def _bf16_rn(f):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF
    return (r << 16).astype(np.uint32).view(np.float32)


def test_bf16_rounding_helper():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1) wins
    assert _bf16_rn(np.float32(1 + 2.0 ** -8)) == 1.0
    assert _bf16_rn(np.float32(1 + 3 * 2.0 ** -8)) == np.float32(1 + 2.0 ** -6)
    assert _bf16_rn(np.float32(-(1 + 2.0 ** -8 + 2.0 ** -20))) == np.float32(-(1 + 2.0 ** -7))


def test_bf16s_spmv(cube):
    """y = A x with each scaled 3x3 block read as s * e, s = float32(max|a|),
    e = bf16_rn(float32(a) / s): equal, up to FP32 accumulation, to the same
    quantization applied to the oracle's scaled A; within 2^-9 |A||x| (plus
    FP32 accumulation) of the exact product; and visibly quantized."""
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    H.hyel_solve_setup(gp.ctx)
    wo = S.diag_scaling(Kd)
    As = S.split_blocks(sp.diags(wo) @ Kd @ sp.diags(wo), N)[0]
    bsr = sp.bsr_matrix(As, blocksize=(3, 3))
    blk = bsr.data
    s = np.abs(blk).max(axis=(1, 2)).astype(np.float32)
    safe = np.where(s > 0, s, np.float32(1))
    e = _bf16_rn(blk.astype(np.float32) / safe[:, None, None])
    Q = sp.bsr_matrix((e.astype(np.float64) * s[:, None, None].astype(np.float64), bsr.indices, bsr.indptr),
                      shape=As.shape)
    x32 = inputs.random_vector(3 * N, seed=19).astype(np.float32)
    x = x32.astype(np.float64)
    y = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_A, H.HYEL_MAT_SCALED_BF16S, _dev(x32, torch.float32).data_ptr(), y.data_ptr())
    yg = y.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(yg - Q @ x) <= 2e-6 * (abs(Q) @ np.abs(x)))
    bound = abs(As) @ np.abs(x)
    dev_exact = np.abs(yg - As @ x)
    assert np.all(dev_exact <= (2.0 ** -9 + 4e-6) * bound)
    assert np.max(dev_exact / bound) > 2.0 ** -14


def _block_jacobi_fold(As, N):
    """A M^-1 with M the 3x3 block diagonal of A (oracle's scaled A)."""
    Ad = As.toarray() if hasattr(As, "toarray") else As
    Minv = np.zeros_like(Ad)
    for i in range(N):
        sl = slice(3 * i, 3 * i + 3)
        Minv[sl, sl] = np.linalg.inv(Ad[sl, sl])
    return sp.csr_matrix(Ad @ Minv)


def test_folded_block_jacobi_operator(cube):
    """A M^-1 (the operator the A-solves iterate on) in FP64, FP32 and BF16
    with block scale, against the oracle's scaled A times its block-diagonal
    inverse."""
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    H.hyel_solve_setup(gp.ctx)
    wo = S.diag_scaling(Kd)
    As = S.split_blocks(sp.diags(wo) @ Kd @ sp.diags(wo), N)[0]
    AM = _block_jacobi_fold(As, N)
    x = inputs.random_vector(3 * N, seed=23)
    bound = abs(AM) @ np.abs(x)
    y = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_AM, H.HYEL_MAT_SCALED64, _dev(x).data_ptr(), y.data_ptr())
    assert np.all(np.abs(y.cpu().numpy() - AM @ x) <= 1e-12 * bound)
    x32 = x.astype(np.float32)
    y32 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_AM, H.HYEL_MAT_SCALED32, _dev(x32, torch.float32).data_ptr(), y32.data_ptr())
    assert np.all(np.abs(y32.cpu().numpy() - AM @ x32.astype(np.float64)) <= 2e-6 * bound)
    y16 = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_AM, H.HYEL_MAT_SCALED_BF16S, _dev(x32, torch.float32).data_ptr(),
                y16.data_ptr())
    d = np.abs(y16.cpu().numpy() - AM @ x32.astype(np.float64))
    assert np.all(d <= (2.0 ** -9 + 4e-6) * bound)
    assert np.max(d / bound) > 2.0 ** -14
    # the diagonal blocks of A M^-1 are the identity
    bsr = sp.bsr_matrix(AM, blocksize=(3, 3))
    for i in range(0, N, 37):
        for q in range(bsr.indptr[i], bsr.indptr[i + 1]):
            if bsr.indices[q] == i:
                assert np.max(np.abs(bsr.data[q] - np.eye(3))) <= 1e-12


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_nested_solve_with_restarts(cube, precision):
    """GMRES(m) restarts at every level (outer FGMRES(2), A- and inner
    GMRES(3), S GMRES(2), sub-tolerances 1e-6 so that every level runs past
    its restart length): the restarted solve still reaches the direct
    solution."""
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    sub = 1e-6 if precision == H.HYEL_PREC_FP64 else 1e-5
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=sub, precision=precision, outer=(2000, 2),
                             a=(3000, 3), s=(2000, 2), inner=(3000, 3))
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())
    # every level ran more iterations per solve than its restart length
    assert st.outer_its > 2
    assert st.a_its > 3 * st.a_solves and st.inner_its > 3 * st.inner_solves and st.s_its > 2 * st.s_solves


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32])
def test_schur_product_algorithm2(cube, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    H.hyel_solve_setup(gp.ctx)
    wo = S.diag_scaling(Kd)
    Ks = sp.diags(wo) @ Kd @ sp.diags(wo)
    Sx = S.explicit_schur(Ks, N)
    x = inputs.random_vector(N, seed=21)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    tight = 1e-14 if precision == H.HYEL_PREC_FP64 else 1e-7
    params = H.solver_params(precision=precision, inner_rtol=tight)
    H.hyel_schur_apply(gp.ctx, params, _dev(x).data_ptr(), y.data_ptr())
    ref = Sx @ x
    err = np.linalg.norm(y.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err <= (1e-9 if precision == H.HYEL_PREC_FP64 else 1e-4), err


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_nested_solve_matches_direct(cube, precision):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    xo = S.direct_solve(Kd, cube["rhs_o"])
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-13, sub_rtol=1e-2, precision=precision)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-9, (err, st.as_dict())
    assert st.rel_residual <= 1e-12
    assert st.outer_its >= 1


def test_exact_ldu_preconditioner_converges_in_two(cube):
    gp, Kd, N = cube["gp"], cube["Kd"], cube["N"]
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-10, sub_rtol=1e-14)
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
    assert st.outer_its <= 2, st.as_dict()


def test_iteration_cap_and_nan(cube):
    gp, N = cube["gp"], cube["N"]
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    params = H.solver_params(outer_rtol=1e-14, sub_rtol=0.5, outer=(1, 1))
    st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr(), raise_on_error=False)
    assert rc == H.HYEL_ENOCONV and st.outer_its == 1
    bad = cube["rhs"].clone()
    bad[5] = float("nan")
    st, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(), bad.data_ptr(), x.data_ptr(), raise_on_error=False)
    assert rc == H.HYEL_ENAN
    # still usable afterwards
    st, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(), cube["rhs"].data_ptr(), x.data_ptr())
    assert rc == H.HYEL_OK


@pytest.mark.parametrize("precision", [H.HYEL_PREC_FP64, H.HYEL_PREC_FP32, H.HYEL_PREC_BF16S])
def test_graph_and_host_driven_loops_agree_bitwise(cube, precision):
    """The CUDA-graph solve (device-driven while loops) and the host-driven
    replay run the same kernels in the same order: identical iterates."""
    gp, N = cube["gp"], cube["N"]
    out = []
    for graph, every in ((1, 1), (0, 3), (1, 1)):
        x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
        params = H.solver_params(outer_rtol=1e-12, precision=precision, graph=graph, check_every=every)
        st, rc = H.hyel_solve_nested(gp.ctx, params, cube["rhs"].data_ptr(), x.data_ptr())
        out.append((x.cpu().numpy(), st.outer_its, st.a_its, st.s_its, st.inner_its))
    for o in out[1:]:
        assert np.array_equal(o[0], out[0][0])
        assert o[1:] == out[0][1:]
