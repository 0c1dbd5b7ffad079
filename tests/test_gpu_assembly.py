"""GPU parity of element assembly (Appendix A) against the FP64 oracle.

Residual, right-hand side of eq. NR_smaller_eqn_1 (with the K_{.,udot} R_k
terms, and the literal -[R_m; R_p] of the multi-corrector stage, which runs
the kernel form without the correction) and the tangent blocks A, B, C, D
with Dirichlet elimination, on random
stage states that exercise every term, for the compressible Gibbs, the
incompressible and the HGO materials, global and per-element parameters, a
body force and a traction. Tangent bar: |a_gpu - a_orc| <= 1e-12 max|block row|
per block type; residuals relative to the largest entry of their kind.
Also: bitwise run-to-run determinism and the inverted-element error.
"""
import numpy as np
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs
from oracle import system as S

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem, oracle_blocks, row_scaled_error  # noqa: E402

CASES = {
    "cube8_gibbs": lambda: (inputs.cube_mesh(8), inputs.material_nh(1e5, 1e6, 1e3, body=(0.1, 0.2, -9.81)), None),
    "cube5_incompressible_fields": lambda: (
        inputs.cube_mesh(5, seed=4), inputs.material_nh(1e5, np.inf, 1e3),
        inputs.element_fields(6 * 125, inputs.material_nh(1e5, np.inf, 1e3), seed=2)),
    "cube6_gibbs_fields": lambda: (
        inputs.cube_mesh(6, seed=1), inputs.material_nh(1e5, 1e6, 1e3),
        inputs.element_fields(6 * 216, inputs.material_nh(1e5, 1e6, 1e3), seed=3)),
    "tube_hgo": lambda: (inputs.tube_mesh(3, 16, 4), inputs.material_hgo(3e4, 2e5, 5.0, 0.1), "fib"),
}


def _case(name):
    m, mat, f = CASES[name]()
    if isinstance(f, str):
        f = inputs.element_fields(m["tets"].shape[0], mat, seed=5, with_fibres=True)
    return m, mat, f


def _state(prob, seed, scale=1.0):
    h = np.cbrt(prob.geo["V"].mean())
    st = inputs.random_state(prob.N, seed=seed, u_scale=0.04 * h * scale, v_scale=0.05, p_scale=2e3,
                             rate_scale=3.0)
    return st


@pytest.mark.parametrize("literal", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_assembly_matches_oracle(name, literal):
    m, mat, fields = _case(name)
    load = {"p_max": 2e4, "t_ramp": 5e-3}
    gp = GpuProblem(m, mat, fields, load)
    prob = gp.prob
    st = _state(prob, 13)
    dt = 1e-3
    am, af, gam = S.gen_alpha(0.5)
    tp = H.time_params(dt=dt, t_n=1e-3, rhs_literal=literal)
    t_alpha = 1e-3 + af * dt
    dev, sst = gp.stage(st)
    N = gp.N
    res = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    norms = H.hyel_assemble(gp.ctx, tp, sst, res.data_ptr(), rhs.data_ptr())
    rp, col, A, B, Cb, D = gp.download()

    ga = (am, af, gam, dt)
    rhs_o, Rm, Rp, Rk = S.newton_rhs(prob, st, t_alpha, ga, exact=(literal == 0))
    K = S.assemble_matrix(prob, st, ga)
    Kd, rhs_o = S.apply_dirichlet(K, rhs_o, S.dirichlet_dofs(prob))
    Ao, Bo, Co, Do = oracle_blocks(Kd, N, rp, col)
    rows = np.repeat(np.arange(N), np.diff(rp))
    errs = {k: row_scaled_error(g, o, rows, N) for k, g, o in
            (("A", A, Ao), ("B", B, Bo), ("C", Cb, Co), ("D", D[:, None], Do[:, None]))}
    for k, e in errs.items():
        assert e <= 1e-12, (name, k, e)

    Rm = np.where(prob.dir_mask, 0.0, Rm)
    r = res.cpu().numpy()
    assert np.max(np.abs(r[:3 * N] - Rm.ravel())) <= 1e-12 * np.max(np.abs(Rm))
    assert np.max(np.abs(r[3 * N:] - Rp)) <= 1e-12 * np.max(np.abs(Rp))
    h = rhs.cpu().numpy()
    assert np.max(np.abs(h[:3 * N] - rhs_o[:3 * N])) <= 1e-12 * np.max(np.abs(rhs_o[:3 * N]))
    assert np.max(np.abs(h[3 * N:] - rhs_o[3 * N:])) <= 1e-12 * np.max(np.abs(rhs_o[3 * N:]))
    free = ~prob.dir_mask
    nrm = np.sqrt(np.sum(Rk[free] ** 2) + np.sum(Rp ** 2) + np.sum(Rm[free] ** 2))
    assert norms[0] == pytest.approx(nrm, rel=1e-12)
    gp.close()


def test_assembly_is_bitwise_reproducible():
    m, mat, fields = _case("cube6_gibbs_fields")
    gp = GpuProblem(m, mat, fields, with_oracle=True)
    st = _state(gp.prob, 3)
    dev, sst = gp.stage(st)
    tp = H.time_params()
    outs = []
    for _ in range(2):
        rhs = torch.zeros(4 * gp.N, dtype=torch.float64, device="cuda")
        H.hyel_assemble(gp.ctx, tp, sst, 0, rhs.data_ptr())
        outs.append((rhs.cpu().numpy().copy(), gp.download()[2].copy()))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    gp.close()


def test_inverted_element_is_reported():
    m = inputs.cube_mesh(3)
    gp = GpuProblem(m, inputs.material_nh(), with_oracle=False)
    st = inputs.zero_state(gp.N)
    st["u"] = -2.0 * m["X"]  # F = -I: J = -1 < 0 everywhere
    dev, sst = gp.stage(st)
    with pytest.raises(H.HyelError) as ei:
        H.hyel_assemble(gp.ctx, H.time_params(), sst)
    assert ei.value.code == H.HYEL_EINVERTED
    # the context stays usable
    st = inputs.zero_state(gp.N)
    dev, sst = gp.stage(st)
    H.hyel_assemble(gp.ctx, H.time_params(), sst)
    gp.close()


def test_invalid_arguments():
    gp = GpuProblem(inputs.cube_mesh(2), inputs.material_nh(), with_oracle=False)
    with pytest.raises(H.HyelError) as ei:
        H.hyel_spmv(gp.ctx, 9, 0, 1, 1)
    assert ei.value.code == H.HYEL_EINVAL
    with pytest.raises(H.HyelError) as ei:  # solve before any assembly
        H.hyel_solve_nested(gp.ctx, H.solver_params(), 1, 1)
    assert ei.value.code == H.HYEL_ESTATE
    bad = inputs.cube_mesh(2)
    bad["tets"] = bad["tets"].copy()
    bad["tets"][0, 0] = 10_000
    inp = H.MeshInputs(bad, inputs.material_nh())
    with pytest.raises(H.HyelError) as ei:
        H.hyel_mesh_upload(gp.ctx, inp.X, inp.tets, inp.bc, inp.mat)
    assert ei.value.code == H.HYEL_EINVAL
    gp.close()
