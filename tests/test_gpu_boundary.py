"""Argument handling at the C-ABI boundary:

* operators that read neighbouring rows of x while writing y reject
  overlapping x and y ranges (not only equal pointers): hyel_spmv for every
  operator, hyel_schur_apply, hyel_schur_hat_cheb, hyel_a_cheb_apply and
  hyel_block_precond_apply, each with y one element past x; adjacent,
  non-overlapping ranges are accepted;
* hyel_assemble's HYEL_RES pass gives the residual and norms of the full
  pass (to rounding) and leaves the stored blocks untouched; a right-hand side needs
  HYEL_TAN; other flag values are rejected;
* a call leaves the host thread's current device where it was.
"""
import numpy as np
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


@pytest.fixture(scope="module")
def cube():
    m = inputs.cube_mesh(4)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), load={"p_max": 2e4, "t_ramp": DT}, with_oracle=False)
    N = gp.N
    st = inputs.random_state(N, seed=11, u_scale=0.01 / 4, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    H.hyel_schur_hat_setup(gp.ctx)
    H.hyel_a_cheb_setup(gp.ctx)
    yield {"gp": gp, "N": N, "sst": sst, "dev": dev, "rhs": rhs}
    gp.close()


def _einval(fn):
    with pytest.raises(H.HyelError) as ei:
        fn()
    assert ei.value.code == H.HYEL_EINVAL, ei.value


# (op, matrix, input length in N, output length in N, element bytes)
OPS = [
    (H.HYEL_OP_FULL, H.HYEL_MAT_SCALED64, 4, 4, 8),
    (H.HYEL_OP_A, H.HYEL_MAT_SCALED64, 3, 3, 8),
    (H.HYEL_OP_AM, H.HYEL_MAT_SCALED64, 3, 3, 8),
    (H.HYEL_OP_B, H.HYEL_MAT_SCALED64, 1, 3, 8),
    (H.HYEL_OP_C, H.HYEL_MAT_SCALED64, 3, 1, 8),
    (H.HYEL_OP_D, H.HYEL_MAT_ASSEMBLED, 1, 1, 8),
    (H.HYEL_OP_A, H.HYEL_MAT_SCALED32, 3, 3, 4),
    (H.HYEL_OP_AM, H.HYEL_MAT_SCALED_BF16S, 3, 3, 4),
    (H.HYEL_OP_SHAT, H.HYEL_MAT_SCALED32, 1, 1, 4),
]


@pytest.mark.parametrize("op,matrix,nx,ny,es", OPS)
def test_spmv_rejects_overlap(cube, op, matrix, nx, ny, es):
    gp, N = cube["gp"], cube["N"]
    dt = torch.float64 if es == 8 else torch.float32
    buf = torch.zeros((nx + ny) * N + 1, dtype=dt, device="cuda")
    base = buf.data_ptr()
    _einval(lambda: H.hyel_spmv(gp.ctx, op, matrix, base, base + es))           # y one element past x
    _einval(lambda: H.hyel_spmv(gp.ctx, op, matrix, base + es, base))           # x one element past y
    H.hyel_spmv(gp.ctx, op, matrix, base, base + nx * N * es)                   # adjacent: accepted
    torch.cuda.synchronize()


def test_other_entry_points_reject_overlap(cube):
    gp, N = cube["gp"], cube["N"]
    p = H.solver_params()
    buf = torch.as_tensor(inputs.random_vector(8 * N + 1, seed=3), device="cuda")
    b = buf.data_ptr()
    _einval(lambda: H.hyel_schur_apply(gp.ctx, p, b, b + 8))
    _einval(lambda: H.hyel_schur_hat_cheb(gp.ctx, 4, 0.0, b, b + 8 * (N - 1)))
    _einval(lambda: H.hyel_a_cheb_apply(gp.ctx, 4, b + 8, b))
    _einval(lambda: H.hyel_block_precond_apply(gp.ctx, p, b, b + 8 * (4 * N - 1)))
    H.hyel_schur_apply(gp.ctx, p, b, b + 8 * N)
    H.hyel_schur_hat_cheb(gp.ctx, 4, 0.0, b, b + 8 * N)
    H.hyel_a_cheb_apply(gp.ctx, 4, b, b + 8 * 3 * N)
    H.hyel_block_precond_apply(gp.ctx, p, b, b + 8 * 4 * N)
    torch.cuda.synchronize()


def test_residual_only_pass(cube):
    gp, N, sst = cube["gp"], cube["N"], cube["sst"]
    tp = H.time_params(dt=DT)
    res_full = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    n_full = H.hyel_assemble(gp.ctx, tp, sst, res_full.data_ptr(), 0)
    blocks0 = [a.copy() for a in gp.download()[2:]]
    # a different state for the residual-only pass: the stored blocks must not move
    st2 = inputs.random_state(N, seed=12, u_scale=0.01 / 4, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev2, sst2 = gp.stage(st2)
    res_only = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    n_only = H.hyel_assemble(gp.ctx, tp, sst2, res_only.data_ptr(), 0, flags=H.HYEL_RES)
    for a, b in zip(blocks0, gp.download()[2:]):
        assert np.array_equal(a, b)
    res_full2 = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    n_full2 = H.hyel_assemble(gp.ctx, tp, sst2, res_full2.data_ptr(), 0, flags=H.HYEL_RES | H.HYEL_TAN)
    # the same formulas in two instantiations of the element kernel: equal up
    # to the compiler's contraction of multiply-adds
    scale = torch.max(torch.abs(res_full2)).item()
    assert torch.max(torch.abs(res_only - res_full2)).item() <= 1e-13 * scale
    assert n_only == pytest.approx(n_full2, rel=1e-13)
    assert not torch.equal(res_full, res_full2) and n_full != n_only
    H.hyel_assemble(gp.ctx, tp, sst2, 0, 0, flags=H.HYEL_TAN)
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    _einval(lambda: H.hyel_assemble(gp.ctx, tp, sst2, 0, rhs.data_ptr(), flags=H.HYEL_RES))
    for bad in (0, 4, 7):
        _einval(lambda: H.hyel_assemble(gp.ctx, tp, sst2, 0, 0, flags=bad))
    # restore the fixture's assembly for the other tests of this module
    H.hyel_assemble(gp.ctx, tp, sst, 0, cube["rhs"].data_ptr())
    H.hyel_schur_hat_setup(gp.ctx)
    H.hyel_a_cheb_setup(gp.ctx)


def test_current_device_is_kept(cube):
    gp = cube["gp"]
    before = torch.cuda.current_device()
    H.hyel_mesh_info(gp.ctx)
    H.hyel_solve_setup(gp.ctx)
    assert torch.cuda.current_device() == before


def test_measurement_probes(cube):
    """The FP64 FMA-chain probe reports its flop count and runs at a
    plausible FP64 rate (0.1 to 3 TFLOP/s: GB300's nominal is 1.25); the
    streaming-read probe checks its arguments."""
    gp = cube["gp"]
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    H.hyel_fp64_fma_probe(gp.ctx, 16, sink.data_ptr())
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    e0.record(stream)
    fl = H.hyel_fp64_fma_probe(gp.ctx, 1 << 12, sink.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(0)
    assert fl == 2.0 * (1 << 12) * 8 * 256 * 8 * props.multi_processor_count
    tflops = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
    assert 0.1 < tflops < 3.0, tflops
    assert sink.item() == 0.0
    buf = torch.zeros(1 << 20, dtype=torch.float32, device="cuda")
    H.hyel_stream_read_probe(gp.ctx, buf.data_ptr(), 4 << 20, sink.data_ptr())
    torch.cuda.synchronize()
    for bad in ((buf.data_ptr(), 15), (buf.data_ptr(), 0), (buf.data_ptr() + 4, 64)):
        _einval(lambda: H.hyel_stream_read_probe(gp.ctx, bad[0], bad[1], sink.data_ptr()))
    _einval(lambda: H.hyel_fp64_fma_probe(gp.ctx, 0, sink.data_ptr()))
