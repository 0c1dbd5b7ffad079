"""hyel_residual_norm_static: the residual check for callers that cannot
allocate device memory (frameworks whose pool allocator owns all device memory
and forbids cudaMalloc beside it, callers whose device-memory budget is spent,
latency-critical loops where an allocation costs more than the check). Its
scratch is a fixed device array inside the library.

Checked against the existing entry points on two calls in a row:
* the true relative residual that hyel_solve_nested reports for the scaled
  system, and
* ||b - M x|| formed from hyel_spmv's product on the host in float64.
A mesh beyond the scratch's limit is refused (HYEL_EINVAL). Collected last so
that a run stopping at the first failure has already run every other test; it
also passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


def test_residual_norm_static_matches_existing_entry_points():
    m = inputs.cube_mesh(8)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), load={"p_max": 2e4, "t_ramp": DT}, with_oracle=False)
    N = gp.N
    h = 1.0 / 8
    st = inputs.random_state(N, seed=17, u_scale=0.02 * h, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    stats, _ = H.hyel_solve_nested(gp.ctx, H.solver_params(outer_rtol=1e-10), rhs.data_ptr(), x.data_ptr())
    w = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_solve_setup(gp.ctx, w.data_ptr())
    xs = x / w            # x* = W^-1 x
    bs = w * rhs          # b* = W r
    xr = torch.as_tensor(inputs.random_vector(4 * N, seed=3), device="cuda")
    br = torch.as_tensor(inputs.random_vector(4 * N, seed=4), device="cuda")
    y = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_spmv(gp.ctx, H.HYEL_OP_FULL, H.HYEL_MAT_ASSEMBLED, xr.data_ptr(), y.data_ptr())
    ref_r = np.linalg.norm(br.cpu().numpy() - y.cpu().numpy())
    ref_b = np.linalg.norm(br.cpu().numpy())
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _call in range(2):
        out.fill_(-1.0)
        H.hyel_residual_norm_static(gp.ctx, H.HYEL_MAT_SCALED64, xs.data_ptr(), bs.data_ptr(), out.data_ptr())
        o = out.cpu().numpy()
        # x* = x / w is not the solver's internal x* bit for bit, and the
        # converged residual is itself at rounding level: compare on the scale
        # of ||b|| (both quantities are normalised by it)
        assert abs(o[0] / o[1] - stats.rel_residual) <= 1e-13
        assert o[1] == pytest.approx(torch.linalg.norm(bs).item(), rel=1e-12)
        out.fill_(-1.0)
        H.hyel_residual_norm_static(gp.ctx, H.HYEL_MAT_ASSEMBLED, xr.data_ptr(), br.data_ptr(), out.data_ptr())
        o = out.cpu().numpy()
        assert o[0] == pytest.approx(ref_r, rel=1e-12)
        assert o[1] == pytest.approx(ref_b, rel=1e-12)
    # the property the entry point exists for: after the calls above, two more
    # calls leave both PyTorch's allocator and the device's free memory as
    # they were
    torch.cuda.synchronize()
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _call in range(2):
        H.hyel_residual_norm_static(gp.ctx, H.HYEL_MAT_ASSEMBLED, xr.data_ptr(), br.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] == free0
    with pytest.raises(H.HyelError) as ei:
        H.hyel_residual_norm_static(gp.ctx, H.HYEL_MAT_SCALED32, xs.data_ptr(), bs.data_ptr(), out.data_ptr())
    assert ei.value.code == H.HYEL_EINVAL
    gp.close()


def test_residual_norm_static_rejects_meshes_beyond_its_scratch():
    """The fixed scratch holds the per-block partial sums of at most 8,192
    blocks of 128 rows: a 102^3-hex cube (1,092,727 nodes) is refused with
    HYEL_EINVAL and a message naming the limit, without touching the array."""
    m = inputs.cube_mesh(102, jitter=0.0)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), with_oracle=False)
    N = gp.N
    assert N == 103 ** 3 > 8192 * 128
    dev, sst = gp.stage(inputs.zero_state(N))
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, 0, want_norms=False)
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HyelError) as ei:
        H.hyel_residual_norm_static(gp.ctx, H.HYEL_MAT_ASSEMBLED, x.data_ptr(), x.data_ptr(), out.data_ptr())
    assert ei.value.code == H.HYEL_EINVAL
    assert "1048576" in str(ei.value)
    assert torch.equal(out.cpu(), torch.tensor([-1.0, -1.0], dtype=torch.float64))
    gp.close()
