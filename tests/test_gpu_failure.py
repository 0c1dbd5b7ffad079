"""Failure detection, with every failure made on the host (no device fault):

* a grid-barrier wait that runs out: hyel_inject_fault makes one block of the
  next persistent launch skip one arrival; with a 50 ms wait limit the other
  blocks give up, every block leaves, and the entry point returns HYEL_ECUDA
  within a bounded time. The context stays usable: the next call, without the
  fault, returns the same result as before the fault, bit for bit. Checked
  for the stand-alone Schur product (one launch of the inner A-solve) and
  for the nested solve in graph and host-driven modes (the fault hits the
  first intermediate A-solve; FGMRES carries on and the solve reports
  HYEL_ECUDA);
* a material whose density and shear modulus vanish (1e-300) gives 3x3
  diagonal blocks of A with no representable determinant: hyel_solve_setup
  and hyel_solve_nested return HYEL_ESINGULAR (a node in no element, the
  other way to a zero block, is refused at upload);
* argument checks of the two failure-detection entry points.
"""
import time

import numpy as np
import pytest
import torch

from paper_1809_06350_gb300 import hyel as H, inputs

pytestmark = pytest.mark.gpu

from gpu_support import GpuProblem  # noqa: E402

DT = 1e-3


@pytest.fixture(scope="module")
def cube():
    m = inputs.cube_mesh(8)
    gp = GpuProblem(m, inputs.material_nh(1e5, 1e6, 1e3), load={"p_max": 2e4, "t_ramp": DT}, with_oracle=False)
    N = gp.N
    st = inputs.random_state(N, seed=17, u_scale=0.02 / 8, v_scale=0.02, p_scale=1e3, rate_scale=2.0)
    dev, sst = gp.stage(st)
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    yield {"gp": gp, "rhs": rhs, "N": N, "dev": dev}
    gp.close()


def _timed(fn):
    t0 = time.perf_counter()
    try:
        fn()
        rc = H.HYEL_OK
    except H.HyelError as e:
        rc = e.code
    return rc, time.perf_counter() - t0


def test_barrier_timeout_in_schur_product(cube):
    gp, N = cube["gp"], cube["N"]
    p = H.solver_params(sub_rtol=1e-6)
    x = torch.as_tensor(inputs.random_vector(N, seed=5), device="cuda")
    y0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    H.hyel_schur_apply(gp.ctx, p, x.data_ptr(), y0.data_ptr())
    torch.cuda.synchronize()
    H.hyel_set_wait_limit(gp.ctx, 0.05)
    H.hyel_inject_fault(gp.ctx, H.HYEL_FAULT_BARRIER_SKIP)
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    rc, secs = _timed(lambda: H.hyel_schur_apply(gp.ctx, p, x.data_ptr(), y.data_ptr()))
    assert rc == H.HYEL_ECUDA
    assert "timed out" in H.hyel_last_error(gp.ctx)
    assert secs < 10.0
    # the fault was taken by one launch: the context works as before
    y.zero_()
    H.hyel_schur_apply(gp.ctx, p, x.data_ptr(), y.data_ptr())
    assert torch.equal(y, y0)
    H.hyel_set_wait_limit(gp.ctx, 1.0)


@pytest.mark.parametrize("graph", [1, 0])
def test_barrier_timeout_in_nested_solve(cube, graph):
    gp, N, rhs = cube["gp"], cube["N"], cube["rhs"]
    p = H.solver_params(outer_rtol=1e-10, graph=graph)
    x0 = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    st0, _ = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x0.data_ptr())
    H.hyel_set_wait_limit(gp.ctx, 0.05)
    H.hyel_inject_fault(gp.ctx, H.HYEL_FAULT_BARRIER_SKIP)
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    st, rc = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr(), raise_on_error=False)
    secs = time.perf_counter() - t0
    assert rc == H.HYEL_ECUDA and st.status == H.HYEL_ECUDA
    assert secs < 20.0
    x.zero_()
    st1, rc1 = H.hyel_solve_nested(gp.ctx, p, rhs.data_ptr(), x.data_ptr())
    assert rc1 == H.HYEL_OK
    assert torch.equal(x, x0) and st1.outer_its == st0.outer_its
    H.hyel_set_wait_limit(gp.ctx, 1.0)


def test_withdrawn_injection_and_arguments(cube):
    gp, N = cube["gp"], cube["N"]
    H.hyel_inject_fault(gp.ctx, H.HYEL_FAULT_BARRIER_SKIP)
    H.hyel_inject_fault(gp.ctx, H.HYEL_FAULT_NONE)
    x = torch.as_tensor(inputs.random_vector(N, seed=6), device="cuda")
    y = torch.zeros(N, dtype=torch.float64, device="cuda")
    H.hyel_schur_apply(gp.ctx, H.solver_params(), x.data_ptr(), y.data_ptr())
    for bad in (0.0, -1.0, 1e3, float("nan")):
        with pytest.raises(H.HyelError) as ei:
            H.hyel_set_wait_limit(gp.ctx, bad)
        assert ei.value.code == H.HYEL_EINVAL
    with pytest.raises(H.HyelError) as ei:
        H.hyel_inject_fault(gp.ctx, 7)
    assert ei.value.code == H.HYEL_EINVAL


def test_vanishing_velocity_block_is_singular():
    """rho0 and mu at 1e-300 (both must be > 0 at upload): the mass and
    stiffness parts of A, and with them every 3x3 diagonal block, fall below
    the range of a double's determinant; kappa stays 1e6, so the pressure
    rows stay regular."""
    m = inputs.cube_mesh(3)
    gp = GpuProblem(m, inputs.material_nh(1e-300, 1e6, 1e-300), load={"p_max": 0.0, "t_ramp": DT},
                    with_oracle=False)
    N = gp.N
    dev, sst = gp.stage(inputs.zero_state(N))
    rhs = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    H.hyel_assemble(gp.ctx, H.time_params(dt=DT), sst, 0, rhs.data_ptr())
    with pytest.raises(H.HyelError) as ei:
        H.hyel_solve_setup(gp.ctx)
    assert ei.value.code == H.HYEL_ESINGULAR
    x = torch.zeros(4 * N, dtype=torch.float64, device="cuda")
    st, rc = H.hyel_solve_nested(gp.ctx, H.solver_params(), rhs.data_ptr(), x.data_ptr(), raise_on_error=False)
    assert rc == H.HYEL_ESINGULAR
    gp.close()
