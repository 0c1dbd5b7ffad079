"""ctypes binding of libhyel (include/hyel.h): the same entry points, argument
marshalling only. Every computation runs in the CUDA library; if the library
is missing this module raises instead of falling back to anything else.

Device arrays are passed as raw pointers (``tensor.data_ptr()`` of CUDA
tensors); the stream is PyTorch's current stream unless given.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhyel.so")

HYEL_OK = 0
HYEL_EINVAL, HYEL_ECUDA, HYEL_ENOMEM, HYEL_ENOCONV = -1, -2, -3, -4
HYEL_EBREAKDOWN, HYEL_ENAN, HYEL_EINVERTED, HYEL_ESINGULAR, HYEL_ESTATE = -5, -6, -7, -8, -9
HYEL_VOL_GIBBS, HYEL_VOL_INCOMPRESSIBLE = 0, 1
HYEL_RES, HYEL_TAN = 1, 2
HYEL_FAULT_NONE, HYEL_FAULT_BARRIER_SKIP = 0, 1
HYEL_PREC_FP64, HYEL_PREC_FP32, HYEL_PREC_BF16S = 0, 1, 2
HYEL_APREC_BJACOBI, HYEL_APREC_AMG, HYEL_APREC_CHEB = 0, 1, 2
HYEL_SPREC_JACOBI, HYEL_SPREC_CHEB = 0, 1
HYEL_BLOCK_LDU, HYEL_BLOCK_DU, HYEL_BLOCK_D, HYEL_BLOCK_SIMPLE = 0, 1, 2, 3
HYEL_INNER_GMRES, HYEL_INNER_CG_SYM = 0, 1
HYEL_OP_FULL, HYEL_OP_A, HYEL_OP_B, HYEL_OP_C, HYEL_OP_D, HYEL_OP_AM, HYEL_OP_SHAT = 0, 1, 2, 3, 4, 5, 6
HYEL_MAT_ASSEMBLED, HYEL_MAT_SCALED64, HYEL_MAT_SCALED32, HYEL_MAT_TRANSPOSED, HYEL_MAT_SCALED_BF16S = 0, 1, 2, 3, 4
(HYEL_K_SPMV_A64, HYEL_K_SPMV_A32, HYEL_K_SPMV_FULL64, HYEL_K_ASSEMBLE, HYEL_K_GATHER, HYEL_K_SPMV_A16,
 HYEL_K_GMRES_A, HYEL_K_GMRES_S, HYEL_K_SCHUR_HAT, HYEL_K_ASSEMBLE_RES, HYEL_K_ASSEMBLE_CORR) = range(11)
HYEL_K_NCLASSES = 11
K_NAMES = ["spmv_A64", "spmv_A32", "spmv_full64", "assemble_elem", "gather", "spmv_A16", "gmres_A", "gmres_S",
           "schur_hat", "assemble_res", "assemble_corr"]

# every symbol include/hyel.h declares
EXPORTS = [
    "hyel_create", "hyel_destroy", "hyel_set_stream", "hyel_last_error", "hyel_mesh_upload",
    "hyel_mesh_info", "hyel_assemble", "hyel_matrix_download", "hyel_spmv", "hyel_solve_setup",
    "hyel_schur_apply", "hyel_solve_nested", "hyel_newton_step", "hyel_profile", "hyel_profile_read",
    "hyel_launch_count", "hyel_residual_norm_static", "hyel_update_material",
    "hyel_solve_nested_transpose", "hyel_param_sensitivity", "hyel_adjoint_step",
    "hyel_schur_hat_setup", "hyel_schur_hat_cheb", "hyel_block_precond_apply", "hyel_a_cheb_setup",
    "hyel_a_cheb_apply", "hyel_amg_info", "hyel_set_wait_limit", "hyel_inject_fault",
    "hyel_fp64_fma_probe", "hyel_stream_read_probe",
]

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class HyelMaterial(C.Structure):
    _fields_ = [("vol_model", C.c_int32), ("n_fibres", C.c_int32), ("rho0", C.c_double), ("mu", C.c_double),
                ("kappa", C.c_double), ("k1", C.c_double), ("k2", C.c_double), ("kd", C.c_double),
                ("c_m", C.c_double), ("body", C.c_double * 3), ("mu_e", _dp), ("kappa_e", _dp),
                ("k1_e", _dp), ("k2_e", _dp), ("fibre_a1", _dp), ("fibre_a2", _dp)]


class HyelBC(C.Structure):
    _fields_ = [("n_dirichlet", C.c_int64), ("dir_node", _ip), ("dir_comp", _ip), ("dir_value", _dp),
                ("n_traction_tris", C.c_int64), ("traction_tris", _ip), ("traction_dir", C.c_double * 3),
                ("p_max", C.c_double), ("t_ramp", C.c_double)]


class HyelState(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("u", "p", "v", "udot", "pdot", "vdot")]


class HyelTimeParams(C.Structure):
    _fields_ = [("rho_inf", C.c_double), ("dt", C.c_double), ("t_n", C.c_double), ("tol_r", C.c_double),
                ("tol_a", C.c_double), ("l_max", C.c_int32), ("rhs_literal", C.c_int32)]


class HyelKrylovLevel(C.Structure):
    _fields_ = [("rtol", C.c_double), ("atol", C.c_double), ("maxit", C.c_int32), ("restart", C.c_int32)]


class HyelSolverParams(C.Structure):
    _fields_ = [("outer", HyelKrylovLevel), ("a", HyelKrylovLevel), ("s", HyelKrylovLevel),
                ("inner", HyelKrylovLevel), ("precision", C.c_int32), ("check_every", C.c_int32),
                ("graph", C.c_int32), ("a_precond", C.c_int32), ("s_precond", C.c_int32),
                ("s_cheb_degree", C.c_int32), ("s_cheb_ratio", C.c_double), ("block_precond", C.c_int32),
                ("inner_solver", C.c_int32), ("a_cheb_degree", C.c_int32), ("reserved_", C.c_int32)]


class HyelSolveStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("outer_its", C.c_int32), ("a_its", C.c_int64), ("s_its", C.c_int64),
                ("inner_its", C.c_int64), ("a_solves", C.c_int32), ("s_solves", C.c_int32),
                ("inner_solves", C.c_int32), ("rel_residual", C.c_double), ("ms_setup", C.c_double),
                ("ms_solve", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class HyelNewtonStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("converged", C.c_int32), ("pad_", C.c_int32),
                ("res_norm0", C.c_double), ("res_norm", C.c_double), ("outer_its", C.c_int64),
                ("a_its", C.c_int64), ("s_its", C.c_int64), ("inner_its", C.c_int64),
                ("ms_assemble", C.c_double), ("ms_solve", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad_"}


class HyelError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hyel error {code}: {msg}")
        self.code = code


_LIB = None


def lib():
    """Load libhyel.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhyel.so is not built ({LIB_PATH}); run "
                               "`python -m paper_1809_06350_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        sig = {
            "hyel_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
            "hyel_destroy": (C.c_int, [vp]),
            "hyel_set_stream": (C.c_int, [vp, vp]),
            "hyel_last_error": (C.c_char_p, [vp]),
            "hyel_mesh_upload": (C.c_int, [vp, C.c_int64, _dp, C.c_int64, _ip, C.POINTER(HyelBC),
                                           C.POINTER(HyelMaterial)]),
            "hyel_mesh_info": (C.c_int, [vp, C.POINTER(C.c_int64), C.c_int]),
            "hyel_assemble": (C.c_int, [vp, C.POINTER(HyelTimeParams), C.POINTER(HyelState), C.c_uint, vp, vp,
                                        _dp]),
            "hyel_matrix_download": (C.c_int, [vp, _ip, _ip, _dp, _dp, _dp, _dp]),
            "hyel_spmv": (C.c_int, [vp, C.c_int, C.c_int, vp, vp]),
            "hyel_solve_setup": (C.c_int, [vp, vp]),
            "hyel_schur_apply": (C.c_int, [vp, C.POINTER(HyelSolverParams), vp, vp, C.POINTER(HyelSolveStats)]),
            "hyel_solve_nested": (C.c_int, [vp, C.POINTER(HyelSolverParams), vp, vp, C.POINTER(HyelSolveStats)]),
            "hyel_newton_step": (C.c_int, [vp, C.POINTER(HyelTimeParams), C.POINTER(HyelSolverParams),
                                           C.POINTER(HyelState), C.POINTER(HyelNewtonStats)]),
            "hyel_profile": (C.c_int, [vp, C.c_int]),
            "hyel_profile_read": (C.c_int, [vp, _dp, C.POINTER(C.c_int64), _dp]),
            "hyel_launch_count": (C.c_int, [C.POINTER(C.c_int64)]),
            "hyel_residual_norm_static": (C.c_int, [vp, C.c_int, vp, vp, vp]),
            "hyel_update_material": (C.c_int, [vp, C.POINTER(HyelMaterial)]),
            "hyel_solve_nested_transpose": (C.c_int, [vp, C.POINTER(HyelSolverParams), vp, vp,
                                                      C.POINTER(HyelSolveStats)]),
            "hyel_param_sensitivity": (C.c_int, [vp, C.POINTER(HyelState), vp, vp]),
            "hyel_adjoint_step": (C.c_int, [vp, C.POINTER(HyelTimeParams), C.POINTER(HyelSolverParams),
                                            C.POINTER(HyelState), C.POINTER(HyelState), vp, vp, vp, vp,
                                            C.POINTER(HyelSolveStats)]),
            "hyel_schur_hat_setup": (C.c_int, [vp, _dp, C.POINTER(C.c_int64), C.c_int]),
            "hyel_schur_hat_cheb": (C.c_int, [vp, C.c_int, C.c_int32, C.c_double, vp, vp]),
            "hyel_a_cheb_setup": (C.c_int, [vp, _dp]),
            "hyel_a_cheb_apply": (C.c_int, [vp, C.c_int32, vp, vp]),
            "hyel_amg_info": (C.c_int, [vp, C.POINTER(C.c_int64), C.c_int]),
            "hyel_block_precond_apply": (C.c_int, [vp, C.POINTER(HyelSolverParams), vp, vp,
                                                   C.POINTER(HyelSolveStats)]),
            "hyel_set_wait_limit": (C.c_int, [vp, C.c_double]),
            "hyel_inject_fault": (C.c_int, [vp, C.c_int]),
            "hyel_fp64_fma_probe": (C.c_int, [vp, C.c_int64, vp, _dp]),
            "hyel_stream_read_probe": (C.c_int, [vp, vp, C.c_int64, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(ctx, rc):
    if rc != HYEL_OK:
        msg = lib().hyel_last_error(ctx)
        raise HyelError(rc, msg.decode() if msg else "")
    return rc


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


# ------------------------------------------------------------------ entry points (same names)

def hyel_create(device=0, stream=None):
    ctx = C.c_void_p()
    rc = lib().hyel_create(C.byref(ctx), int(device), C.c_void_p(stream or 0))
    if rc != HYEL_OK:
        raise HyelError(rc, lib().hyel_last_error(None).decode())
    return ctx


def hyel_destroy(ctx):
    return _check(ctx, lib().hyel_destroy(ctx))


def hyel_set_stream(ctx, stream):
    return _check(ctx, lib().hyel_set_stream(ctx, C.c_void_p(stream or 0)))


def hyel_last_error(ctx):
    return lib().hyel_last_error(ctx).decode()


def hyel_mesh_upload(ctx, X, tets, bc, mat):
    X = _arr(X, np.float64)
    tets = _arr(tets, np.int32)
    return _check(ctx, lib().hyel_mesh_upload(ctx, X.shape[0], _ptr(X, C.c_double), tets.shape[0],
                                              _ptr(tets, C.c_int32), C.byref(bc), C.byref(mat)))


def hyel_mesh_info(ctx):
    out = (C.c_int64 * 5)()
    _check(ctx, lib().hyel_mesh_info(ctx, out, 5))
    return {"N": out[0], "E": out[1], "nnzb": out[2], "nslots": out[3], "bytes": out[4]}


def hyel_assemble(ctx, tp, stage, res_out=0, rhs_out=0, want_norms=True, flags=HYEL_RES | HYEL_TAN):
    norms = (C.c_double * 4)()
    _check(ctx, lib().hyel_assemble(ctx, C.byref(tp), C.byref(stage), int(flags), C.c_void_p(res_out or 0),
                                    C.c_void_p(rhs_out or 0), norms if want_norms else None))
    return list(norms)


def hyel_matrix_download(ctx, N, nnzb):
    rp = np.zeros(N + 1, np.int32)
    col = np.zeros(nnzb, np.int32)
    A = np.zeros(nnzb * 9)
    B = np.zeros(nnzb * 3)
    Cm = np.zeros(nnzb * 3)
    D = np.zeros(nnzb)
    _check(ctx, lib().hyel_matrix_download(ctx, _ptr(rp, C.c_int32), _ptr(col, C.c_int32), _ptr(A, C.c_double),
                                           _ptr(B, C.c_double), _ptr(Cm, C.c_double), _ptr(D, C.c_double)))
    return rp, col, A.reshape(nnzb, 3, 3), B.reshape(nnzb, 3), Cm.reshape(nnzb, 3), D


def hyel_spmv(ctx, op, matrix, x_ptr, y_ptr):
    return _check(ctx, lib().hyel_spmv(ctx, int(op), int(matrix), C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def hyel_solve_setup(ctx, w_out=0):
    return _check(ctx, lib().hyel_solve_setup(ctx, C.c_void_p(w_out or 0)))


def hyel_schur_hat_setup(ctx):
    """Builds the explicit S^ of the current scaled system; returns
    ((lmin, lmax) estimated for the Chebyshev interval, info dict)."""
    b = (C.c_double * 2)()
    info = (C.c_int64 * 4)()
    _check(ctx, lib().hyel_schur_hat_setup(ctx, b, info, 4))
    return (b[0], b[1]), {"nnz": info[0], "slots": info[1], "contributions": info[2], "max_row": info[3]}


def hyel_schur_hat_cheb(ctx, degree, ratio, x_ptr, y_ptr, matrix=HYEL_MAT_SCALED64):
    _check(ctx, lib().hyel_schur_hat_cheb(ctx, int(matrix), int(degree), float(ratio), C.c_void_p(x_ptr),
                                          C.c_void_p(y_ptr)))


def hyel_a_cheb_setup(ctx):
    """The A-Chebyshev interval (lmin, lmax) of the current scaled system."""
    b = (C.c_double * 2)()
    _check(ctx, lib().hyel_a_cheb_setup(ctx, b))
    return b[0], b[1]


def hyel_a_cheb_apply(ctx, degree, x_ptr, y_ptr):
    _check(ctx, lib().hyel_a_cheb_apply(ctx, int(degree), C.c_void_p(x_ptr), C.c_void_p(y_ptr)))


def hyel_amg_info(ctx):
    """[(block-nodes, stored blocks) per level] of the multigrid hierarchy ([] before it is built)."""
    out = (C.c_int64 * 33)()
    _check(ctx, lib().hyel_amg_info(ctx, out, 33))
    return [(out[1 + 2 * l], out[2 + 2 * l]) for l in range(out[0])]


def hyel_block_precond_apply(ctx, params, r_ptr, z_ptr):
    st = HyelSolveStats()
    _check(ctx, lib().hyel_block_precond_apply(ctx, C.byref(params), C.c_void_p(r_ptr), C.c_void_p(z_ptr),
                                               C.byref(st)))
    return st


def hyel_schur_apply(ctx, params, x_ptr, y_ptr):
    st = HyelSolveStats()
    _check(ctx, lib().hyel_schur_apply(ctx, C.byref(params), C.c_void_p(x_ptr), C.c_void_p(y_ptr), C.byref(st)))
    return st


def hyel_solve_nested(ctx, params, rhs_ptr, x_ptr, raise_on_error=True):
    st = HyelSolveStats()
    rc = lib().hyel_solve_nested(ctx, C.byref(params), C.c_void_p(rhs_ptr), C.c_void_p(x_ptr), C.byref(st))
    if raise_on_error:
        _check(ctx, rc)
    return st, rc


def hyel_newton_step(ctx, tp, sp, state, raise_on_error=True):
    st = HyelNewtonStats()
    rc = lib().hyel_newton_step(ctx, C.byref(tp), C.byref(sp), C.byref(state), C.byref(st))
    if raise_on_error:
        _check(ctx, rc)
    return st, rc


def hyel_profile(ctx, enable):
    return _check(ctx, lib().hyel_profile(ctx, int(enable)))


def hyel_profile_read(ctx):
    ms = (C.c_double * HYEL_K_NCLASSES)()
    n = (C.c_int64 * HYEL_K_NCLASSES)()
    by = (C.c_double * HYEL_K_NCLASSES)()
    _check(ctx, lib().hyel_profile_read(ctx, ms, n, by))
    return {K_NAMES[k]: {"ms": ms[k], "launches": n[k], "bytes": by[k]} for k in range(HYEL_K_NCLASSES)}


def hyel_update_material(ctx, mat):
    return _check(ctx, lib().hyel_update_material(ctx, C.byref(mat)))


def hyel_solve_nested_transpose(ctx, params, rhs_ptr, x_ptr, raise_on_error=True):
    st = HyelSolveStats()
    rc = lib().hyel_solve_nested_transpose(ctx, C.byref(params), C.c_void_p(rhs_ptr), C.c_void_p(x_ptr),
                                           C.byref(st))
    if raise_on_error:
        _check(ctx, rc)
    return st, rc


def hyel_param_sensitivity(ctx, stage, lam_ptr, grad_ptr):
    return _check(ctx, lib().hyel_param_sensitivity(ctx, C.byref(stage), C.c_void_p(lam_ptr), C.c_void_p(grad_ptr)))


def hyel_adjoint_step(ctx, tp, sp, state_n, state_np1, ybar_ptr, ydbar_ptr, grad_ptr=0, lam_ptr=0):
    st = HyelSolveStats()
    _check(ctx, lib().hyel_adjoint_step(ctx, C.byref(tp), C.byref(sp), C.byref(state_n), C.byref(state_np1),
                                        C.c_void_p(ybar_ptr), C.c_void_p(ydbar_ptr), C.c_void_p(grad_ptr or 0),
                                        C.c_void_p(lam_ptr or 0), C.byref(st)))
    return st


def hyel_residual_norm_static(ctx, matrix, x_ptr, b_ptr, out_ptr):
    """out[0] = ||b - M x||, out[1] = ||b|| (device [2]); allocates nothing on
    the device (fixed scratch array inside the library)."""
    return _check(ctx, lib().hyel_residual_norm_static(ctx, int(matrix), C.c_void_p(x_ptr), C.c_void_p(b_ptr),
                                                       C.c_void_p(out_ptr)))


def hyel_set_wait_limit(ctx, seconds):
    return _check(ctx, lib().hyel_set_wait_limit(ctx, float(seconds)))


def hyel_inject_fault(ctx, kind):
    return _check(ctx, lib().hyel_inject_fault(ctx, int(kind)))


def hyel_fp64_fma_probe(ctx, iters, sink_ptr):
    """Launches the FP64 FMA probe on the context's stream; returns its flops."""
    f = C.c_double()
    _check(ctx, lib().hyel_fp64_fma_probe(ctx, int(iters), C.c_void_p(sink_ptr), C.byref(f)))
    return f.value


def hyel_stream_read_probe(ctx, buf_ptr, nbytes, sink_ptr):
    return _check(ctx, lib().hyel_stream_read_probe(ctx, C.c_void_p(buf_ptr), int(nbytes), C.c_void_p(sink_ptr)))


def hyel_launch_count():
    n = C.c_int64()
    rc = lib().hyel_launch_count(C.byref(n))
    if rc != HYEL_OK:
        raise HyelError(rc, "launch_count")
    return n.value


# ------------------------------------------------------------------ marshalling helpers

def level(rtol, maxit, restart, atol=1e-50):
    return HyelKrylovLevel(rtol, atol, maxit, restart)


def solver_params(outer_rtol=1e-10, sub_rtol=1e-2, precision=HYEL_PREC_FP64, outer=(200, 200),
                  a=(500, 500), s=(200, 200), inner=(500, 500), check_every=4, inner_rtol=None, graph=1,
                  a_precond=0, s_precond=0, s_cheb_degree=4, s_cheb_ratio=0.0, block_precond=0,
                  inner_solver=0, a_cheb_degree=8):
    """Solver controls with the paper's defaults (§5: FGMRES(200), A: GMRES(500),
    S: GMRES(200), inner GMRES(500), absolute tolerances 1e-50). a_precond:
    HYEL_APREC_BJACOBI (default), HYEL_APREC_AMG or HYEL_APREC_CHEB; s_precond: HYEL_SPREC_JACOBI
    (default) or HYEL_SPREC_CHEB (degree s_cheb_degree on [lmin, lmax] from Ritz
    estimates, or on [lmax / s_cheb_ratio, lmax] when s_cheb_ratio > 1);
    block_precond: HYEL_BLOCK_LDU (Algorithm 1, default), _DU, _D or _SIMPLE;
    inner_solver: HYEL_INNER_GMRES (default) or HYEL_INNER_CG_SYM (CG on (A + A^T)/2);
    a_cheb_degree: the degree of the HYEL_APREC_CHEB polynomial."""
    ir = sub_rtol if inner_rtol is None else inner_rtol
    return HyelSolverParams(level(outer_rtol, *outer), level(sub_rtol, *a), level(sub_rtol, *s),
                            level(ir, *inner), precision, check_every, graph, a_precond, s_precond,
                            s_cheb_degree, s_cheb_ratio, block_precond, inner_solver, a_cheb_degree, 0)


def time_params(dt=1e-3, t_n=0.0, rho_inf=0.5, tol_r=1e-6, tol_a=1e-6, l_max=20, rhs_literal=0):
    return HyelTimeParams(rho_inf, dt, t_n, tol_r, tol_a, l_max, rhs_literal)


def material_struct(mat, fields=None, mesh=None):
    """HyelMaterial for a material dict (and optional per-element fields);
    returns (struct, keepalive) -- keep the second alive while the struct is used."""
    fields = fields or {}
    keep = {}

    def opt(name):
        if name in fields:
            a = _arr(fields[name], np.float64)
            keep[name] = a
            return _ptr(a, C.c_double)
        return None

    fa1 = fa2 = None
    if mat["fibres"]:
        keep["a1"] = _arr(mesh["fibre_a1"], np.float64)
        keep["a2"] = _arr(mesh["fibre_a2"], np.float64)
        fa1 = _ptr(keep["a1"], C.c_double)
        fa2 = _ptr(keep["a2"], C.c_double)
    vol = HYEL_VOL_INCOMPRESSIBLE if mat["vol"] == "incompressible" else HYEL_VOL_GIBBS
    m = HyelMaterial(vol, int(mat["fibres"]), mat["rho0"], mat["mu"], mat["kappa"], mat["k1"],
                     mat["k2"], mat["kd"], mat["c_m"], (C.c_double * 3)(*mat["body"]),
                     opt("mu_e"), opt("kappa_e"), opt("k1_e"), opt("k2_e"), fa1, fa2)
    return m, keep


class MeshInputs:
    """Keeps the host arrays that the C structs point to alive."""

    def __init__(self, mesh, mat, fields=None, load=None):
        fields = fields or {}
        load = load or {"p_max": 0.0, "t_ramp": 1.0}
        self.X = _arr(mesh["X"], np.float64)
        self.tets = _arr(mesh["tets"], np.int32)
        d = _arr(mesh["dirichlet"], np.int32)
        self.dir_node = _arr(d[:, 0], np.int32)
        self.dir_comp = _arr(d[:, 1], np.int32)
        self.dir_val = _arr(mesh["dirichlet_values"], np.float64)
        self.tris = _arr(mesh["traction_tris"], np.int32).reshape(-1, 3)
        self.bc = HyelBC(len(self.dir_node), _ptr(self.dir_node, C.c_int32), _ptr(self.dir_comp, C.c_int32),
                         _ptr(self.dir_val, C.c_double), self.tris.shape[0], _ptr(self.tris, C.c_int32),
                         (C.c_double * 3)(*np.asarray(mesh["traction_dir"], dtype=np.float64)),
                         float(load["p_max"]), float(load["t_ramp"]))
        self.mat, self.keep = material_struct(mat, fields, mesh)


def state_struct(u, p, v, udot, pdot, vdot):
    """HyelState from six CUDA tensors (float64, contiguous)."""
    return HyelState(*(t.data_ptr() for t in (u, p, v, udot, pdot, vdot)))
