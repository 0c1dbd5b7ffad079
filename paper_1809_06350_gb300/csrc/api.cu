// C-ABI entry points of libhyel (see include/hyel.h): argument checks, error
// translation, context and memory management, kernel-class event timing.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <exception>

#include "internal.h"

struct hyel_ctx {
    hyel::Ctx c;
};

namespace hyel {

static std::atomic<long long> g_launches{0};
thread_local int *g_capture_count = nullptr;
void count_launch() {
    if (g_capture_count) {
        ++*g_capture_count;
        return;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
}

void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        char buf[512];
        std::snprintf(buf, sizeof buf, "CUDA error %s (%s) in %s", cudaGetErrorName(e), cudaGetErrorString(e), what);
        (void)cudaGetLastError();
        throw Error{e == cudaErrorMemoryAllocation ? HYEL_ENOMEM : HYEL_ECUDA, buf};
    }
}

void *dalloc(Ctx &c, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        fail(HYEL_ENOMEM, "cudaMalloc failed (" + std::to_string(bytes) + " bytes)");
    }
    c.allocations.push_back(p);
    c.bytes_held += bytes;
    return p;
}

void dfree_all(Ctx &c) {
    if (!c.allocations.empty()) cudaStreamSynchronize(c.stream);
    for (void *p : c.allocations) cudaFree(p);
    c.allocations.clear();
    c.bytes_held = 0;
}

void prof_begin(Ctx &c, int cls, cudaEvent_t *ev) {
    (void)cls;
    *ev = nullptr;
    if (!c.prof.on || g_capture_count) return;  // no event nodes inside recorded graphs
    if (c.prof.pool.empty()) {
        cudaEvent_t e;
        HYEL_CK(cudaEventCreate(&e));
        c.prof.pool.push_back(e);
    }
    *ev = c.prof.pool.back();
    c.prof.pool.pop_back();
    HYEL_CK(cudaEventRecord(*ev, c.stream));
}

void prof_end(Ctx &c, int cls, cudaEvent_t ev, double bytes) {
    if (!c.prof.on || !ev) return;
    cudaEvent_t e2;
    if (c.prof.pool.empty()) {
        HYEL_CK(cudaEventCreate(&e2));
    } else {
        e2 = c.prof.pool.back();
        c.prof.pool.pop_back();
    }
    HYEL_CK(cudaEventRecord(e2, c.stream));
    c.prof.pending.push_back({ev, e2, cls, bytes});
    if (c.prof.pending.size() >= 4096) {  // drain to bound the number of live events
        HYEL_CK(cudaStreamSynchronize(c.stream));
        for (auto &r : c.prof.pending) {
            float ms = 0;
            HYEL_CK(cudaEventElapsedTime(&ms, r.a, r.b));
            c.prof.ms[r.cls] += ms;
            c.prof.launches[r.cls] += 1;
            c.prof.bytes[r.cls] += r.bytes;
            c.prof.pool.push_back(r.a);
            c.prof.pool.push_back(r.b);
        }
        c.prof.pending.clear();
    }
}

void bar_reset(Ctx &c, unsigned *bar) {
    HYEL_CK(cudaMemsetAsync(bar, 0, kBarWords * sizeof(unsigned), c.stream));
    HYEL_CK(cudaMemcpyAsync(bar + kBarCtl, c.ctl, 32 * sizeof(unsigned), cudaMemcpyDeviceToDevice, c.stream));
}

}  // namespace hyel

namespace {

thread_local std::string g_create_error;

// Makes the context's device current for the duration of one entry point and
// gives the caller's current device back on every exit path, so that a call
// on a context for another device leaves the host thread (and any framework
// that tracks the current device on it) where it was.
struct DeviceGuard {
    int prev = -1;
    // raise = false (teardown): a failure to switch is ignored, not thrown
    explicit DeviceGuard(int dev, bool raise = true) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            (void)cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) {
            cudaError_t e = cudaSetDevice(dev);
            if (e != cudaSuccess) {
                if (raise) hyel::check_cuda(e, "cudaSetDevice");
                (void)cudaGetLastError();
            }
        }
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) (void)cudaSetDevice(prev);
    }
};

// [a, a + na) and [b, b + nb) (bytes) share at least one byte
bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

template <typename F>
int guarded(hyel_ctx *ctx, F &&f) {
    if (!ctx) return HYEL_EINVAL;
    ctx->c.last_error.clear();
    try {
        DeviceGuard dg(ctx->c.device);
        f(ctx->c);
        return HYEL_OK;
    } catch (const hyel::Error &e) {
        ctx->c.last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        ctx->c.last_error = "host allocation failed";
        return HYEL_ENOMEM;
    } catch (const std::exception &e) {
        ctx->c.last_error = e.what();
        return HYEL_EINVAL;
    }
}

}  // namespace

extern "C" {

int hyel_create(hyel_ctx **out, int device, void *cuda_stream) {
    if (!out) return HYEL_EINVAL;
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        g_create_error = "hyel_create: no such CUDA device";
        (void)cudaGetLastError();
        return e != cudaSuccess ? HYEL_ECUDA : HYEL_EINVAL;
    }
    hyel_ctx *ctx = new hyel_ctx();
    ctx->c.device = device;
    ctx->c.stream = (cudaStream_t)cuda_stream;
    int rc = guarded(ctx, [](hyel::Ctx &c) {
        HYEL_CK(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device));
        HYEL_CK(cudaMallocHost(&c.h_red, 64 * sizeof(double)));
        HYEL_CK(cudaMallocHost(&c.h_err, 4 * sizeof(unsigned)));
        HYEL_CK(cudaMalloc(&c.ctl, 32 * sizeof(unsigned)));
        // words 4..5: the control line's own address, so that the block that
        // takes an injected fault can withdraw it at the source (one-shot,
        // also across replays of a CUDA graph)
        unsigned h[32] = {0};
        const unsigned long long self = (unsigned long long)(uintptr_t)c.ctl;
        std::memcpy(h + 4, &self, sizeof self);
        HYEL_CK(cudaMemcpy(c.ctl, h, sizeof h, cudaMemcpyHostToDevice));
    });
    if (rc != HYEL_OK) {
        g_create_error = ctx->c.last_error;
        if (ctx->c.ctl) cudaFree(ctx->c.ctl);
        if (ctx->c.h_red) cudaFreeHost(ctx->c.h_red);
        if (ctx->c.h_err) cudaFreeHost(ctx->c.h_err);
        delete ctx;
        return rc;
    }
    *out = ctx;
    return HYEL_OK;
}

int hyel_destroy(hyel_ctx *ctx) {
    if (!ctx) return HYEL_EINVAL;
    DeviceGuard dg(ctx->c.device, false);
    cudaStreamSynchronize(ctx->c.stream);
    hyel::free_workspace(ctx->c);
    hyel::amg_free(ctx->c);
    hyel::shat_free(ctx->c);
    hyel::acheb_free(ctx->c);
    hyel::dfree_all(ctx->c);
    for (auto &r : ctx->c.prof.pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->c.prof.pool) cudaEventDestroy(e);
    if (ctx->c.h_red) cudaFreeHost(ctx->c.h_red);
    if (ctx->c.h_err) cudaFreeHost(ctx->c.h_err);
    if (ctx->c.ctl) cudaFree(ctx->c.ctl);
    delete ctx;
    return HYEL_OK;
}

int hyel_set_stream(hyel_ctx *ctx, void *cuda_stream) {
    return guarded(ctx, [&](hyel::Ctx &c) { c.stream = (cudaStream_t)cuda_stream; });
}

const char *hyel_last_error(const hyel_ctx *ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->c.last_error.c_str();
}

int hyel_mesh_upload(hyel_ctx *ctx, int64_t n_nodes, const double *X, int64_t n_tets, const int32_t *tets,
                     const hyel_bc *bc, const hyel_material *mat) {
    return guarded(ctx, [&](hyel::Ctx &c) { hyel::mesh_upload(c, n_nodes, X, n_tets, tets, bc, mat); });
}

int hyel_mesh_info(hyel_ctx *ctx, int64_t *info, int n) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!info || n < 0) hyel::fail(HYEL_EINVAL, "mesh_info: null output");
        int64_t v[5] = {c.mesh.N, c.mesh.E, c.mesh.nnzb, c.mesh.nslots, (int64_t)c.bytes_held};
        for (int k = 0; k < n && k < 5; k++) info[k] = v[k];
    });
}

int hyel_assemble(hyel_ctx *ctx, const hyel_time_params *tp, const hyel_state *stage, unsigned flags,
                  double *res_out, double *rhs_out, double *norms_out) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!tp || !stage || !stage->u || !stage->p || !stage->v || !stage->udot || !stage->pdot || !stage->vdot)
            hyel::fail(HYEL_EINVAL, "assemble: null argument");
        if (flags == 0 || (flags & ~(unsigned)(HYEL_RES | HYEL_TAN)))
            hyel::fail(HYEL_EINVAL, "assemble: flags must be HYEL_RES, HYEL_TAN or both");
        const bool tangent = (flags & HYEL_TAN) != 0;
        if (!tangent && rhs_out)
            hyel::fail(HYEL_EINVAL, "assemble: the right-hand side needs HYEL_TAN (its K_{.,udot} R_k terms)");
        hyel::TimeConsts tc = hyel::time_consts(c.mesh, *tp);
        hyel::assemble(c, tc, *stage, res_out, rhs_out, norms_out, tangent);
    });
}

int hyel_matrix_download(hyel_ctx *ctx, int32_t *row_ptr, int32_t *col, double *A, double *B, double *C,
                         double *D) {
    return guarded(ctx, [&](hyel::Ctx &c) { hyel::matrix_download(c, row_ptr, col, A, B, C, D); });
}

int hyel_spmv(hyel_ctx *ctx, int op, int matrix, const void *x, void *y) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!x || !y) hyel::fail(HYEL_EINVAL, "spmv: null vector");
        if (op < HYEL_OP_FULL || op > HYEL_OP_SHAT) hyel::fail(HYEL_EINVAL, "spmv: bad op");
        {
            // input and output lengths of the operator, in elements
            const size_t N = (size_t)c.mesh.N;
            size_t nx = N, ny = N;
            switch (op) {
                case HYEL_OP_FULL: nx = ny = 4 * N; break;
                case HYEL_OP_A:
                case HYEL_OP_AM: nx = ny = 3 * N; break;
                case HYEL_OP_B: ny = 3 * N; break;
                case HYEL_OP_C: nx = 3 * N; break;
                default: break;
            }
            const size_t es = (matrix == HYEL_MAT_SCALED32 || matrix == HYEL_MAT_SCALED_BF16S) ? 4 : 8;
            if (overlaps(x, nx * es, y, ny * es)) hyel::fail(HYEL_EINVAL, "spmv: x and y must not overlap");
        }
        if (op == HYEL_OP_SHAT) {
            if (matrix == HYEL_MAT_SCALED64)
                hyel::shat_spmv<double>(c, (const double *)x, (double *)y);
            else if (matrix == HYEL_MAT_SCALED32)
                hyel::shat_spmv<float>(c, (const float *)x, (float *)y);
            else
                hyel::fail(HYEL_EINVAL, "spmv: S^ exists as HYEL_MAT_SCALED64 and HYEL_MAT_SCALED32 only");
            return;
        }
        if (op == HYEL_OP_AM && (matrix == HYEL_MAT_ASSEMBLED || matrix == HYEL_MAT_TRANSPOSED))
            hyel::fail(HYEL_EINVAL, "spmv: A M^-1 exists for the scaled matrices only");
        if (matrix < HYEL_MAT_ASSEMBLED || matrix > HYEL_MAT_SCALED_BF16S) hyel::fail(HYEL_EINVAL, "spmv: bad matrix");
        if (!c.mat.assembled) hyel::fail(HYEL_ESTATE, "spmv: nothing assembled");
        if (matrix == HYEL_MAT_TRANSPOSED) {
            if (op != HYEL_OP_FULL) hyel::fail(HYEL_EINVAL, "spmv: the transposed matrix supports HYEL_OP_FULL only");
            hyel::spmv_transpose(c, (const double *)x, (double *)y);
            HYEL_CK(cudaGetLastError());
            return;
        }
        if (matrix != HYEL_MAT_ASSEMBLED && !c.mat.scaled) hyel::fail(HYEL_ESTATE, "spmv: call hyel_solve_setup first");
        hyel::DeviceMatrix &M = c.mat;
        if (matrix == HYEL_MAT_SCALED_BF16S) {
            if (op == HYEL_OP_A)
                hyel::spmv_A16_ind(c, M.Ah8, M.Ah1, M.Ahs, (const float *)x, (float *)y, 0, nullptr);
            else if (op == HYEL_OP_AM)
                hyel::spmv_A16_ind(c, M.Amh8, M.Amh1, M.Amhs, (const float *)x, (float *)y, 0, nullptr);
            else
                hyel::fail(HYEL_EINVAL, "spmv: the BF16 copies hold A and A M^-1 only");
        } else if (matrix == HYEL_MAT_SCALED32) {
            const float *xf = (const float *)x;
            float *yf = (float *)y;
            switch (op) {
                case HYEL_OP_A: hyel::spmv_A<float>(c, M.Af, xf, yf); break;
                case HYEL_OP_AM: hyel::spmv_A<float>(c, M.Amf, xf, yf); break;
                case HYEL_OP_B: hyel::spmv_B<float>(c, M.Bf, xf, yf, nullptr); break;
                case HYEL_OP_C: hyel::spmv_C<float>(c, M.Cf, xf, yf, nullptr); break;
                case HYEL_OP_D: hyel::spmv_D<float>(c, M.Df, xf, yf); break;
                default: hyel::fail(HYEL_EINVAL, "spmv: FULL is available for FP64 matrices only");
            }
        } else {
            const double *Av = matrix == HYEL_MAT_ASSEMBLED ? M.A : M.As;
            const double *Bv = matrix == HYEL_MAT_ASSEMBLED ? M.B : M.Bs;
            const double *Cv = matrix == HYEL_MAT_ASSEMBLED ? M.C : M.Cs;
            const double *Dv = matrix == HYEL_MAT_ASSEMBLED ? M.D : M.Ds;
            const double *xd = (const double *)x;
            double *yd = (double *)y;
            switch (op) {
                case HYEL_OP_FULL: hyel::spmv_full64(c, Av, Bv, Cv, Dv, xd, yd); break;
                case HYEL_OP_A: hyel::spmv_A<double>(c, Av, xd, yd); break;
                case HYEL_OP_AM: hyel::spmv_A<double>(c, M.Ams, xd, yd); break;
                case HYEL_OP_B: hyel::spmv_B<double>(c, Bv, xd, yd, nullptr); break;
                case HYEL_OP_C: hyel::spmv_C<double>(c, Cv, xd, yd, nullptr); break;
                case HYEL_OP_D: hyel::spmv_D<double>(c, Dv, xd, yd); break;
            }
        }
        HYEL_CK(cudaGetLastError());
    });
}

int hyel_solve_setup(hyel_ctx *ctx, double *w_out) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        hyel::solve_setup(c);
        if (w_out)
            HYEL_CK(cudaMemcpyAsync(w_out, c.mat.w, 4 * c.mesh.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        HYEL_CK(cudaStreamSynchronize(c.stream));
    });
}

int hyel_schur_hat_setup(hyel_ctx *ctx, double *bounds_out, int64_t *info, int n_info) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (n_info < 0 || (n_info > 0 && !info)) hyel::fail(HYEL_EINVAL, "schur_hat_setup: bad info array");
        hyel::shat_setup(c);
        const hyel::SchurHat &h = *c.sh;
        if (bounds_out) {
            bounds_out[0] = h.h_bounds[0];
            bounds_out[1] = h.h_bounds[1];
        }
        const int64_t v[4] = {h.nnz, h.nslots, h.ncontrib, h.max_row};
        for (int k = 0; k < n_info && k < 4; k++) info[k] = v[k];
    });
}

int hyel_schur_hat_cheb(hyel_ctx *ctx, int matrix, int32_t degree, double ratio, const double *x, double *y) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!x || !y) hyel::fail(HYEL_EINVAL, "schur_hat_cheb: null vector");
        const size_t n = (size_t)c.mesh.N * sizeof(double);
        if (overlaps(x, n, y, n)) hyel::fail(HYEL_EINVAL, "schur_hat_cheb: x and y must not overlap");
        hyel::shat_cheb_apply(c, matrix, degree, ratio, x, y);
    });
}

int hyel_schur_apply(hyel_ctx *ctx, const hyel_solver_params *params, const double *x, double *y,
                     hyel_solve_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!params || !x || !y) hyel::fail(HYEL_EINVAL, "schur_apply: null argument");
        const size_t n = (size_t)c.mesh.N * sizeof(double);
        if (overlaps(x, n, y, n)) hyel::fail(HYEL_EINVAL, "schur_apply: x and y must not overlap");
        hyel::schur_apply(c, *params, x, y, stats);
    });
}

int hyel_a_cheb_setup(hyel_ctx *ctx, double *bounds_out) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        hyel::acheb_setup(c);
        if (bounds_out) {
            bounds_out[0] = c.ach->h_bounds[0];
            bounds_out[1] = c.ach->h_bounds[1];
        }
    });
}

int hyel_a_cheb_apply(hyel_ctx *ctx, int32_t degree, const double *x, double *y) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!x || !y) hyel::fail(HYEL_EINVAL, "a_cheb_apply: null vector");
        const size_t n = 3 * (size_t)c.mesh.N * sizeof(double);
        if (overlaps(x, n, y, n)) hyel::fail(HYEL_EINVAL, "a_cheb_apply: x and y must not overlap");
        hyel::acheb_apply(c, degree, x, y);
    });
}

int hyel_amg_info(hyel_ctx *ctx, int64_t *info, int n) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!info || n < 1) hyel::fail(HYEL_EINVAL, "amg_info: need an output of at least one entry");
        int64_t v[1 + 2 * 16] = {0};
        const int L = hyel::amg_levels(c, v + 1, 2 * 16);
        v[0] = L;
        for (int k = 0; k < n && k < 1 + 2 * std::min(L, 16); k++) info[k] = v[k];
    });
}

int hyel_block_precond_apply(hyel_ctx *ctx, const hyel_solver_params *params, const double *r, double *z,
                             hyel_solve_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!params || !r || !z) hyel::fail(HYEL_EINVAL, "block_precond_apply: null argument");
        const size_t n = 4 * (size_t)c.mesh.N * sizeof(double);
        if (overlaps(r, n, z, n)) hyel::fail(HYEL_EINVAL, "block_precond_apply: r and z must not overlap");
        hyel::block_precond_apply(c, *params, r, z, stats);
    });
}

int hyel_solve_nested(hyel_ctx *ctx, const hyel_solver_params *params, const double *rhs, double *x,
                      hyel_solve_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!params || !rhs || !x) hyel::fail(HYEL_EINVAL, "solve_nested: null argument");
        hyel::solve_nested(c, *params, rhs, x, stats);
    });
}

int hyel_newton_step(hyel_ctx *ctx, const hyel_time_params *tp, const hyel_solver_params *sp, hyel_state *state,
                     hyel_newton_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!tp || !sp || !state || !state->u || !state->p || !state->v || !state->udot || !state->pdot ||
            !state->vdot)
            hyel::fail(HYEL_EINVAL, "newton_step: null argument");
        hyel::newton_step(c, *tp, *sp, *state, stats);
    });
}

int hyel_profile(hyel_ctx *ctx, int enable) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        HYEL_CK(cudaStreamSynchronize(c.stream));
        for (auto &r : c.prof.pending) {
            c.prof.pool.push_back(r.a);
            c.prof.pool.push_back(r.b);
        }
        c.prof.pending.clear();
        for (int k = 0; k < HYEL_K_NCLASSES; k++) {
            c.prof.ms[k] = 0;
            c.prof.launches[k] = 0;
            c.prof.bytes[k] = 0;
        }
        c.prof.on = enable != 0;
    });
}

int hyel_update_material(hyel_ctx *ctx, const hyel_material *mat) {
    return guarded(ctx, [&](hyel::Ctx &c) { hyel::update_material(c, mat); });
}

int hyel_solve_nested_transpose(hyel_ctx *ctx, const hyel_solver_params *params, const double *rhs, double *x,
                                hyel_solve_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!params || !rhs || !x) hyel::fail(HYEL_EINVAL, "solve_nested_transpose: null argument");
        hyel::solve_nested_transpose(c, *params, rhs, x, stats);
    });
}

int hyel_param_sensitivity(hyel_ctx *ctx, const hyel_state *stage, const double *lambda, double *grad) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!stage || !lambda || !grad || !stage->u || !stage->p || !stage->v || !stage->udot || !stage->pdot ||
            !stage->vdot)
            hyel::fail(HYEL_EINVAL, "param_sensitivity: null argument");
        hyel::param_sensitivity(c, *stage, lambda, grad);
        HYEL_CK(cudaStreamSynchronize(c.stream));
    });
}

int hyel_adjoint_step(hyel_ctx *ctx, const hyel_time_params *tp, const hyel_solver_params *sp,
                      const hyel_state *state_n, const hyel_state *state_np1, double *ybar, double *ydotbar,
                      double *grad, double *lambda_out, hyel_solve_stats *stats) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!tp || !sp || !state_n || !state_np1 || !ybar || !ydotbar)
            hyel::fail(HYEL_EINVAL, "adjoint_step: null argument");
        hyel::adjoint_step(c, *tp, *sp, *state_n, *state_np1, ybar, ydotbar, grad, lambda_out, stats);
    });
}

int hyel_residual_norm_static(hyel_ctx *ctx, int matrix, const double *x, const double *b, double *out) {
    return guarded(ctx, [&](hyel::Ctx &c) { hyel::residual_norm_static(c, matrix, x, b, out); });
}

int hyel_set_wait_limit(hyel_ctx *ctx, double seconds) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (!(seconds >= 1e-6 && seconds <= 60.0)) hyel::fail(HYEL_EINVAL, "set_wait_limit: seconds must be in [1e-6, 60]");
        const unsigned long long ns = (unsigned long long)(seconds * 1e9);
        HYEL_CK(cudaMemcpyAsync(c.ctl, &ns, sizeof ns, cudaMemcpyHostToDevice, c.stream));
        HYEL_CK(cudaStreamSynchronize(c.stream));
    });
}

int hyel_inject_fault(hyel_ctx *ctx, int kind) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        if (kind != HYEL_FAULT_NONE && kind != HYEL_FAULT_BARRIER_SKIP)
            hyel::fail(HYEL_EINVAL, "inject_fault: unknown kind");
        const unsigned v = kind == HYEL_FAULT_BARRIER_SKIP ? 1u : 0u;  // block 0 + 1
        HYEL_CK(cudaMemcpyAsync(c.ctl + 2, &v, sizeof v, cudaMemcpyHostToDevice, c.stream));
        HYEL_CK(cudaStreamSynchronize(c.stream));
    });
}

int hyel_fp64_fma_probe(hyel_ctx *ctx, int64_t iters, double *sink, double *flops_out) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        const double f = hyel::fp64_fma_probe(c, iters, sink);
        if (flops_out) *flops_out = f;
    });
}

int hyel_stream_read_probe(hyel_ctx *ctx, const void *buf, int64_t bytes, double *sink) {
    return guarded(ctx, [&](hyel::Ctx &c) { hyel::stream_read_probe(c, buf, bytes, sink); });
}

int hyel_launch_count(int64_t *count) {
    if (!count) return HYEL_EINVAL;
    *count = (int64_t)hyel::g_launches.load(std::memory_order_relaxed);
    return HYEL_OK;
}

int hyel_profile_read(hyel_ctx *ctx, double *ms, int64_t *launches, double *bytes) {
    return guarded(ctx, [&](hyel::Ctx &c) {
        HYEL_CK(cudaStreamSynchronize(c.stream));
        for (auto &r : c.prof.pending) {
            float t = 0;
            HYEL_CK(cudaEventElapsedTime(&t, r.a, r.b));
            c.prof.ms[r.cls] += t;
            c.prof.launches[r.cls] += 1;
            c.prof.bytes[r.cls] += r.bytes;
            c.prof.pool.push_back(r.a);
            c.prof.pool.push_back(r.b);
        }
        c.prof.pending.clear();
        for (int k = 0; k < HYEL_K_NCLASSES; k++) {
            if (ms) ms[k] = c.prof.ms[k];
            if (launches) launches[k] = c.prof.launches[k];
            if (bytes) bytes[k] = c.prof.bytes[k];
        }
    });
}

}  // extern "C"
