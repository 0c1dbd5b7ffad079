// Predictor multi-corrector Newton step of the generalized-alpha scheme (§3.3).
//
//   predictor:  y_{n+1,(0)} = y_n, ydot_{n+1,(0)} = (gamma-1)/gamma ydot_n;
//               Dirichlet components take u = g(t_{n+1}), v = dg/dt(t_{n+1}) and
//               the rates that the update y_{n+1} = y_n + dt ydot_n
//               + gamma dt (ydot_{n+1} - ydot_n) implies (eq. gen_alpha_def_y_n_plus_1,
//               read without its stray comma).
//   corrector:  stage values (eq. gen_alpha_def_y_n_alpha_m/_f), assembly,
//               the stopping test ||R||/||R_(0)|| <= tol_r or ||R|| <= tol_a with
//               ||R_(0)|| the predictor residual, the nested solve, Delta udot
//               from eq. NR_smaller_eqn_2 (zero on Dirichlet components), and the
//               update ydot += Delta ydot, y += gamma dt Delta ydot.
#include <chrono>
#include <cmath>

#include "internal.h"

namespace hyel {

namespace {

struct NArgs {
    int64_t N;
    const uint8_t *dir;
    const double *dir_val;
    // states: [u 3N | p N | v 3N]
    const double *yn, *ydn;
    double *y1, *yd1, *st;
    const double *dx;  // [dv 3N | dp N]
    double am, af, gam, dt, c1;
    double g_s, g_sd;  // ramp s(t_{n+1}) and ds/dt
};

__global__ void k_predictor(NArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n7 = 7 * a.N;
    if (k >= n7) return;
    double y = a.yn[k];
    double yd = (a.gam - 1.0) / a.gam * a.ydn[k];
    // Dirichlet: u in [0, 3N), v in [4N, 7N)
    int64_t node = -1;
    int comp = 0;
    bool is_v = false;
    if (k < 3 * a.N) {
        node = k / 3;
        comp = (int)(k - 3 * node);
    } else if (k >= 4 * a.N) {
        node = (k - 4 * a.N) / 3;
        comp = (int)(k - 4 * a.N - 3 * node);
        is_v = true;
    }
    if (node >= 0 && ((a.dir[node] >> comp) & 1u)) {
        const double G = a.dir_val[3 * node + comp];
        const double target = is_v ? G * a.g_sd : G * a.g_s;
        y = target;
        yd = a.ydn[k] + (target - a.yn[k] - a.dt * a.ydn[k]) / (a.gam * a.dt);
    }
    a.y1[k] = y;
    a.yd1[k] = yd;
}

__global__ void k_stage(NArgs a) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n7 = 7 * a.N;
    if (k >= n7) return;
    a.st[k] = a.yn[k] + a.af * (a.y1[k] - a.yn[k]);
    a.st[n7 + k] = a.ydn[k] + a.am * (a.yd1[k] - a.ydn[k]);
}

// thread per node: Delta udot = (c1/am) Delta vdot - R_k/am; update rates and values
__global__ void k_update(NArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int64_t N = a.N, n7 = 7 * N;
    const unsigned d = a.dir[i];
    const double gdt = a.gam * a.dt;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const bool fixed = (d >> c) & 1u;
        const double dv = fixed ? 0.0 : a.dx[3 * i + c];
        const double rk = a.st[n7 + 3 * i + c] - a.st[4 * N + 3 * i + c];  // udot_am - v_af
        const double du = fixed ? 0.0 : (a.c1 / a.am) * dv - rk / a.am;
        a.yd1[3 * i + c] += du;
        a.y1[3 * i + c] += gdt * du;
        a.yd1[4 * N + 3 * i + c] += dv;
        a.y1[4 * N + 3 * i + c] += gdt * dv;
    }
    const double dp = a.dx[3 * N + i];
    a.yd1[3 * N + i] += dp;
    a.y1[3 * N + i] += gdt * dp;
}

__global__ void k_pack(const double *u, const double *p, const double *v, double *dst, int64_t N) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 3 * N) {
        dst[k] = u[k];
        dst[4 * N + k] = v[k];
    }
    if (k < N) dst[3 * N + k] = p[k];
}

__global__ void k_unpack(const double *src, double *u, double *p, double *v, int64_t N) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < 3 * N) {
        u[k] = src[k];
        v[k] = src[4 * N + k];
    }
    if (k < N) p[k] = src[3 * N + k];
}

}  // namespace

void newton_step(Ctx &c, const hyel_time_params &tp, const hyel_solver_params &sp, hyel_state &s,
                 hyel_newton_stats *out) {
    DeviceMesh &m = c.mesh;
    if (m.N == 0) fail(HYEL_ESTATE, "newton_step: no mesh uploaded");
    if (tp.l_max < 1) fail(HYEL_EINVAL, "newton_step: l_max must be >= 1");
    auto t0 = std::chrono::steady_clock::now();
    const int64_t N = m.N, n7 = 7 * N;
    TimeConsts tc = time_consts(m, tp);
    double *yn = c.vec, *ydn = c.vec + n7, *y1 = c.vec + 2 * n7, *yd1 = c.vec + 3 * n7, *st = c.vec + 4 * n7;
    double *rhs = c.vec + 6 * n7, *dx = rhs + 4 * N;
    const int nb = blocks_for(3 * N, 256);
    (k_pack<<<nb, 256, 0, c.stream>>>(s.u, s.p, s.v, yn, N), ::hyel::count_launch());
    (k_pack<<<nb, 256, 0, c.stream>>>(s.udot, s.pdot, s.vdot, ydn, N), ::hyel::count_launch());
    NArgs a;
    a.N = N;
    a.dir = m.dir;
    a.dir_val = m.dir_val;
    a.yn = yn;
    a.ydn = ydn;
    a.y1 = y1;
    a.yd1 = yd1;
    a.st = st;
    a.dx = dx;
    a.am = tc.am;
    a.af = tc.af;
    a.gam = tc.gam;
    a.dt = tc.dt;
    a.c1 = tc.c1;
    const double t1 = tp.t_n + tp.dt;
    a.g_s = std::fmin(t1 / m.t_ramp, 1.0);
    a.g_sd = t1 < m.t_ramp ? 1.0 / m.t_ramp : 0.0;
    (k_predictor<<<blocks_for(n7, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    hyel_state stage;
    stage.u = st;
    stage.p = st + 3 * N;
    stage.v = st + 4 * N;
    stage.udot = st + n7;
    stage.pdot = st + n7 + 3 * N;
    stage.vdot = st + n7 + 4 * N;
    hyel_newton_stats ns{};
    double norm0 = 0.0, ms_asm = 0.0, ms_sol = 0.0;
    int status = HYEL_OK;
    int l = 1;
    for (; l <= tp.l_max; l++) {
        (k_stage<<<blocks_for(n7, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
        auto ta = std::chrono::steady_clock::now();
        double norms[4];
        // after a corrector update the kinematic residual R_k vanishes up to
        // rounding (the Delta udot of eq. NR_smaller_eqn_2 cancels it), so the
        // K_{.,udot} R_k correction of the right-hand side is formed at l = 1 only
        TimeConsts tcl = tc;
        tcl.skip_corr = l > 1 ? 1 : 0;
        // the stopping test runs on a residual-only pass when the previous
        // residual, squared as quadratic convergence would, already meets the
        // tolerance (to within 10x); the tangent follows only if Newton goes
        // on. Otherwise the tangent pass comes first and its norms decide.
        const double prev = ns.res_norm;
        const bool likely = l > 1 && norm0 > 0 &&
                            ((prev / norm0) * (prev / norm0) <= 10.0 * tp.tol_r || prev * prev / norm0 <= 10.0 * tp.tol_a);
        assemble(c, tcl, stage, nullptr, likely ? nullptr : rhs, norms, !likely);
        if (l == 1) norm0 = norms[0];
        ns.res_norm = norms[0];
        const bool conv = norms[0] <= tp.tol_a || (norm0 > 0 && norms[0] / norm0 <= tp.tol_r);
        if (!conv && likely) assemble(c, tcl, stage, nullptr, rhs, nullptr, true);
        ms_asm += 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - ta).count();
        if (conv) {
            ns.converged = 1;
            break;
        }
        hyel_solve_stats ss{};
        auto tsol = std::chrono::steady_clock::now();
        // after the first correction the Chebyshev intervals of this time
        // step's first iteration are kept (the tangent moves little)
        struct KeepIntervals {
            Ctx &c;
            KeepIntervals(Ctx &cc, bool on) : c(cc) { c.keep_intervals = on; }
            ~KeepIntervals() { c.keep_intervals = false; }
        } keep(c, l > 1);
        try {
            solve_nested(c, sp, rhs, dx, &ss);
        } catch (const Error &e) {
            if (e.code != HYEL_ENOCONV) throw;
            status = HYEL_ENOCONV;
        }
        ms_sol += 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - tsol).count();
        ns.outer_its += ss.outer_its;
        ns.a_its += ss.a_its;
        ns.s_its += ss.s_its;
        ns.inner_its += ss.inner_its;
        (k_update<<<blocks_for(N, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
        HYEL_CK(cudaGetLastError());
    }
    ns.iterations = ns.converged ? l - 1 : tp.l_max;
    ns.res_norm0 = norm0;
    (k_unpack<<<nb, 256, 0, c.stream>>>(y1, s.u, s.p, s.v, N), ::hyel::count_launch());
    (k_unpack<<<nb, 256, 0, c.stream>>>(yd1, s.udot, s.pdot, s.vdot, N), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaStreamSynchronize(c.stream));
    ns.ms_assemble = ms_asm;
    ns.ms_solve = ms_sol;
    ns.ms_total = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (!ns.converged && status == HYEL_OK) status = HYEL_ENOCONV;
    ns.status = status;
    if (out) *out = ns;
    if (status != HYEL_OK) fail(status, "newton_step: Newton did not converge within l_max iterations");
}

}  // namespace hyel
