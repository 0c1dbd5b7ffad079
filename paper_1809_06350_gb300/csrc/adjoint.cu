// Discrete adjoint of the generalized-alpha Newton step (pattern 3):
// transposed nested solve, parameter sensitivities, and one reverse step.
//
// Step map (§3.2, §3.3): z = ydot_{n+1} solves F(z; y_n, ydot_n, theta) = 0 with
// F = [R_k bar ; R_p ; R_m] at the stage values ydot_{n+am} = (1-am) ydot_n +
// am z, y_{n+af} = y_n + af dt (1-gam) ydot_n + af gam dt z, and
// y_{n+1} = y_n + dt (1-gam) ydot_n + gam dt z. For an objective of the final
// state, with ybar = dJ/dy_{n+1} and ydbar = dJ/dydot_{n+1}:
//   K^T lam = g,  g = ydbar + gam dt ybar,  K = dF/dz = am F_ydot + af gam dt F_y,
//   ybar_n  = ybar - F_y^T lam,
//   ydbar_n = dt (1-gam) ybar - ((1-am) F_ydot + af dt (1-gam) F_y)^T lam,
//   thetabar -= (dF/dtheta)^T lam,
// F_y = dF/dy_{n+af}, F_ydot = dF/dydot_{n+am}. The kinematic factorization
// K = L U (eq. K_block_decomposition) gives K^T = U^T L^T: U^T mu = g is
// explicit (mu_u = g_u/am, mu_p = g_p, mu_v = g_v + (c1/am) g_u), the
// momentum/mass rows of L^T are the transposed reduced system
// [[A^T, C^T], [B^T, D^T]] [lam_m ; lam_p] = [mu_v ; mu_p], solved by the
// same nested FGMRES on the transposed blocks, and
// lam_k = mu_u - (c1/am) (dR/du)^T lam.
// The partial Jacobians are the reduced tangent assembled with unit weights
// (am, c1, c2) = (1, 0, 0): d/dydot; (0, 1, 0): d/d(p, v); (0, 0, 1): d/du.
// Dirichlet components (homogeneous constraints) carry zero adjoint.
#include <chrono>
#include <cmath>

#include "internal.h"

namespace hyel {

namespace {

// ------------------------------------------------------------ dual numbers
template <int NP>
struct Dual {
    double v;
    double d[NP];
};
template <int NP>
__device__ __forceinline__ Dual<NP> dconst(double v) {
    Dual<NP> r;
    r.v = v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = 0.0;
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> operator+(const Dual<NP> &a, const Dual<NP> &b) {
    Dual<NP> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = a.d[k] + b.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> operator-(const Dual<NP> &a, const Dual<NP> &b) {
    Dual<NP> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = a.d[k] - b.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> operator*(const Dual<NP> &a, const Dual<NP> &b) {
    Dual<NP> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = a.d[k] * b.v + a.v * b.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> operator*(double s, const Dual<NP> &a) {
    Dual<NP> r;
    r.v = s * a.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = s * a.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> operator+(double s, const Dual<NP> &a) {
    Dual<NP> r = a;
    r.v += s;
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> dinv(const Dual<NP> &a) {
    Dual<NP> r;
    r.v = 1.0 / a.v;
    const double dd = -r.v * r.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = dd * a.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> dsqrt(const Dual<NP> &a) {
    Dual<NP> r;
    r.v = sqrt(a.v);
    const double dd = 0.5 / r.v;
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = dd * a.d[k];
    return r;
}
template <int NP>
__device__ __forceinline__ Dual<NP> dexp(const Dual<NP> &a) {
    Dual<NP> r;
    r.v = exp(a.v);
#pragma unroll
    for (int k = 0; k < NP; k++) r.d[k] = r.v * a.d[k];
    return r;
}

constexpr double QA = 0.58541019662496845446;
constexpr double QB = 0.13819660112501051518;
constexpr double QAB = QA - QB;

struct SensArgs {
    const int4 *tets;
    const double *geo, *mat, *fib;
    const uint8_t *dir;
    int64_t E, N;
    int vol, nfib;
    double rho0, kd, b0, b1, b2;
    const double *u, *p, *v, *ud, *pd, *vd;
    const double *lam;  // [lam_k 3N | lam_p N | lam_m 3N]
    double *grad;       // [E][4], accumulated
};

// -lam^T dR_e/dtheta_e for theta = (mu, kappa, k1, k2): the element residual of
// Appendix A evaluated with forward-mode dual numbers in the parameters.
__global__ void __launch_bounds__(128) k_param_sensitivity(SensArgs a) {
    typedef Dual<4> D4;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    const int64_t E = a.E, N = a.N;
    const int4 t4 = a.tets[e];
    const int nd[4] = {t4.x, t4.y, t4.z, t4.w};
    double g[4][3];
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int I = 0; I < 3; I++) g[A][I] = a.geo[(A * 3 + I) * E + e];
    const double V = a.geo[12 * E + e];
    const double tau0 = a.geo[13 * E + e];
    D4 mu = dconst<4>(a.mat[e]);
    mu.d[0] = 1.0;
    D4 kappa = dconst<4>(a.mat[E + e]);
    kappa.d[1] = 1.0;
    D4 k1 = dconst<4>(a.nfib ? a.mat[2 * E + e] : 0.0);
    k1.d[2] = 1.0;
    D4 k2 = dconst<4>(a.nfib ? a.mat[3 * E + e] : 1.0);
    k2.d[3] = 1.0;
    const double bf[3] = {a.b0, a.b1, a.b2};
    double u[4][3], vdb[4][3], p[4], pd[4], lm[4][3], lp[4];  // the velocity terms carry no material parameter
#pragma unroll
    for (int A = 0; A < 4; A++) {
        const int64_t n = nd[A];
        const unsigned df = a.dir[n];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            u[A][i] = a.u[3 * n + i];
            vdb[A][i] = a.vd[3 * n + i] - bf[i];
            lm[A][i] = ((df >> i) & 1u) ? 0.0 : a.lam[4 * N + 3 * n + i];
        }
        p[A] = a.p[n];
        pd[A] = a.pd[n];
        lp[A] = a.lam[3 * N + n];
    }
    double F[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int I = 0; I < 3; I++)
            F[i][I] = (i == I ? 1.0 : 0.0) + u[0][i] * g[0][I] + u[1][i] * g[1][I] + u[2][i] * g[2][I] + u[3][i] * g[3][I];
    double cof[3][3];
    cof[0][0] = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    cof[0][1] = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    cof[0][2] = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    cof[1][0] = F[0][2] * F[2][1] - F[0][1] * F[2][2];
    cof[1][1] = F[0][0] * F[2][2] - F[0][2] * F[2][0];
    cof[1][2] = F[0][1] * F[2][0] - F[0][0] * F[2][1];
    cof[2][0] = F[0][1] * F[1][2] - F[0][2] * F[1][1];
    cof[2][1] = F[0][2] * F[1][0] - F[0][0] * F[1][2];
    cof[2][2] = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    const double J = F[0][0] * cof[0][0] + F[0][1] * cof[0][1] + F[0][2] * cof[0][2];
    if (!(J > 0.0)) return;
    const double iJ = 1.0 / J;
    double n[4][3], f[4][3];
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            n[A][i] = (g[A][0] * cof[i][0] + g[A][1] * cof[i][1] + g[A][2] * cof[i][2]) * iJ;
            f[A][i] = F[i][0] * g[A][0] + F[i][1] * g[A][1] + F[i][2] * g[A][2];
        }
    double I1 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int I = 0; I < 3; I++) I1 += F[i][I] * F[i][I];
    const double cJ = cbrt(J);
    const double aJ = 1.0 / (cJ * cJ);
    double gp[3];
#pragma unroll
    for (int i = 0; i < 3; i++) gp[i] = p[0] * n[0][i] + p[1] * n[1][i] + p[2] * n[2][i] + p[3] * n[3][i];
    const double W = 0.25 * V * J, JV = J * V;
    // quadrature values depending on kappa
    D4 xrv[3][4], xb[4];
    for (int q = 0; q < 4; q++) {
        const double pq = QAB * p[q] + QB * (p[0] + p[1] + p[2] + p[3]);
        const double pdq = QAB * pd[q] + QB * (pd[0] + pd[1] + pd[2] + pd[3]);
        D4 rho, beta;
        if (a.vol == HYEL_VOL_GIBBS) {
            const D4 s = dsqrt(dconst<4>(pq * pq) + kappa * kappa);
            beta = dinv(s);
            rho = a.rho0 * ((pq + s) * dinv(kappa));
        } else {
            rho = dconst<4>(a.rho0);
            beta = dconst<4>(0.0);
        }
        xb[q] = pdq * beta;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const double vq = QAB * vdb[q][i] + QB * (vdb[0][i] + vdb[1][i] + vdb[2][i] + vdb[3][i]);
            xrv[i][q] = vq * rho;
        }
    }
    // tau = c_m h / (c rho0) with c(mu, kappa): tau = tau0 c0 / c
    D4 c2w = a.vol == HYEL_VOL_GIBBS ? (1.0 / a.rho0) * (kappa + (4.0 / 3.0) * mu) : (1.0 / a.rho0) * mu;
    const D4 cw = dsqrt(c2w);
    const D4 tau = (tau0 * cw.v) * dinv(cw);
    double grad[4] = {0, 0, 0, 0};
    D4 Srv[3];
#pragma unroll
    for (int i = 0; i < 3; i++) Srv[i] = xrv[i][0] + xrv[i][1] + xrv[i][2] + xrv[i][3];
    const D4 Sb = xb[0] + xb[1] + xb[2] + xb[3];
    D4 sig[3];
#pragma unroll
    for (int i = 0; i < 3; i++) sig[i] = JV * gp[i] + W * Srv[i];
    // fibre stress factors phi'_t(k1, k2)
    D4 phi[2];
    double fE[2][4][3];
    const double kd = a.kd, kd3 = 1.0 - 3.0 * a.kd;
    if (a.nfib) {
        for (int tf = 0; tf < 2; tf++) {
            double av[3], Fa[3], Fa2 = 0.0;
#pragma unroll
            for (int I = 0; I < 3; I++) av[I] = a.fib[(3 * tf + I) * E + e];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                Fa[i] = F[i][0] * av[0] + F[i][1] * av[1] + F[i][2] * av[2];
                Fa2 += Fa[i] * Fa[i];
            }
            const double hc = kd * I1 + kd3 * Fa2;
            const double Eb = aJ * hc - 1.0;
            phi[tf] = (Eb * 1.0) * (k1 * dexp((Eb * Eb) * k2));
#pragma unroll
            for (int A = 0; A < 4; A++) {
                const double ga = g[A][0] * av[0] + g[A][1] * av[1] + g[A][2] * av[2];
#pragma unroll
                for (int i = 0; i < 3; i++)
                    fE[tf][A][i] = aJ * (2.0 * (kd * f[A][i] + kd3 * Fa[i] * ga) - (2.0 / 3.0) * hc * n[A][i]);
            }
        }
    }
    for (int A = 0; A < 4; A++) {
#pragma unroll
        for (int i = 0; i < 3; i++) {
            // R_m = W sum_q rho_q N_qA (vdot - b)_i + V (mu/2 E0 + sum phi' E) - n Pbar  (Pbar: no theta)
            const double E0 = aJ * (2.0 * f[A][i] - (2.0 / 3.0) * I1 * n[A][i]);
            D4 rm = W * (QAB * xrv[i][A] + QB * Srv[i]) + (0.5 * V * E0) * mu;
            if (a.nfib) rm = rm + (V * fE[0][A][i]) * phi[0] + (V * fE[1][A][i]) * phi[1];
#pragma unroll
            for (int k = 0; k < 4; k++) grad[k] -= lm[A][i] * rm.d[k];
        }
        // R_p = W sum_q beta_q pdot_q N_qA + JV/4 div v + tau n_A . sigma
        const D4 ns = n[A][0] * sig[0] + n[A][1] * sig[1] + n[A][2] * sig[2];
        const D4 rp = W * (QAB * xb[A] + QB * Sb) + tau * ns;
#pragma unroll
        for (int k = 0; k < 4; k++) grad[k] -= lp[A] * rp.d[k];
    }
#pragma unroll
    for (int k = 0; k < 4; k++) a.grad[4 * e + k] += grad[k];
}

// ------------------------------------------------------------ vector kernels of the reverse step

struct RevArgs {
    int64_t N;
    const uint8_t *dir;
    double am, af, gam, dt, c1;
    const double *ybar, *ydbar;  // in [u|p|v], [udot|pdot|vdot] (7N)
    double *rt;                  // out reduced rhs [mu_v 3N | mu_p N]
    double *mu_u;                // out [3N]
};

// mu = U^{-T} g with g = ydbar + gam dt ybar; the reduced right-hand side
__global__ void k_rev_rhs(RevArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int64_t N = a.N;
    const unsigned d = a.dir[i];
    const double gdt = a.gam * a.dt;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const bool fixed = (d >> c) & 1u;
        const double gu = a.ydbar[3 * i + c] + gdt * a.ybar[3 * i + c];
        const double gv = a.ydbar[4 * N + 3 * i + c] + gdt * a.ybar[4 * N + 3 * i + c];
        const double mu = gu / a.am;
        a.mu_u[3 * i + c] = fixed ? 0.0 : mu;
        a.rt[3 * i + c] = fixed ? 0.0 : gv + a.c1 * mu;
    }
    a.rt[3 * N + i] = a.ydbar[3 * N + i] + gdt * a.ybar[3 * N + i];
}

struct RevUpd {
    int64_t N;
    const uint8_t *dir;
    double am, af, gam, dt, c1;
    const double *mu_u;   // [3N]
    const double *lam;    // reduced solution [lam_m 3N | lam_p N]
    const double *y1;     // (dR/dydot)^T lam: [v 3N | p N]   (weights 1,0,0)
    const double *y2;     // (dR/d(p,v))^T lam: [v 3N | p N] (weights 0,1,0)
    const double *y3;     // (dR/du)^T lam: [u 3N | 0]       (weights 0,0,1)
    double *ybar, *ydbar; // in/out
    double *lam_full;     // out [lam_k 3N | lam_p N | lam_m 3N]
};

__global__ void k_rev_update(RevUpd a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int64_t N = a.N;
    const unsigned d = a.dir[i];
    const double w_ydot = 1.0 - a.am, w_y = a.af * a.dt * (1.0 - a.gam), carry = a.dt * (1.0 - a.gam);
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const bool fixed = (d >> c) & 1u;
        const int64_t ku = 3 * i + c, kv = 4 * N + 3 * i + c;
        const double lk = fixed ? 0.0 : a.mu_u[ku] - (a.c1 / a.am) * a.y3[ku];
        const double lmv = fixed ? 0.0 : a.lam[ku];
        // F_y^T lam and F_ydot^T lam, components u and v (R_k bar = udot - v)
        const double Fy_u = fixed ? 0.0 : a.y3[ku];
        const double Fy_v = fixed ? 0.0 : a.y2[ku] - lk;
        const double Fd_u = lk;
        const double Fd_v = fixed ? 0.0 : a.y1[ku];
        const double yb_u = a.ybar[ku], yb_v = a.ybar[kv];
        a.ybar[ku] = fixed ? 0.0 : yb_u - Fy_u;
        a.ybar[kv] = fixed ? 0.0 : yb_v - Fy_v;
        a.ydbar[ku] = fixed ? 0.0 : carry * yb_u - w_ydot * Fd_u - w_y * Fy_u;
        a.ydbar[kv] = fixed ? 0.0 : carry * yb_v - w_ydot * Fd_v - w_y * Fy_v;
        a.lam_full[ku] = lk;
        a.lam_full[kv] = lmv;
    }
    const int64_t kp = 3 * N + i;
    const double Fy_p = a.y2[kp], Fd_p = a.y1[kp], yb_p = a.ybar[kp];
    a.ybar[kp] = yb_p - Fy_p;
    a.ydbar[kp] = carry * yb_p - w_ydot * Fd_p - w_y * Fy_p;
    a.lam_full[kp] = a.lam[3 * N + i];
}

__global__ void k_stage_from(const double *yn_u, const double *yn_p, const double *yn_v, const double *ydn_u,
                             const double *ydn_p, const double *ydn_v, const double *y1_u, const double *y1_p,
                             const double *y1_v, const double *yd1_u, const double *yd1_p, const double *yd1_v,
                             double *st, int64_t N, double am, double af) {
    // st: [u 3N | p N | v 3N | udot 3N | pdot N | vdot 3N] at the stage
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n7 = 7 * N;
    if (k < 3 * N) {
        st[k] = yn_u[k] + af * (y1_u[k] - yn_u[k]);
        st[4 * N + k] = yn_v[k] + af * (y1_v[k] - yn_v[k]);
        st[n7 + k] = ydn_u[k] + am * (yd1_u[k] - ydn_u[k]);
        st[n7 + 4 * N + k] = ydn_v[k] + am * (yd1_v[k] - ydn_v[k]);
    }
    if (k < N) {
        st[3 * N + k] = yn_p[k] + af * (y1_p[k] - yn_p[k]);
        st[n7 + 3 * N + k] = ydn_p[k] + am * (yd1_p[k] - ydn_p[k]);
    }
}

SensArgs sens_args(Ctx &c, const hyel_state &st, const double *lam, double *grad) {
    DeviceMesh &m = c.mesh;
    SensArgs a;
    a.tets = m.tets;
    a.geo = m.geo;
    a.mat = m.mat;
    a.fib = m.fib;
    a.dir = m.dir;
    a.E = m.E;
    a.N = m.N;
    a.vol = m.vol_model;
    a.nfib = m.n_fibres;
    a.rho0 = m.rho0;
    a.kd = m.kd;
    a.b0 = m.body[0];
    a.b1 = m.body[1];
    a.b2 = m.body[2];
    a.u = st.u;
    a.p = st.p;
    a.v = st.v;
    a.ud = st.udot;
    a.pd = st.pdot;
    a.vd = st.vdot;
    a.lam = lam;
    a.grad = grad;
    return a;
}

// RAII: swap the assembled blocks with their transpose for a transposed solve
struct TransposeSwap {
    Ctx &c;
    explicit TransposeSwap(Ctx &cc) : c(cc) {
        transpose_assembled(c);
        std::swap(c.mat.A, c.mat.At);
        std::swap(c.mat.B, c.mat.Bt);
        std::swap(c.mat.C, c.mat.Ct);
        std::swap(c.mat.D, c.mat.Dt);
        c.mat.scaled = false;
    }
    ~TransposeSwap() {
        std::swap(c.mat.A, c.mat.At);
        std::swap(c.mat.B, c.mat.Bt);
        std::swap(c.mat.C, c.mat.Ct);
        std::swap(c.mat.D, c.mat.Dt);
        c.mat.scaled = false;  // scaled copies now hold the transpose
    }
};

}  // namespace

void solve_nested_transpose(Ctx &c, const hyel_solver_params &p, const double *rhs, double *x,
                            hyel_solve_stats *st) {
    if (!c.mat.assembled) fail(HYEL_ESTATE, "solve_transpose: nothing assembled");
    TransposeSwap sw(c);
    solve_nested(c, p, rhs, x, st);
}

void spmv_transpose(Ctx &c, const double *x, double *y) {
    transpose_assembled(c);
    spmv_full64(c, c.mat.At, c.mat.Bt, c.mat.Ct, c.mat.Dt, x, y);
}

void param_sensitivity(Ctx &c, const hyel_state &st, const double *lam, double *grad) {
    if (c.mesh.N == 0) fail(HYEL_ESTATE, "param_sensitivity: no mesh");
    SensArgs a = sens_args(c, st, lam, grad);
    (k_param_sensitivity<<<blocks_for(c.mesh.E, 128), 128, 0, c.stream>>>(a), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
}

void adjoint_step(Ctx &c, const hyel_time_params &tp, const hyel_solver_params &sp, const hyel_state &sn,
                  const hyel_state &s1, double *ybar, double *ydbar, double *grad, double *lam_out,
                  hyel_solve_stats *stats) {
    DeviceMesh &m = c.mesh;
    if (m.N == 0) fail(HYEL_ESTATE, "adjoint_step: no mesh");
    const int64_t N = m.N, n7 = 7 * N;
    TimeConsts tc = time_consts(m, tp);
    double *st = c.vec + 4 * n7;  // stage values (14N), as in the Newton step
    double *rt = c.vec;           // [4N] reduced rhs
    double *lam = c.vec + 4 * N;  // [4N] reduced solution
    double *mu_u = c.vec + 8 * N; // [3N]
    double *y1 = c.vec + 11 * N;  // [4N] each
    double *y2 = c.vec + 15 * N;
    double *y3 = c.vec + 19 * N;
    double *lam_full = lam_out ? lam_out : c.vec + 6 * n7;  // [7N], after the stage values
    (k_stage_from<<<blocks_for(3 * N, 256), 256, 0, c.stream>>>(sn.u, sn.p, sn.v, sn.udot, sn.pdot, sn.vdot, s1.u,
                                                                s1.p, s1.v, s1.udot, s1.pdot, s1.vdot, st, N, tc.am,
                                                                tc.af),
     ::hyel::count_launch());
    hyel_state stage;
    stage.u = st;
    stage.p = st + 3 * N;
    stage.v = st + 4 * N;
    stage.udot = st + n7;
    stage.pdot = st + n7 + 3 * N;
    stage.vdot = st + n7 + 4 * N;
    // tangent at the converged stage, transposed solve
    assemble(c, tc, stage, nullptr, nullptr, nullptr);
    RevArgs ra;
    ra.N = N;
    ra.dir = m.dir;
    ra.am = tc.am;
    ra.af = tc.af;
    ra.gam = tc.gam;
    ra.dt = tc.dt;
    ra.c1 = tc.c1;
    ra.ybar = ybar;
    ra.ydbar = ydbar;
    ra.rt = rt;
    ra.mu_u = mu_u;
    (k_rev_rhs<<<blocks_for(N, 256), 256, 0, c.stream>>>(ra), ::hyel::count_launch());
    solve_nested_transpose(c, sp, rt, lam, stats);
    // partial Jacobians: unit-weight assemblies, transposed products
    double *outs[3] = {y1, y2, y3};
    const double w[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}};
    for (int k = 0; k < 3; k++) {
        TimeConsts tk = tc;
        tk.am = w[k][0];
        tk.c1 = w[k][1];
        tk.c2 = w[k][2];
        tk.literal = 1;  // no right-hand-side correction (it divides by am)
        assemble(c, tk, stage, nullptr, nullptr, nullptr);
        spmv_transpose(c, lam, outs[k]);
    }
    // parameter sensitivities use lam in the full [k | p | m] layout
    RevUpd ru;
    ru.N = N;
    ru.dir = m.dir;
    ru.am = tc.am;
    ru.af = tc.af;
    ru.gam = tc.gam;
    ru.dt = tc.dt;
    ru.c1 = tc.c1;
    ru.mu_u = mu_u;
    ru.lam = lam;
    ru.y1 = y1;
    ru.y2 = y2;
    ru.y3 = y3;
    ru.ybar = ybar;
    ru.ydbar = ydbar;
    ru.lam_full = lam_full;
    (k_rev_update<<<blocks_for(N, 256), 256, 0, c.stream>>>(ru), ::hyel::count_launch());
    if (grad) param_sensitivity(c, stage, lam_full, grad);
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaStreamSynchronize(c.stream));
    // the context's matrix now holds a partial Jacobian: require a new assembly
    c.mat.assembled = false;
}

}  // namespace hyel
