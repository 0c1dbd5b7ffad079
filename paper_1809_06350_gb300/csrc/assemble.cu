// Element assembly of the residual and the consistent tangent (Appendix A),
// with the deterministic slot gather into the SELL-32 block storage.
//
// One thread per element computes, in FP64, the residuals R_m, R_p of
// Appendix A and the 16 node-pair blocks of A, B, C, D (eq. def_matrix_A,
// def_matrix_D, entry formulas of Appendix A) and writes them to the element's
// staging records. A second kernel sums, for every block slot, the records of
// the elements sharing that node pair, in ascending element order (the same
// order on every run: results are bitwise reproducible), and applies the
// Dirichlet elimination. A third sums the nodal residuals.
//
// Exact-derivative readings (the paper's formulas are checked against the
// complex-step Jacobian of the residual by the test suite):
//   * the C-block term tau N_A,j N_B,i (rho J vdot_i + J p_,i - rho J b_i)
//     enters with a minus sign (d N_A,i / d u_Bj = -N_A,j N_B,i);
//   * "S~ delta_ij + A^iso" of the A block is the full derivative
//     d P~_iI / d F_jJ of P~ = d Psi_iso / d F;
//   * P1 elements: P~_iJ,J = 0 and N_B,MN = 0;
//   * every integral uses the 4-point rule (a,b,b,b), a = (5+3 sqrt5)/20,
//     b = (5-sqrt5)/20, weights V/4.
#include <cmath>

#include "internal.h"

namespace hyel {

namespace {

constexpr double QA = 0.58541019662496845446;  // (5 + 3 sqrt 5)/20
constexpr double QB = 0.13819660112501051518;  // (5 - sqrt 5)/20
constexpr double QAB = QA - QB;
constexpr double QAA_BB = QA * QA - QB * QB;
constexpr double QAB_BB = QA * QB - QB * QB;
constexpr double QBB = QB * QB;

struct ElemArgs {
    const int4 *tets;
    const double *geo, *mat, *fib;
    const uint8_t *dir;
    int64_t E;
    int vol;      // HYEL_VOL_*
    int nfib;     // 0 or 2
    int corr;     // compute the K_{.,udot} R_k correction
    double rho0, kd, b0, b1, b2;
    double am, c1, c2;
    const double *u, *p, *v, *ud, *pd, *vd;
    double *stage;
    unsigned *err;
};

__device__ __forceinline__ double *record(double *stage, int64_t e, int k) {
    return stage + ((((e >> 5) * kRecords + k) * 32 + (e & 31)) * kRecordDoubles);
}

__device__ __forceinline__ double qone(const double *X, double S, int A) { return QAB * X[A] + QB * S; }

// TAN: also the tangent blocks; CORR: also the K_{.,udot} R_k right-hand-side
// correction (record 17; zeros otherwise)
template <bool TAN, bool CORR>
__global__ void __launch_bounds__(128) k_element(ElemArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.E) return;
    const int64_t E = a.E;
    const int4 t4 = a.tets[e];
    const int nd[4] = {t4.x, t4.y, t4.z, t4.w};

    double g[4][3];
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int I = 0; I < 3; I++) g[A][I] = a.geo[(A * 3 + I) * E + e];
    const double V = a.geo[12 * E + e];
    const double tau = a.geo[13 * E + e];
    const double mu = a.mat[e];
    const double kappa = a.mat[E + e];

    // ---- gather the stage state
    double u[4][3], v[4][3], vdb[4][3], p[4], pd[4], rk[4][3];
    const double bf[3] = {a.b0, a.b1, a.b2};
#pragma unroll
    for (int A = 0; A < 4; A++) {
        const int64_t n = nd[A];
        const unsigned df = a.dir[n];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            u[A][i] = a.u[3 * n + i];
            v[A][i] = a.v[3 * n + i];
            vdb[A][i] = a.vd[3 * n + i] - bf[i];
            rk[A][i] = ((df >> i) & 1u) ? 0.0 : a.ud[3 * n + i] - v[A][i];
        }
        p[A] = a.p[n];
        pd[A] = a.pd[n];
    }

    // ---- kinematics: F = I + sum_A u_A (x) g_A, J, cof(F) = J F^-T
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
    if (!(J > 0.0)) {
        atomicOr(a.err, ERR_INVERTED);
        return;
    }
    const double iJ = 1.0 / J;
    // spatial gradients n[A][i] = N_A,i = g_AI F^-1_Ii = g_AI cof_iI / J; f = F g_A
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
    const double rJ = rcbrt(J);
    const double aJ = rJ * rJ;  // J^{-2/3} (one reciprocal cube root: fewer FP64 steps than cbrt and a division)

    // velocity and pressure gradients
    double Lv[3][3];  // v_i,j
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Lv[i][j] = v[0][i] * n[0][j] + v[1][i] * n[1][j] + v[2][i] * n[2][j] + v[3][i] * n[3][j];
    const double divv = Lv[0][0] + Lv[1][1] + Lv[2][2];
    double gp[3];
#pragma unroll
    for (int i = 0; i < 3; i++) gp[i] = p[0] * n[0][i] + p[1] * n[1][i] + p[2] * n[2][i] + p[3] * n[3][i];

    // ---- quadrature-point values; point q lies nearest node q
    // W = (V/4) J; X-arrays hold the value at the point nearest each node
    const double W = 0.25 * V * J;
    double xr[4], xb[4], xd[4], xrv[3][4], xrp[3][4];
    double Sp = 0.0;
    const double rk0 = a.rho0 / kappa;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const double pq = QAB * p[q] + QB * (p[0] + p[1] + p[2] + p[3]);
        const double pdq = QAB * pd[q] + QB * (pd[0] + pd[1] + pd[2] + pd[3]);
        Sp += pq;
        double rho, beta, rhop, betap;
        if (a.vol == HYEL_VOL_GIBBS) {
            // beta = 1 / sqrt(p^2 + kappa^2) by one reciprocal square root, s = (p^2 + kappa^2) beta
            const double s2 = fma(pq, pq, kappa * kappa);
            beta = rsqrt(s2);
            const double s = s2 * beta;
            rho = rk0 * (pq + s);
            rhop = rho * beta;
            betap = -pq * beta * beta * beta;
        } else {
            rho = a.rho0;
            beta = 0.0;
            rhop = 0.0;
            betap = 0.0;
        }
        xr[q] = rho;
        xb[q] = beta * pdq;
        xd[q] = a.am * beta + a.c1 * betap * pdq;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            const double vq = QAB * vdb[q][i] + QB * (vdb[0][i] + vdb[1][i] + vdb[2][i] + vdb[3][i]);
            xrv[i][q] = rho * vq;
            xrp[i][q] = rhop * vq;
        }
    }
    const double Sr = xr[0] + xr[1] + xr[2] + xr[3];
    const double Sb = xb[0] + xb[1] + xb[2] + xb[3];
    const double Sd = xd[0] + xd[1] + xd[2] + xd[3];
    double Srv[3], Srp[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Srv[i] = xrv[i][0] + xrv[i][1] + xrv[i][2] + xrv[i][3];
        Srp[i] = xrp[i][0] + xrp[i][1] + xrp[i][2] + xrp[i][3];
    }
    const double Pbar = W * Sp;                 // int J p
    const double JV = J * V, JV4 = 0.25 * J * V;
    // sigma_i = int rho J (vdot_i - b_i) + J V p_,i
    double sig[3];
#pragma unroll
    for (int i = 0; i < 3; i++) sig[i] = W * Srv[i] + JV * gp[i];

    // ---- isochoric stress: sum over structure terms of phi' E (NH: H = I, phi' = mu/2)
    // E[A][i] = J^{-2/3} (2 (F H g_A)_i - 2/3 (H:C) n_Ai)
    double E0[4][3], PgA[4][3];
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            E0[A][i] = aJ * (2.0 * f[A][i] - (2.0 / 3.0) * I1 * n[A][i]);
            PgA[A][i] = 0.5 * mu * E0[A][i];
        }
    // fibre data (HGO, §5.2)
    double fE[2][4][3], fFa[2][3], fga[2][4], fd1[2], fd2[2], fhc[2];
    const double k1 = a.nfib ? a.mat[2 * E + e] : 0.0;
    const double k2 = a.nfib ? a.mat[3 * E + e] : 1.0;
    const double kd = a.kd, kd3 = 1.0 - 3.0 * a.kd;
    if (a.nfib) {
#pragma unroll
        for (int tf = 0; tf < 2; tf++) {
            double av[3];
#pragma unroll
            for (int I = 0; I < 3; I++) av[I] = a.fib[(3 * tf + I) * E + e];
            double Fa2 = 0.0;
#pragma unroll
            for (int i = 0; i < 3; i++) {
                fFa[tf][i] = F[i][0] * av[0] + F[i][1] * av[1] + F[i][2] * av[2];
                Fa2 += fFa[tf][i] * fFa[tf][i];
            }
            const double hc = kd * I1 + kd3 * Fa2;  // H : C
            const double Eb = aJ * hc - 1.0;
            const double ex = exp(k2 * Eb * Eb);
            fd1[tf] = k1 * Eb * ex;                           // phi'
            fd2[tf] = k1 * (1.0 + 2.0 * k2 * Eb * Eb) * ex;   // phi''
            fhc[tf] = hc;
#pragma unroll
            for (int A = 0; A < 4; A++) {
                fga[tf][A] = g[A][0] * av[0] + g[A][1] * av[1] + g[A][2] * av[2];
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    const double FHg = kd * f[A][i] + kd3 * fFa[tf][i] * fga[tf][A];
                    fE[tf][A][i] = aJ * (2.0 * FHg - (2.0 / 3.0) * hc * n[A][i]);
                    PgA[A][i] += fd1[tf] * fE[tf][A][i];
                }
            }
        }
    }

    // ---- residuals (Appendix A): R_m = m + V P~ g - n Pbar; R_p = bp + JV/4 div v + tau n . sigma
    double ns[4];
    {
        double *rr = record(a.stage, e, 16);
#pragma unroll
        for (int A = 0; A < 4; A++) {
            ns[A] = n[A][0] * sig[0] + n[A][1] * sig[1] + n[A][2] * sig[2];
            double out[4];
#pragma unroll
            for (int i = 0; i < 3; i++) out[i] = W * qone(xrv[i], Srv[i], A) + V * PgA[A][i] - n[A][i] * Pbar;
            out[3] = W * qone(xb, Sb, A) + JV4 * divv + tau * ns[A];
            reinterpret_cast<double2 *>(rr)[2 * A] = make_double2(out[0], out[1]);
            reinterpret_cast<double2 *>(rr)[2 * A + 1] = make_double2(out[2], out[3]);
        }
    }
    if (!TAN) return;

    // ---- tangent. The weights c2 = (a_f g dt)^2/a_m, c1 = a_f g dt and a_m are
    // folded into per-element and per-node coefficients first, so that each
    // of the 16 node pairs costs about 70 FP64 operations.
    const double c1 = a.c1, c2 = a.c2, am = a.am;
    // A_u(A,B,i,j) = Q1_Ai n_Bj + Q2_Ai f_Bj + q3 n_Aj n_Bi + [i==j] q4 gg + fibre terms; here times c2
    double Q1[4][3], Q2[4][3];
    double q3 = V * mu * aJ * I1 / 3.0 + Pbar;
    const double q4 = c2 * V * mu * aJ;
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int i = 0; i < 3; i++) {
            Q1[A][i] = -V * (mu / 3.0) * E0[A][i] - Pbar * n[A][i] + W * qone(xrv[i], Srv[i], A);
            Q2[A][i] = c2 * (-V * (2.0 / 3.0) * mu * aJ * n[A][i]);
        }
    if (a.nfib) {
#pragma unroll
        for (int tf = 0; tf < 2; tf++) {
            q3 += V * (2.0 / 3.0) * fd1[tf] * aJ * fhc[tf];
#pragma unroll
            for (int A = 0; A < 4; A++)
#pragma unroll
                for (int i = 0; i < 3; i++) Q1[A][i] -= V * (2.0 / 3.0) * fd1[tf] * fE[tf][A][i];
        }
    }
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int i = 0; i < 3; i++) Q1[A][i] *= c2;
    q3 *= c2;
    // mass (a_m int rho J N_A N_B), B-block and D-block quadrature values, pre-weighted
    double xm[4], xpc[3][4], xdw[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        xm[q] = am * W * xr[q];
        xdw[q] = W * xd[q];
#pragma unroll
        for (int i = 0; i < 3; i++) xpc[i][q] = c1 * W * xrp[i][q];
    }
    const double Sm = am * W * Sr, Sdw = W * Sd;
    double Spc[3];
#pragma unroll
    for (int i = 0; i < 3; i++) Spc[i] = c1 * W * Srp[i];
    // pair integrals split per node: sum_q X_q N_qA N_qB = d[A] (A = B) or
    // o[A] + o[B] (A != B), with d = QAA_BB X + QBB S, o = QAB_BB X + QBB S / 2
    double dm[4], om[4], ddw[4], odw[4], dpc[3][4], opc[3][4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
        dm[q] = QAA_BB * xm[q] + QBB * Sm;
        om[q] = QAB_BB * xm[q] + 0.5 * QBB * Sm;
        ddw[q] = QAA_BB * xdw[q] + QBB * Sdw;
        odw[q] = QAB_BB * xdw[q] + 0.5 * QBB * Sdw;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            dpc[i][q] = QAA_BB * xpc[i][q] + QBB * Spc[i];
            opc[i][q] = QAB_BB * xpc[i][q] + 0.5 * QBB * Spc[i];
        }
    }
    const double jv4c1 = c1 * JV4;
    // C^j_AB = cAs_A n_Bj + cBs_B n_Aj - LvTnc_Bj - gpc_j nn
    //   cAs_A = c2 (W rb_A + JV/4 div v + tau n_A.sigma) + c1 JV/4,
    //   cBs_B = -c2 tau n_B.sigma + a_m tau int(rho J N_B), LvTnc = c2 JV/4 (grad v^T n), gpc = c2 tau J V p_,j
    // D_AB = int J (a_m beta + c1 beta_,p pdot) N_A N_B + c1 tau J V nn + n_A . qrc_B,
    //   qrc_B,i = c1 tau int J rho_,p (vdot_i - b_i) N_B
    double cA[4], cB[4], cAs[4], cBs[4], LvTn[4][3], qrc[4][3], gpc[3];
    const double c1tJV = c1 * tau * JV;
#pragma unroll
    for (int A = 0; A < 4; A++) {
        cA[A] = W * qone(xb, Sb, A) + JV4 * divv + tau * ns[A];
        cB[A] = -tau * ns[A];
        cAs[A] = c2 * cA[A] + c1 * JV4;
        cBs[A] = c2 * cB[A] + am * tau * W * qone(xr, Sr, A);
#pragma unroll
        for (int j = 0; j < 3; j++) {
            LvTn[A][j] = Lv[0][j] * n[A][0] + Lv[1][j] * n[A][1] + Lv[2][j] * n[A][2];
            qrc[A][j] = c1 * tau * W * qone(xrp[j], Srp[j], A);
        }
    }
#pragma unroll
    for (int j = 0; j < 3; j++) gpc[j] = c2 * tau * JV * gp[j];
    double w2c[2] = {0.0, 0.0}, w1c[2] = {0.0, 0.0}, w0c[2] = {0.0, 0.0};
    if (a.nfib) {
#pragma unroll
        for (int tf = 0; tf < 2; tf++) {
            w2c[tf] = c2 * V * fd2[tf];
            w1c[tf] = -c2 * V * (4.0 / 3.0) * fd1[tf] * aJ;
            w0c[tf] = c2 * 2.0 * V * fd1[tf] * aJ;
        }
    }
    double q3n[4][3];  // q3 n_A (times c2)
#pragma unroll
    for (int A = 0; A < 4; A++)
#pragma unroll
        for (int j = 0; j < 3; j++) q3n[A][j] = q3 * n[A][j];
    const double c2jv4 = c2 * JV4;
    // K_{.,udot} R_k: A_u R_k and C_u R_k, A_u = dR_m/du (the A block less its
    // mass part, over c2) and C_u = dR_p/du. Every part of A_u and C_u is a sum
    // of rank-one node-pair terms, so the products with R_k contract over the
    // second node once per element (s_n = sum_B n_B . R_B and the like) instead
    // of once per pair: C_u R_k here, c2 A_u R_k after the pair loop (fewer
    // values live through the loop).
    double cu[4] = {0.0, 0.0, 0.0, 0.0};
    if (CORR) {
        double sn = 0.0, sL = 0.0, cbr[3] = {0.0, 0.0, 0.0}, ngp[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int B = 0; B < 4; B++) {
            const double gr = gp[0] * rk[B][0] + gp[1] * rk[B][1] + gp[2] * rk[B][2];
#pragma unroll
            for (int j = 0; j < 3; j++) {
                sn = fma(n[B][j], rk[B][j], sn);
                sL = fma(LvTn[B][j], rk[B][j], sL);
                cbr[j] = fma(cB[B], rk[B][j], cbr[j]);
                ngp[j] = fma(n[B][j], gr, ngp[j]);
            }
        }
#pragma unroll
        for (int A = 0; A < 4; A++)
            cu[A] = fma(cA[A], sn, n[A][0] * cbr[0] + n[A][1] * cbr[1] + n[A][2] * cbr[2]) - JV4 * sL -
                    tau * JV * (n[A][0] * ngp[0] + n[A][1] * ngp[1] + n[A][2] * ngp[2]);
    }

    // the pair loop's C block takes -c2 JV/4 (grad v^T n_B) as its addend
#pragma unroll
    for (int B = 0; B < 4; B++)
#pragma unroll
        for (int j = 0; j < 3; j++) LvTn[B][j] *= -c2jv4;

#pragma unroll 1
    for (int A = 0; A < 4; A++) {
        // B block of the pairs (A, B): db_i (B = A), ub_i + opc_iB (B != A)
        double ubA[3], dbA[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            ubA[i] = fma(-jv4c1, n[A][i], opc[i][A]);
            dbA[i] = fma(-jv4c1, n[A][i], dpc[i][A]);
        }
#pragma unroll
        for (int B = 0; B < 4; B++) {
            double out[16];
            const double gg = g[A][0] * g[B][0] + g[A][1] * g[B][1] + g[A][2] * g[B][2];
            const double nn = n[A][0] * n[B][0] + n[A][1] * n[B][1] + n[A][2] * n[B][2];
            // A block: c2 A_u + a_m (mass) on the diagonal (the diagonal terms
            // are the innermost addend of the entry's multiply-add chain)
            const bool same = A == B;
            const double mass = same ? dm[A] : om[A] + om[B];
            const double dg = fma(q4, gg, mass);
#pragma unroll
            for (int i = 0; i < 3; i++)
#pragma unroll
                for (int j = 0; j < 3; j++) {
                    const double s0 = i == j ? fma(q3n[A][j], n[B][i], dg) : q3n[A][j] * n[B][i];
                    out[3 * i + j] = fma(Q1[A][i], n[B][j], fma(Q2[A][i], f[B][j], s0));
                }
            if (a.nfib) {
#pragma unroll
                for (int tf = 0; tf < 2; tf++) {
                    const double gHg = kd * gg + kd3 * fga[tf][A] * fga[tf][B];
                    const double d0 = w0c[tf] * gHg;
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        const double e2 = w2c[tf] * fE[tf][A][i], e1 = w1c[tf] * n[A][i];
#pragma unroll
                        for (int j = 0; j < 3; j++) {
                            const double FHgB = kd * f[B][j] + kd3 * fFa[tf][j] * fga[tf][B];
                            out[3 * i + j] += e2 * fE[tf][B][j] + e1 * FHgB + (i == j ? d0 : 0.0);
                        }
                    }
                }
            }
            // B^i_AB = c1 (int rho_,p J (vdot_i - b_i) N_A N_B - J N_A,i V/4)
#pragma unroll
            for (int i = 0; i < 3; i++) out[9 + i] = same ? dbA[i] : ubA[i] + opc[i][B];
#pragma unroll
            for (int j = 0; j < 3; j++)
                out[12 + j] = fma(cAs[A], n[B][j], fma(cBs[B], n[A][j], fma(-gpc[j], nn, LvTn[B][j])));
            const double md = same ? ddw[A] : odw[A] + odw[B];
            out[15] = fma(n[A][0], qrc[B][0], fma(n[A][1], qrc[B][1], fma(n[A][2], qrc[B][2], fma(c1tJV, nn, md))));
            double2 *rec = reinterpret_cast<double2 *>(record(a.stage, e, 4 * A + B));
#pragma unroll
            for (int k = 0; k < 8; k++) rec[k] = make_double2(out[2 * k], out[2 * k + 1]);
        }
    }
    // A_u = dR_m/du and C_u = dR_p/du; since K_{.,udot} = c1 d(.)/du,
    // (1/a_m) K_{.,udot} R_k = (c1/a_m) [A_u ; C_u] R_k, c2 A_u R_k formed
    // below (c2 > 0 whenever the correction is formed: dt > 0).
    double2 *rc = reinterpret_cast<double2 *>(record(a.stage, e, 17));
    if (CORR) {
        double sn = 0.0, sf = 0.0, Gn[3][3], Rg[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) Gn[i][j] = Rg[i][j] = 0.0;
#pragma unroll
        for (int B = 0; B < 4; B++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                sn = fma(n[B][j], rk[B][j], sn);
                sf = fma(f[B][j], rk[B][j], sf);
#pragma unroll
                for (int i = 0; i < 3; i++) {
                    Gn[i][j] = fma(n[B][i], rk[B][j], Gn[i][j]);  // sum_B n_Bi R_Bj
                    Rg[i][j] = fma(rk[B][i], g[B][j], Rg[i][j]);  // sum_B R_Bi g_Bj
                }
            }
        double sfe[2] = {0.0, 0.0}, sfa[2] = {0.0, 0.0}, tfa[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
        if (a.nfib) {
#pragma unroll
            for (int tf = 0; tf < 2; tf++)
#pragma unroll
                for (int B = 0; B < 4; B++) {
                    const double far = fFa[tf][0] * rk[B][0] + fFa[tf][1] * rk[B][1] + fFa[tf][2] * rk[B][2];
                    sfa[tf] = fma(fga[tf][B], far, sfa[tf]);
#pragma unroll
                    for (int i = 0; i < 3; i++) {
                        sfe[tf] = fma(fE[tf][B][i], rk[B][i], sfe[tf]);
                        tfa[tf][i] = fma(fga[tf][B], rk[B][i], tfa[tf][i]);
                    }
                }
        }
        const double su = c1 / (am * c2), sp = c1 / am;
#pragma unroll
        for (int A = 0; A < 4; A++) {
            double cv[3];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const double gnA = Gn[i][0] * n[A][0] + Gn[i][1] * n[A][1] + Gn[i][2] * n[A][2];
                const double rgA = Rg[i][0] * g[A][0] + Rg[i][1] * g[A][1] + Rg[i][2] * g[A][2];
                double s = fma(Q1[A][i], sn, fma(Q2[A][i], sf, fma(q3, gnA, q4 * rgA)));
                if (a.nfib) {
#pragma unroll
                    for (int tf = 0; tf < 2; tf++)
                        s += w2c[tf] * fE[tf][A][i] * sfe[tf] + w1c[tf] * n[A][i] * (kd * sf + kd3 * sfa[tf]) +
                             w0c[tf] * (kd * rgA + kd3 * fga[tf][A] * tfa[tf][i]);
                }
                cv[i] = su * s;
            }
            rc[2 * A] = make_double2(cv[0], cv[1]);
            rc[2 * A + 1] = make_double2(cv[2], sp * cu[A]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < 8; k++) rc[k] = make_double2(0.0, 0.0);
    }
}

// ---- slot gather: sum the staged pair blocks into the SELL-32 matrix, with
// Dirichlet rows/columns of constrained velocity components set to identity.
struct GatherArgs {
    const int32_t *col_slice, *slice_ptr, *row_len, *col, *slot_ptr, *slot_list;
    const uint8_t *dir;
    const double *stage;
    double *A, *B, *C, *D;
    int64_t N, nslots;
};

// Eight lanes per slot: lane l sums components 2l and 2l+1 of the slot's
// records (one 16-byte load per record), so one warp-wide load reads four
// whole 128-byte records; every lane adds in ascending element order.
__global__ void __launch_bounds__(256) k_gather(GatherArgs g) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t q = gt >> 3;
    const int l = (int)(gt & 7);
    if (q >= g.nslots) return;
    const int64_t b = q >> 5;
    const int t = (int)(q & 31);
    const int s = g.col_slice[b];
    const int64_t r = (int64_t)s * 32 + t;
    if (r >= g.N) return;
    if (b - g.slice_ptr[s] >= g.row_len[r]) return;  // padding stays zero
    double a0 = 0.0, a1 = 0.0;
    const int k0 = g.slot_ptr[q], k1 = g.slot_ptr[q + 1];
    for (int k = k0; k < k1; k++) {
        const int rec = __ldg(g.slot_list + k);
        const int64_t e = rec / kRecords;
        const int kk = rec - (int)e * kRecords;
        const double2 v = __ldg(reinterpret_cast<const double2 *>(
                                    g.stage + ((((e >> 5) * kRecords + kk) * 32 + (e & 31)) * kRecordDoubles)) +
                                l);
        a0 += v.x;
        a1 += v.y;
    }
    const int c = g.col[q];
    const unsigned dr = g.dir[r], dc = g.dir[c];
    const double val[2] = {a0, a1};
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int comp = 2 * l + h;  // 0..8 A (row-major), 9..11 B, 12..14 C, 15 D
        if (comp < 9) {
            const int i = comp / 3, j = comp % 3;
            double v = val[h];
            if (((dr >> i) & 1u) || ((dc >> j) & 1u)) v = (r == c && i == j) ? 1.0 : 0.0;
            g.A[(b * 9 + comp) * 32 + t] = v;
        } else if (comp < 12) {
            const int i = comp - 9;
            g.B[(b * 3 + i) * 32 + t] = ((dr >> i) & 1u) ? 0.0 : val[h];
        } else if (comp < 15) {
            const int i = comp - 12;
            g.C[(b * 3 + i) * 32 + t] = ((dc >> i) & 1u) ? 0.0 : val[h];
        } else {
            g.D[b * 32 + t] = val[h];
        }
    }
}

// ---- nodal residual gather, traction, Dirichlet, rhs and squared norms
struct ResArgs {
    const int32_t *node_ptr, *node_list;
    const uint8_t *dir;
    const double *stage, *trac, *ud, *v;
    double load;
    int64_t N;
    int literal;
    int use_g;           // add the K_{.,udot} R_k records (record 17) to the rhs
    double *res_out, *rhs_out;
    double *partial;     // [gridDim.x][3]
    unsigned *counter;
    double *norms;       // [4] final: total, Rk, Rp, Rm (sqrt applied)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Four lanes per node (kResLanes): lane k sums the node's element records
// k, k + 4, ...; the four partial sums meet by shuffles in a fixed order, so
// the result is the same on every run. (One thread per node left a chain of
// about 24 dependent record loads per thread.)
constexpr int kResLanes = 4;
constexpr int kResThreads = 1024;  // 256 nodes per block

__global__ void __launch_bounds__(kResThreads) k_residual(ResArgs a) {
    __shared__ double sm[kResThreads / 32][3];
    __shared__ bool last;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = g / kResLanes;
    const int lane = (int)(g % kResLanes);
    const bool live = i < a.N;
    double sk = 0.0, sp = 0.0, sr = 0.0;
    double R[4] = {0, 0, 0, 0}, G[4] = {0, 0, 0, 0};
    if (live) {
        for (int k = a.node_ptr[i] + lane; k < a.node_ptr[i + 1]; k += kResLanes) {
            const int ent = a.node_list[k];
            const int64_t e = ent >> 2;
            const int A = ent & 3;
            const double *r16 = a.stage + ((((e >> 5) * kRecords + 16) * 32 + (e & 31)) * kRecordDoubles) + 4 * A;
            const double *r17 = a.stage + ((((e >> 5) * kRecords + 17) * 32 + (e & 31)) * kRecordDoubles) + 4 * A;
#pragma unroll
            for (int m = 0; m < 4; m++) R[m] += r16[m];
            if (a.use_g)
#pragma unroll
                for (int m = 0; m < 4; m++) G[m] += r17[m];
        }
    }
#pragma unroll
    for (int o = 1; o < kResLanes; o <<= 1)
#pragma unroll
        for (int m = 0; m < 4; m++) {
            R[m] += __shfl_xor_sync(0xffffffffu, R[m], o);
            G[m] += __shfl_xor_sync(0xffffffffu, G[m], o);
        }
    if (live && lane == 0) {
        const unsigned d = a.dir[i];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            R[c] -= a.load * a.trac[3 * i + c];
            const bool fixed = (d >> c) & 1u;
            const double rm = fixed ? 0.0 : R[c];
            const double rkc = fixed ? 0.0 : a.ud[3 * i + c] - a.v[3 * i + c];
            if (a.res_out) a.res_out[3 * i + c] = rm;
            if (a.rhs_out) a.rhs_out[3 * i + c] = fixed ? 0.0 : -(R[c] - (a.literal ? 0.0 : G[c]));
            sr += rm * rm;
            sk += rkc * rkc;
        }
        if (a.res_out) a.res_out[3 * a.N + i] = R[3];
        if (a.rhs_out) a.rhs_out[3 * a.N + i] = -(R[3] - (a.literal ? 0.0 : G[3]));
        sp = R[3] * R[3];
    }
    sk = warp_sum(sk);
    sp = warp_sum(sp);
    sr = warp_sum(sr);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sm[w][0] = sk;
        sm[w][1] = sp;
        sm[w][2] = sr;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += sm[k][threadIdx.x];
        a.partial[3 * blockIdx.x + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) {
        __threadfence();
        // warps 0..2 each sum one quantity over the block partials (fixed order)
        if (w < 3) {
            double s = 0.0;
            for (unsigned k = l; k < gridDim.x; k += 32) s += ((volatile double *)a.partial)[3 * k + w];
            s = warp_sum(s);
            if (l == 0) sm[0][w] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            a.norms[0] = sqrt(sm[0][0] + sm[0][1] + sm[0][2]);
            a.norms[1] = sqrt(sm[0][0]);
            a.norms[2] = sqrt(sm[0][1]);
            a.norms[3] = sqrt(sm[0][2]);
            *a.counter = 0u;
        }
    }
}

}  // namespace

TimeConsts time_consts(const DeviceMesh &m, const hyel_time_params &tp) {
    if (!(tp.rho_inf >= 0.0 && tp.rho_inf <= 1.0)) fail(HYEL_EINVAL, "time params: rho_inf must be in [0, 1]");
    if (!(tp.dt > 0.0)) fail(HYEL_EINVAL, "time params: dt must be > 0");
    TimeConsts tc;
    tc.am = 0.5 * (3.0 - tp.rho_inf) / (1.0 + tp.rho_inf);
    tc.af = 1.0 / (1.0 + tp.rho_inf);
    tc.gam = tc.af;
    tc.dt = tp.dt;
    tc.c1 = tc.af * tc.gam * tp.dt;
    tc.c2 = tc.c1 * tc.c1 / tc.am;
    tc.t_alpha = tp.t_n + tc.af * tp.dt;
    tc.load = std::fmin(tc.t_alpha / m.t_ramp, 1.0);
    tc.literal = tp.rhs_literal;
    return tc;
}

void assemble(Ctx &c, const TimeConsts &tc, const hyel_state &st, double *res_out, double *rhs_out, double *norms4,
              bool tangent) {
    DeviceMesh &m = c.mesh;
    if (m.N == 0) fail(HYEL_ESTATE, "assemble: no mesh uploaded");
    if (!tangent && rhs_out) fail(HYEL_EINVAL, "assemble: a right-hand side needs the tangent pass");
    ElemArgs a;
    a.tets = m.tets;
    a.geo = m.geo;
    a.mat = m.mat;
    a.fib = m.fib;
    a.dir = m.dir;
    a.E = m.E;
    a.vol = m.vol_model;
    a.nfib = m.n_fibres;
    a.corr = (tc.literal || tc.skip_corr || !tangent) ? 0 : 1;
    a.rho0 = m.rho0;
    a.kd = m.kd;
    a.b0 = m.body[0];
    a.b1 = m.body[1];
    a.b2 = m.body[2];
    a.am = tc.am;
    a.c1 = tc.c1;
    a.c2 = tc.c2;
    a.u = st.u;
    a.p = st.p;
    a.v = st.v;
    a.ud = st.udot;
    a.pd = st.pdot;
    a.vd = st.vdot;
    a.stage = c.stage;
    a.err = c.err;
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    cudaEvent_t ev;
    const int cls = !tangent ? HYEL_K_ASSEMBLE_RES : a.corr ? HYEL_K_ASSEMBLE_CORR : HYEL_K_ASSEMBLE;
    prof_begin(c, cls, &ev);
    if (!tangent)
        (k_element<false, false><<<blocks_for(m.E, 128), 128, 0, c.stream>>>(a), ::hyel::count_launch());
    else if (a.corr)
        (k_element<true, true><<<blocks_for(m.E, 128), 128, 0, c.stream>>>(a), ::hyel::count_launch());
    else
        (k_element<true, false><<<blocks_for(m.E, 128), 128, 0, c.stream>>>(a), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    // algorithmic bytes: element geometry+material (18 doubles), 4 nodes x 17 state doubles, staging writes
    prof_end(c, cls, ev,
             (double)m.E * (8.0 * 18 + 16 + 4 * 8.0 * 17 + 8.0 * (tangent ? kRecords : 1) * kRecordDoubles));

    if (tangent) {
        GatherArgs g;
        g.col_slice = m.col_slice;
        g.slice_ptr = m.slice_ptr;
        g.row_len = m.row_len;
        g.col = m.col;
        g.slot_ptr = m.slot_ptr;
        g.slot_list = m.slot_list;
        g.dir = m.dir;
        g.stage = c.stage;
        g.A = c.mat.A;
        g.B = c.mat.B;
        g.C = c.mat.C;
        g.D = c.mat.D;
        g.N = m.N;
        g.nslots = m.nslots;
        prof_begin(c, HYEL_K_GATHER, &ev);
        (k_gather<<<blocks_for(8 * m.nslots, 256), 256, 0, c.stream>>>(g), ::hyel::count_launch());
        HYEL_CK(cudaGetLastError());
        prof_end(c, HYEL_K_GATHER, ev, (double)m.E * 16 * (128.0 + 4.0) + (double)m.nnzb * 128.0);
    }

    ResArgs r;
    r.node_ptr = m.node_ptr;
    r.node_list = m.node_list;
    r.dir = m.dir;
    r.stage = c.stage;
    r.trac = m.trac;
    r.ud = st.udot;
    r.v = st.v;
    r.load = tc.load;
    r.N = m.N;
    r.literal = tc.literal;
    r.res_out = res_out;
    r.rhs_out = rhs_out;
    // kResLanes lanes per node, 256 nodes per block: the partials of at most
    // (65536 - 64) / 3 blocks fit the context's reduction buffer
    int nb = blocks_for(m.N, kResThreads / kResLanes);
    r.partial = c.red + 64;
    r.counter = c.counter;
    r.norms = c.red;
    r.use_g = (rhs_out && !tc.literal) ? 1 : 0;
    (k_residual<<<nb, kResThreads, 0, c.stream>>>(r), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    if (tangent) {
        c.mat.assembled = true;
        c.mat.scaled = false;
        c.mat.transposed = false;
    }
    HYEL_CK(cudaMemcpyAsync(c.h_red, c.red, 4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & ERR_INVERTED) {
        c.mat.assembled = false;
        fail(HYEL_EINVERTED, "assemble: an element has J <= 0");
    }
    if (norms4)
        for (int k = 0; k < 4; k++) norms4[k] = c.h_red[k];
    if (!std::isfinite(c.h_red[0])) fail(HYEL_ENAN, "assemble: residual norm is not finite");
}

void matrix_download(Ctx &c, int32_t *row_ptr, int32_t *col, double *A, double *B, double *C, double *D) {
    DeviceMesh &m = c.mesh;
    if (m.N == 0) fail(HYEL_ESTATE, "matrix_download: no mesh");
    if (row_ptr) std::copy(m.h_row_ptr.begin(), m.h_row_ptr.end(), row_ptr);
    if (col) std::copy(m.h_col.begin(), m.h_col.end(), col);
    if (!A && !B && !C && !D) return;
    if (!c.mat.assembled) fail(HYEL_ESTATE, "matrix_download: nothing assembled");
    size_t ns = (size_t)m.nslots;
    std::vector<double> hA(A ? 9 * ns : 0), hB(B ? 3 * ns : 0), hC(C ? 3 * ns : 0), hD(D ? ns : 0);
    if (A) HYEL_CK(cudaMemcpyAsync(hA.data(), c.mat.A, 9 * ns * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (B) HYEL_CK(cudaMemcpyAsync(hB.data(), c.mat.B, 3 * ns * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (C) HYEL_CK(cudaMemcpyAsync(hC.data(), c.mat.C, 3 * ns * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    if (D) HYEL_CK(cudaMemcpyAsync(hD.data(), c.mat.D, ns * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    for (int64_t k = 0; k < m.nnzb; k++) {
        const int64_t q = m.h_csr_slot[k];
        const int64_t b = q >> 5, t = q & 31;
        if (A)
            for (int e = 0; e < 9; e++) A[9 * k + e] = hA[(b * 9 + e) * 32 + t];
        if (B)
            for (int e = 0; e < 3; e++) B[3 * k + e] = hB[(b * 3 + e) * 32 + t];
        if (C)
            for (int e = 0; e < 3; e++) C[3 * k + e] = hC[(b * 3 + e) * 32 + t];
        if (D) D[k] = hD[b * 32 + t];
    }
}

}  // namespace hyel
