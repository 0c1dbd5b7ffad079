// Smoothed-aggregation multigrid for the A-solves, with the rigid-body modes
// of 3-D elasticity in the coarse space. The paper applies A^-1 through
// algebraic multigrid (§4.4, §5); this is a GPU-native stand-in for BoomerAMG.
//
// * Hierarchy pattern, once per mesh, on the host. Level 0 is the mesh's
//   block pattern: one 3x3 block-node per mesh node. Super-nodes (the mesh
//   nodes on level 0, the aggregates of the finer level on the others) are
//   aggregated greedily: a super-node and all its free neighbours form an
//   aggregate, and leftovers join a neighbouring aggregate. Every aggregate K
//   gets two coarse block-nodes. 2K is the translation t_K. 2K + 1 is the
//   rotation, scaled as l_K omega_K, where l_K is the RMS distance of the
//   members from their centroid c_K. So every level keeps 3x3 blocks in the
//   SELL-32 layout.
// * Tentative prolongator P0 (the rigid-body modes). A mesh node i of K moves
//   by t_K + omega_K x (X_i - c_K). On coarser levels a member I of K takes
//   t_I = t_K + omega_K x (c_I - c_K) and omega_I = omega_K. On level 0 the
//   rows are scaled by W^-1, because the modes of the scaled A~ = W A W are
//   W^-1 times those of A. They are zero for constrained velocity components.
// * Smoothed prolongator P = (I - w_P D^-1 A_l) P0, with D the 3x3 block
//   diagonal of A_l and w_P = 4 / (3 lambda). lambda bounds the spectral
//   radius of D^-1 A_l: 15 power steps, times 1.1. The Galerkin operator
//   A_{l+1} = P^T A_l P is formed as Q = A_l P, then P^T Q. Every sum runs
//   over a fixed list in ascending order, so results are bitwise
//   reproducible. These numeric parts run on the GPU after every scaling of a
//   new assembly.
// * Coarsest level, at most kDenseMax block-nodes: a dense inverse by
//   Gauss-Jordan elimination with partial pivoting, in one thread block. A
//   coarse unknown whose row and column vanish (a rigid mode that the
//   constraints remove entirely) gets a unit diagonal and stays zero.
// * Application: one V-cycle in FP32 (for FP64 and FP32 levels alike). A
//   degree-kSmoothDegree Chebyshev smoother on [lambda / kSmoothRatio, lambda]
//   runs before and after the coarse correction. Coarse-level products use 8
//   lanes per row, or a warp on small levels; restrictions and the dense
//   apply use a warp per row (their rows are long and few). The V-cycle is a fixed linear operator, used as the right
//   preconditioner of the A-level (F)GMRES.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace hyel {

namespace {

constexpr int64_t kDenseMax = 96;  // block-nodes of a coarsest level solved by its dense inverse
constexpr int kMaxLevels = 10;
constexpr int kSmoothDegree = 3;    // Chebyshev smoother before and after the coarse correction
constexpr double kSmoothRatio = 30.0;  // its interval [lambda / kSmoothRatio, lambda]
constexpr int kCoarseDegree = 12;   // the smoother alone on a coarsest level above kDenseMax (coarsening stalled)
constexpr int kPowerSteps = 15;
constexpr double kLamMargin = 1.1;
constexpr int kGjThreads = 256;
constexpr int64_t kWarpRowsBelow = 8192;  // coarse levels with fewer block-nodes use a warp per row, others 8 lanes

struct SellHost {
    std::vector<int32_t> slice_ptr, row_len, col, diag_slot, col_slice;
    int64_t nslots = 0, ncols = 0;
};

SellHost build_sell(int64_t N, const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &cols) {
    SellHost s;
    const int64_t ns = (N + 31) / 32;
    s.slice_ptr.assign(ns + 1, 0);
    s.row_len.assign(N, 0);
    for (int64_t sl = 0; sl < ns; sl++) {
        int32_t len = 0;
        for (int t = 0; t < 32; t++) {
            const int64_t r = sl * 32 + t;
            if (r < N) len = std::max(len, row_ptr[r + 1] - row_ptr[r]);
        }
        s.slice_ptr[sl + 1] = s.slice_ptr[sl] + len;
    }
    s.ncols = s.slice_ptr[ns];
    s.nslots = s.ncols * 32;
    if (s.nslots >= ((int64_t)1 << 31) / 9) fail(HYEL_EINVAL, "amg: coarse pattern too large");
    s.col.assign(s.nslots, 0);
    s.col_slice.assign(s.ncols, 0);
    for (int64_t sl = 0; sl < ns; sl++)
        for (int32_t b = s.slice_ptr[sl]; b < s.slice_ptr[sl + 1]; b++) s.col_slice[b] = (int32_t)sl;
    s.diag_slot.assign(N, -1);
    for (int64_t r = 0; r < N; r++) {
        const int32_t len = row_ptr[r + 1] - row_ptr[r];
        s.row_len[r] = len;
        const int32_t slen = s.slice_ptr[(r >> 5) + 1] - s.slice_ptr[r >> 5];
        for (int32_t j = 0; j < slen; j++) {
            const int64_t q = ((int64_t)s.slice_ptr[r >> 5] + j) * 32 + (r & 31);
            s.col[q] = j < len ? cols[row_ptr[r] + j] : (int32_t)r;
            if (j < len && cols[row_ptr[r] + j] == r) s.diag_slot[r] = (int32_t)q;
        }
        if (s.diag_slot[r] < 0) fail(HYEL_EINVAL, "amg: a block row without its diagonal");
    }
    return s;
}

struct Level {
    int64_t N = 0, nslots = 0;  // block-nodes (3 unknowns each), SELL slots
    // SELL-32 pattern (device); level 0 borrows the mesh's arrays
    const int32_t *slice_ptr = nullptr, *row_len = nullptr, *col = nullptr, *diag_slot = nullptr;
    int32_t *col_slice = nullptr;  // coarse levels: slice owning each slice column
    // values: level 0 borrows the scaled matrix and its block inverses
    double *A64 = nullptr, *jac64 = nullptr;
    float *A32 = nullptr, *jac32 = nullptr;
    double *lam = nullptr;  // device [1]: kLamMargin x the power estimate of the spectral radius of D^-1 A_l
    // transfer to the next coarser level (every level but the coarsest)
    int64_t nnzP = 0, nnzQ = 0;
    int32_t *agg = nullptr;   // [N] coarse aggregate of each block-node
    double *tent = nullptr;   // [N][18] P0 blocks: translation T then rotation R, row-major
    int32_t *p_ptr = nullptr, *p_col = nullptr, *p_row = nullptr;  // CSR of P, columns ascending
    double *P64 = nullptr;    // [nnzP][9] row-major
    float *P32 = nullptr;
    int32_t *pt_ptr = nullptr, *pt_row = nullptr, *pt_slot = nullptr;  // per coarse block-node: (row, P entry)
    int32_t *q_ptr = nullptr, *q_col = nullptr, *q_row = nullptr;      // CSR of Q = A_l P
    double *Q64 = nullptr;    // [nnzQ][9]
    // coarsest level with N <= kDenseMax: dense matrix and its inverse,
    // row-major (dinv[i n + j] = A^-1(i, j), n = 3N; FP64 in dwork64)
    double *dense64 = nullptr, *dwork64 = nullptr;
    float *dinv32 = nullptr;
    // FP32 work vectors of the V-cycle [3N]: right-hand side, iterate, residual;
    // two smoother directions [2][3N]; an FP64 [3N] pair for the power steps
    float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *e32 = nullptr;
    double *x64 = nullptr, *r64 = nullptr;
    int64_t nnzb = 0;  // stored blocks (valid entries)
    int lanes = 1;     // lanes per row of this level's products: 1 on level 0, 8 or 32 on coarse levels (long rows)
};

}  // namespace

struct Amg {
    std::vector<Level> lv;
    double *partial = nullptr;  // power-step partial sums, one per 128-thread block of level 0
    double *pscale = nullptr;   // device [1]: 1 / norm of the current power iterate
    bool numeric_ok = false;
};

namespace {

template <typename T>
T *up(Ctx &c, const std::vector<T> &h) {
    T *d = dalloc_n<T>(c, std::max<size_t>(1, h.size()));
    if (!h.empty()) HYEL_CK(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, c.stream));
    return d;
}

// ---------------------------------------------------------------- kernels

// block of a SELL level at slot q, row-major
__device__ __forceinline__ void sell_block(const double *A, int64_t q, double M[9]) {
    const double *Ab = A + (q >> 5) * 288 + (q & 31);
#pragma unroll
    for (int k = 0; k < 9; k++) M[k] = Ab[32 * k];
}

// C += A B and C += A^T B for row-major 3x3 blocks
__device__ __forceinline__ void mm_add(const double *A, const double *B, double *C) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double s = C[3 * i + j];
#pragma unroll
            for (int m = 0; m < 3; m++) s = fma(A[3 * i + m], B[3 * m + j], s);
            C[3 * i + j] = s;
        }
}
__device__ __forceinline__ void mtm_add(const double *A, const double *B, double *C) {
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            double s = C[3 * i + j];
#pragma unroll
            for (int m = 0; m < 3; m++) s = fma(A[3 * m + i], B[3 * m + j], s);
            C[3 * i + j] = s;
        }
}

// position of key in the ascending cols[lo, hi), or -1
__device__ __forceinline__ int find_col(const int32_t *cols, int lo, int hi, int32_t key) {
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const int32_t v = cols[mid];
        if (v == key) return mid;
        if (v < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return -1;
}

struct SaArgs {
    const int32_t *slice_ptr, *row_len, *col;  // SELL pattern of A_l
    const double *A;                           // A_l
    const double *jac;                         // [9][N] inverses of its diagonal blocks
    const int32_t *agg;                        // [N]
    const double *tent;                        // [N][18]
    const double *w;                           // level 0: the velocity scaling [3N]; nullptr otherwise
    const uint8_t *dir;                        // level 0: constrained-component bits [N]
    const double *lam;
    const int32_t *p_ptr, *p_col, *p_row;
    double *P64;
    float *P32;
    const int32_t *q_ptr, *q_col, *q_row;
    double *Q64;
    int64_t N, nnzP, nnzQ;
};

// P0 block of block-node b for the translation (which = 0) or rotation (1)
// column of its aggregate; on level 0 scaled by W^-1, zero rows for
// constrained components
__device__ __forceinline__ void tent_block(const SaArgs &a, int64_t b, int which, double X[9]) {
    const double *t = a.tent + b * 18 + 9 * which;
#pragma unroll
    for (int k = 0; k < 9; k++) X[k] = t[k];
    if (a.w) {
        const unsigned df = a.dir[b];
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const double s = ((df >> r) & 1u) ? 0.0 : 1.0 / a.w[3 * b + r];
#pragma unroll
            for (int k = 0; k < 3; k++) X[3 * r + k] *= s;
        }
    }
}

// P(r, J) = [agg(r) = K] P0(r, J) - w_P D_r^-1 sum_{b in row r, agg(b) = K} A_rb P0(b, J), K = J / 2
__global__ void __launch_bounds__(128) k_sa_prolongator(SaArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nnzP) return;
    const int64_t r = a.p_row[p];
    const int32_t J = a.p_col[p], K = J >> 1;
    const int which = J & 1;
    double S[9];
#pragma unroll
    for (int k = 0; k < 9; k++) S[k] = 0.0;
    const int t = (int)(r & 31);
    const int64_t b0 = a.slice_ptr[r >> 5];
    const int len = a.row_len[r];
    for (int j = 0; j < len; j++) {
        const int64_t q = (b0 + j) * 32 + t;
        const int64_t cb = a.col[q];
        if (a.agg[cb] != K) continue;
        double M[9], X[9];
        sell_block(a.A, q, M);
        tent_block(a, cb, which, X);
        mm_add(M, X, S);
    }
    const double om = (4.0 / 3.0) / a.lam[0];
    double X[9];
#pragma unroll
    for (int k = 0; k < 9; k++) X[k] = 0.0;
    if (a.agg[r] == K) tent_block(a, r, which, X);
    const int64_t N = a.N;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            double d = 0.0;
#pragma unroll
            for (int m = 0; m < 3; m++) d = fma(a.jac[(3 * i + m) * N + r], S[3 * m + k], d);
            const double v = X[3 * i + k] - om * d;
            a.P64[p * 9 + 3 * i + k] = v;
            a.P32[p * 9 + 3 * i + k] = (float)v;
        }
}

// Q(r, J) = sum_{b in row r} A_rb P(b, J)
__global__ void __launch_bounds__(128) k_sa_q(SaArgs a) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.nnzQ) return;
    const int64_t r = a.q_row[p];
    const int32_t J = a.q_col[p];
    double S[9];
#pragma unroll
    for (int k = 0; k < 9; k++) S[k] = 0.0;
    const int t = (int)(r & 31);
    const int64_t b0 = a.slice_ptr[r >> 5];
    const int len = a.row_len[r];
    for (int j = 0; j < len; j++) {
        const int64_t q = (b0 + j) * 32 + t;
        const int64_t cb = a.col[q];
        const int idx = find_col(a.p_col, a.p_ptr[cb], a.p_ptr[cb + 1], J);
        if (idx < 0) continue;
        double M[9];
        sell_block(a.A, q, M);
        mm_add(M, a.P64 + (int64_t)idx * 9, S);
    }
#pragma unroll
    for (int k = 0; k < 9; k++) a.Q64[p * 9 + k] = S[k];
}

struct GalArgs {
    const int32_t *pt_ptr, *pt_row, *pt_slot;
    const double *P64;
    const int32_t *q_ptr, *q_col;
    const double *Q64;
    const int32_t *slice_ptr, *row_len, *col, *col_slice;  // coarse SELL pattern
    double *Ac64;
    float *Ac32;
    int64_t Nc, nslots;
};

// A_c(J, C) = sum_{(r, p) in PT(J)} P_p^T Q(r, C), one thread per coarse slot
// (padding slots get zeros)
__global__ void __launch_bounds__(128) k_sa_galerkin(GalArgs a) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.nslots) return;
    const int64_t sc = s >> 5;
    const int t = (int)(s & 31);
    const int64_t sl = a.col_slice[sc];
    const int64_t J = sl * 32 + t;
    const int64_t j = sc - a.slice_ptr[sl];
    double S[9];
#pragma unroll
    for (int k = 0; k < 9; k++) S[k] = 0.0;
    if (J < a.Nc && j < a.row_len[J]) {
        const int32_t C = a.col[s];
        for (int32_t e = a.pt_ptr[J]; e < a.pt_ptr[J + 1]; e++) {
            const int64_t r = a.pt_row[e];
            const int idx = find_col(a.q_col, a.q_ptr[r], a.q_ptr[r + 1], C);
            if (idx < 0) continue;
            mtm_add(a.P64 + (int64_t)a.pt_slot[e] * 9, a.Q64 + (int64_t)idx * 9, S);
        }
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        a.Ac64[(sc * 9 + k) * 32 + t] = S[k];
        a.Ac32[(sc * 9 + k) * 32 + t] = (float)S[k];
    }
}

// inverses of the 3x3 diagonal blocks of a coarse level, stored [9][N]; a
// component whose row and column of the block are zero gets a unit diagonal
__global__ void k_block_inverse(const int32_t *__restrict__ diag_slot, const double *__restrict__ A, int64_t N,
                                double *__restrict__ jac64, float *__restrict__ jac32, unsigned *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t q = diag_slot[i], b = q >> 5, t = q & 31;
    double m[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) m[r][s] = A[(b * 9 + 3 * r + s) * 32 + t];
#pragma unroll
    for (int r = 0; r < 3; r++) {
        bool zero = true;
#pragma unroll
        for (int s = 0; s < 3; s++) zero = zero && m[r][s] == 0.0 && m[s][r] == 0.0;
        if (zero) m[r][r] = 1.0;
    }
    double inv[3][3];
    inv[0][0] = m[1][1] * m[2][2] - m[1][2] * m[2][1];
    inv[0][1] = m[0][2] * m[2][1] - m[0][1] * m[2][2];
    inv[0][2] = m[0][1] * m[1][2] - m[0][2] * m[1][1];
    inv[1][0] = m[1][2] * m[2][0] - m[1][0] * m[2][2];
    inv[1][1] = m[0][0] * m[2][2] - m[0][2] * m[2][0];
    inv[1][2] = m[0][2] * m[1][0] - m[0][0] * m[1][2];
    inv[2][0] = m[1][0] * m[2][1] - m[1][1] * m[2][0];
    inv[2][1] = m[0][1] * m[2][0] - m[0][0] * m[2][1];
    inv[2][2] = m[0][0] * m[1][1] - m[0][1] * m[1][0];
    const double det = m[0][0] * inv[0][0] + m[0][1] * inv[1][0] + m[0][2] * inv[2][0];
    double scale = 0.0;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) scale = fmax(scale, fabs(m[r][s]));
    if (!(fabs(det) > 1e-300 && fabs(det) > 1e-14 * scale * scale * scale)) {
        atomicOr(err, ERR_SINGULAR);
        return;
    }
    const double id = 1.0 / det;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) {
            jac64[(3 * r + s) * N + i] = inv[r][s] * id;
            jac32[(3 * r + s) * N + i] = (float)(inv[r][s] * id);
        }
}

// power steps for lambda: y = D^-1 A (s x) with s = sc[0] (init: y = a fixed
// start vector, the golden-ratio Weyl sequence in [-1, 1)); partial[block] =
// sum of y.y over the block's rows
__global__ void __launch_bounds__(128) k_power_step(const int32_t *__restrict__ slice_ptr,
                                                    const int32_t *__restrict__ row_len,
                                                    const int32_t *__restrict__ col, const double *__restrict__ A,
                                                    const double *__restrict__ jac, const double *__restrict__ x,
                                                    const double *__restrict__ sc, double *__restrict__ y,
                                                    double *__restrict__ partial, int64_t N, int init) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double yy = 0.0;
    if (i < N) {
        if (init) {
#pragma unroll
            for (int r = 0; r < 3; r++) {
                const double g = (double)(3 * i + r + 1) * 0.61803398874989484820;
                const double v = 2.0 * (g - floor(g)) - 1.0;
                y[3 * i + r] = v;
                yy = fma(v, v, yy);
            }
        } else {
            const int t = (int)(i & 31);
            const int64_t b0 = slice_ptr[i >> 5];
            const int len = row_len[i];
            double a0 = 0.0, a1 = 0.0, a2 = 0.0;
            for (int j = 0; j < len; j++) {
                const int64_t q = (b0 + j) * 32 + t;
                const int64_t c = col[q];
                const double *Ab = A + (q >> 5) * 288 + t;
                const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
                a0 = fma(Ab[0], x0, fma(Ab[32], x1, fma(Ab[64], x2, a0)));
                a1 = fma(Ab[96], x0, fma(Ab[128], x1, fma(Ab[160], x2, a1)));
                a2 = fma(Ab[192], x0, fma(Ab[224], x1, fma(Ab[256], x2, a2)));
            }
            const double s = sc[0];
#pragma unroll
            for (int r = 0; r < 3; r++) {
                const double v =
                    s * (jac[(3 * r) * N + i] * a0 + jac[(3 * r + 1) * N + i] * a1 + jac[(3 * r + 2) * N + i] * a2);
                y[3 * i + r] = v;
                yy = fma(v, v, yy);
            }
        }
    }
    __shared__ double red[4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) yy += __shfl_down_sync(0xffffffffu, yy, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = yy;
    __syncthreads();
    if (threadIdx.x == 0) partial[blockIdx.x] = (red[0] + red[1]) + (red[2] + red[3]);
}

// sum of the partials in a fixed order (one block of 256 threads): sc = 1 /
// norm; on the last step lam = kLamMargin x norm (the norm of D^-1 A applied
// to a unit vector)
__global__ void __launch_bounds__(256) k_power_fin(const double *__restrict__ partial, int nb, double *sc,
                                                   double *lam, int last) {
    __shared__ double red[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < nb; k += 256) s += partial[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nrm = sqrt(red[0]);
        const bool ok = nrm > 0.0 && isfinite(nrm);
        sc[0] = ok ? 1.0 / nrm : 1.0;
        if (last) lam[0] = ok ? kLamMargin * nrm : 1.0;
    }
}

// dense matrix of a coarsest SELL level, n = 3N, row-major (zeroed before)
__global__ void k_dense_scatter(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                                const int32_t *__restrict__ col, const int32_t *__restrict__ col_slice,
                                const double *__restrict__ A, double *__restrict__ M, int64_t N, int64_t nslots) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const int64_t sc = s >> 5;
    const int t = (int)(s & 31);
    const int64_t sl = col_slice[sc];
    const int64_t J = sl * 32 + t, j = sc - slice_ptr[sl];
    if (J >= N || j >= row_len[J]) return;
    const int64_t C = col[s], n = 3 * N;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) M[(3 * J + r) * n + 3 * C + k] = A[(sc * 9 + 3 * r + k) * 32 + t];
}

// Gauss-Jordan elimination with partial pivoting of the n x n matrix M (row-
// major, overwritten; ties in the pivot search go to the lower row), one
// block; W receives the inverse (row-major) and inv32 its FP32 copy. A row
// and column that are entirely zero get a unit diagonal first. A pivot below
// 1e-14 max|M| sets ERR_SINGULAR.
__global__ void __launch_bounds__(kGjThreads) k_gauss_jordan(double *__restrict__ M, double *__restrict__ W,
                                                             float *__restrict__ inv32, int n, unsigned *err) {
    __shared__ double fcol[3 * kDenseMax];
    __shared__ double s_val[kGjThreads];
    __shared__ int s_idx[kGjThreads];
    __shared__ double s_scale;
    const int tid = threadIdx.x;
    const int64_t nn = (int64_t)n * n;
    for (int64_t e = tid; e < nn; e += kGjThreads) W[e] = (e / n == e % n) ? 1.0 : 0.0;
    for (int d = tid; d < n; d += kGjThreads) {
        bool zero = true;
        for (int k = 0; k < n && zero; k++) zero = M[(int64_t)d * n + k] == 0.0 && M[(int64_t)k * n + d] == 0.0;
        if (zero) M[(int64_t)d * n + d] = 1.0;
    }
    __syncthreads();
    double mx = 0.0;
    for (int64_t e = tid; e < nn; e += kGjThreads) mx = fmax(mx, fabs(M[e]));
    s_val[tid] = mx;
    __syncthreads();
    for (int w = kGjThreads / 2; w > 0; w >>= 1) {
        if (tid < w) s_val[tid] = fmax(s_val[tid], s_val[tid + w]);
        __syncthreads();
    }
    if (tid == 0) s_scale = s_val[0];
    __syncthreads();
    const double tiny = 1e-14 * s_scale;
    for (int k = 0; k < n; k++) {
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < n; i += kGjThreads) {
            const double v = fabs(M[(int64_t)i * n + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        s_val[tid] = best;
        s_idx[tid] = bi;
        __syncthreads();
        for (int w = kGjThreads / 2; w > 0; w >>= 1) {
            if (tid < w) {
                const double v2 = s_val[tid + w];
                const int i2 = s_idx[tid + w];
                if (v2 > s_val[tid] || (v2 == s_val[tid] && i2 < s_idx[tid])) {
                    s_val[tid] = v2;
                    s_idx[tid] = i2;
                }
            }
            __syncthreads();
        }
        const int pr = s_idx[0];
        const double pv = s_val[0];
        __syncthreads();
        if (!(pv > tiny)) {
            if (tid == 0) atomicOr(err, ERR_SINGULAR);
            return;
        }
        if (pr != k)
            for (int j = tid; j < n; j += kGjThreads) {
                const double a = M[(int64_t)k * n + j], b = W[(int64_t)k * n + j];
                M[(int64_t)k * n + j] = M[(int64_t)pr * n + j];
                W[(int64_t)k * n + j] = W[(int64_t)pr * n + j];
                M[(int64_t)pr * n + j] = a;
                W[(int64_t)pr * n + j] = b;
            }
        __syncthreads();
        const double ip = 1.0 / M[(int64_t)k * n + k];
        __syncthreads();
        for (int j = tid; j < n; j += kGjThreads) {
            M[(int64_t)k * n + j] *= ip;
            W[(int64_t)k * n + j] *= ip;
        }
        __syncthreads();
        for (int i = tid; i < n; i += kGjThreads) fcol[i] = M[(int64_t)i * n + k];
        __syncthreads();
        for (int64_t e = tid; e < nn; e += kGjThreads) {
            const int i = (int)(e / n), j = (int)(e % n);
            if (i == k) continue;
            const double f = fcol[i];
            if (f == 0.0) continue;
            M[e] -= f * M[(int64_t)k * n + j];
            W[e] -= f * W[(int64_t)k * n + j];
        }
        __syncthreads();
    }
    for (int64_t e = tid; e < nn; e += kGjThreads) inv32[e] = (float)W[e];
}

// x = A^-1 b on the coarsest level from the row-major dense inverse, one warp
// per row (lane l takes the columns j = l, l + 32, ...; shuffle sum)
template <typename T>
__global__ void __launch_bounds__(128) k_dense_apply(const T *__restrict__ inv, const T *__restrict__ b,
                                                     T *__restrict__ x, int n) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g >> 5, lane = g & 31;
    T s = 0;
    if (i < n)
        for (int j = lane; j < n; j += 32) s = fma(inv[(int64_t)i * n + j], b[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && i < n) x[i] = s;
}

// (A x)_i of a SELL level over L lanes per row: lane l takes the entries
// j = l, l + L, ..., the lane sums are combined by shuffles and every lane
// gets the row's result. A row i >= N takes no entries (all lanes of the warp
// reach the shuffles).
template <typename T, int L>
__device__ __forceinline__ void row_lanes(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                                          const int32_t *__restrict__ col, const T *__restrict__ A, int64_t i,
                                          int64_t N, int lane, const T *__restrict__ x, T &y0, T &y1, T &y2) {
    T a0 = 0, a1 = 0, a2 = 0;
    if (i < N) {
        const int t = (int)(i & 31);
        const int64_t b0 = slice_ptr[i >> 5];
        const int len = row_len[i];
        for (int j = lane; j < len; j += L) {
            const int64_t bb = b0 + j;
            const int64_t c = __ldg(col + bb * 32 + t);
            const T *Ab = A + bb * 288 + t;
            const T x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2];
            a0 = fma(__ldg(Ab + 0), x0, fma(__ldg(Ab + 32), x1, fma(__ldg(Ab + 64), x2, a0)));
            a1 = fma(__ldg(Ab + 96), x0, fma(__ldg(Ab + 128), x1, fma(__ldg(Ab + 160), x2, a1)));
            a2 = fma(__ldg(Ab + 192), x0, fma(__ldg(Ab + 224), x1, fma(__ldg(Ab + 256), x2, a2)));
        }
    }
    if constexpr (L > 1) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
    }
    y0 = a0;
    y1 = a1;
    y2 = a2;
}

// the operator of one level as the kernels read it
template <typename T>
struct LvOp {
    const int32_t *slice_ptr, *row_len, *col;
    const T *A, *jac;  // values, [9][N] diagonal-block inverses
    const double *lam;
    int64_t N;
};

// Chebyshev interval of the smoother on D^-1 A_l: [lam / kSmoothRatio, lam]
__device__ __forceinline__ void smooth_interval(const double *lam, double &theta, double &delta) {
    const double lmax = lam[0], lmin = lmax / kSmoothRatio;
    theta = 0.5 * (lmax + lmin);
    delta = 0.5 * (lmax - lmin);
}

template <typename T>
__device__ __forceinline__ void dinv_row(const T *__restrict__ jac, int64_t N, int64_t i, T r0, T r1, T r2, T out[3]) {
#pragma unroll
    for (int k = 0; k < 3; k++)
        out[k] = jac[(3 * k) * N + i] * r0 + jac[(3 * k + 1) * N + i] * r1 + jac[(3 * k + 2) * N + i] * r2;
}

// r = b - A x; with from_zero r = b and x = 0. Then d = D^-1 r / theta (the
// first direction of the Chebyshev smoother). with_d = 0: r only.
template <typename T, int L>
__global__ void __launch_bounds__(128) k_cheb_start(LvOp<T> o, T *__restrict__ x, const T *__restrict__ b,
                                                    T *__restrict__ r, T *__restrict__ d, int from_zero, int with_d) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = g / L;
    const int lane = (int)(g % L);
    T y0 = 0, y1 = 0, y2 = 0;
    if (!from_zero) row_lanes<T, L>(o.slice_ptr, o.row_len, o.col, o.A, i, o.N, lane, x, y0, y1, y2);
    if (lane != 0 || i >= o.N) return;
    const T r0 = b[3 * i] - y0, r1 = b[3 * i + 1] - y1, r2 = b[3 * i + 2] - y2;
    r[3 * i] = r0;
    r[3 * i + 1] = r1;
    r[3 * i + 2] = r2;
    if (from_zero) x[3 * i] = x[3 * i + 1] = x[3 * i + 2] = 0;
    if (!with_d) return;
    double theta, delta;
    smooth_interval(o.lam, theta, delta);
    const T it = (T)(1.0 / theta);
    T z[3];
    dinv_row<T>(o.jac, o.N, i, r0, r1, r2, z);
#pragma unroll
    for (int k = 0; k < 3; k++) d[3 * i + k] = z[k] * it;
}

// Chebyshev step k (1 <= k < degree): r -= A d; x += d;
// d' = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r, with rho_0 = 1 / sigma,
// rho_k = 1 / (2 sigma - rho_{k-1}), sigma = theta / delta
template <typename T, int L>
__global__ void __launch_bounds__(128) k_cheb_step(LvOp<T> o, T *__restrict__ x, T *__restrict__ r,
                                                   const T *__restrict__ d, T *__restrict__ dn, int k) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = g / L;
    const int lane = (int)(g % L);
    T y0, y1, y2;
    row_lanes<T, L>(o.slice_ptr, o.row_len, o.col, o.A, i, o.N, lane, d, y0, y1, y2);
    if (lane != 0 || i >= o.N) return;
    double theta, delta;
    smooth_interval(o.lam, theta, delta);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma, rho1 = rho;
    for (int q = 1; q <= k; q++) {
        rho1 = 1.0 / (2.0 * sigma - rho);
        if (q < k) rho = rho1;
    }
    const T c0 = (T)(rho1 * rho), c1 = (T)(2.0 * rho1 / delta);
    const T r0 = r[3 * i] - y0, r1 = r[3 * i + 1] - y1, r2 = r[3 * i + 2] - y2;
    r[3 * i] = r0;
    r[3 * i + 1] = r1;
    r[3 * i + 2] = r2;
    T z[3];
    dinv_row<T>(o.jac, o.N, i, r0, r1, r2, z);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const T dv = d[3 * i + q];
        x[3 * i + q] += dv;
        dn[3 * i + q] = c0 * dv + c1 * z[q];
    }
}

template <typename T>
__global__ void k_axpy1(T *__restrict__ x, const T *__restrict__ d, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] += d[i];
}

// b_c(J) = sum_{(r, p) in PT(J)} P_p^T r_r over L lanes per coarse row (lane
// l takes the entries e = l, l + L, ... of the ascending list)
template <typename T, int L>
__global__ void __launch_bounds__(128) k_sa_restrict(const int32_t *__restrict__ pt_ptr,
                                                     const int32_t *__restrict__ pt_row,
                                                     const int32_t *__restrict__ pt_slot, const T *__restrict__ P,
                                                     const T *__restrict__ r, T *__restrict__ bc, int64_t Nc) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t J = g / L;
    const int lane = (int)(g % L);
    T s0 = 0, s1 = 0, s2 = 0;
    if (J < Nc)
        for (int32_t e = pt_ptr[J] + lane; e < pt_ptr[J + 1]; e += L) {
            const int64_t i = pt_row[e];
            const T *Pb = P + (int64_t)pt_slot[e] * 9;
            const T r0 = r[3 * i], r1 = r[3 * i + 1], r2 = r[3 * i + 2];
            s0 = fma(Pb[0], r0, fma(Pb[3], r1, fma(Pb[6], r2, s0)));
            s1 = fma(Pb[1], r0, fma(Pb[4], r1, fma(Pb[7], r2, s1)));
            s2 = fma(Pb[2], r0, fma(Pb[5], r1, fma(Pb[8], r2, s2)));
        }
    if constexpr (L > 1) {
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
    }
    if (lane != 0 || J >= Nc) return;
    bc[3 * J] = s0;
    bc[3 * J + 1] = s1;
    bc[3 * J + 2] = s2;
}

// x(i) += sum_p P_p x_c(col p), over row i of P
template <typename T>
__global__ void k_sa_prolong(const int32_t *__restrict__ p_ptr, const int32_t *__restrict__ p_col,
                             const T *__restrict__ P, const T *__restrict__ xc, T *__restrict__ x, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T a0 = 0, a1 = 0, a2 = 0;
    for (int32_t p = p_ptr[i]; p < p_ptr[i + 1]; p++) {
        const int64_t J = p_col[p];
        const T *Pb = P + (int64_t)p * 9;
        const T c0 = xc[3 * J], c1 = xc[3 * J + 1], c2 = xc[3 * J + 2];
        a0 = fma(Pb[0], c0, fma(Pb[1], c1, fma(Pb[2], c2, a0)));
        a1 = fma(Pb[3], c0, fma(Pb[4], c1, fma(Pb[5], c2, a1)));
        a2 = fma(Pb[6], c0, fma(Pb[7], c1, fma(Pb[8], c2, a2)));
    }
    x[3 * i] += a0;
    x[3 * i + 1] += a1;
    x[3 * i + 2] += a2;
}

template <typename Tin, typename Tout>
__global__ void k_copy(const Tin *__restrict__ a, Tout *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (Tout)a[i];
}

template <typename T>
struct LvView;
template <>
struct LvView<float> {
    static const float *A(const Level &l) { return l.A32; }
    static const float *J(const Level &l) { return l.jac32; }
    static const float *P(const Level &l) { return l.P32; }
    static const float *D(const Level &l) { return l.dinv32; }
    static float *b(Level &l) { return l.b32; }
    static float *x(Level &l) { return l.x32; }
    static float *r(Level &l) { return l.r32; }
    static float *e(Level &l) { return l.e32; }
};

#define AMG_LAUNCH(...) ((__VA_ARGS__), ::hyel::count_launch())

template <typename T>
LvOp<T> lv_op(const Level &L) {
    using V = LvView<T>;
    return LvOp<T>{L.slice_ptr, L.row_len, L.col, V::A(L), V::J(L), L.lam, L.N};
}

// L lanes per row: r = b - A x (from_zero: r = b, x = 0) and the smoother's
// first direction
template <typename T>
void start_launch(Ctx &c, Level &L, T *x, const T *b, T *r, T *d, int from_zero, int with_d) {
    const LvOp<T> o = lv_op<T>(L);
    const int64_t th = L.N * L.lanes;
    if (L.lanes == 32)
        AMG_LAUNCH(k_cheb_start<T, 32><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, b, r, d, from_zero, with_d));
    else if (L.lanes == 8)
        AMG_LAUNCH(k_cheb_start<T, 8><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, b, r, d, from_zero, with_d));
    else
        AMG_LAUNCH(k_cheb_start<T, 1><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, b, r, d, from_zero, with_d));
}

// degree steps of the Chebyshev iteration for A_l x = b on
// [lambda / kSmoothRatio, lambda], preconditioned by the block diagonal, from
// x = 0 (from_zero) or from the current x
template <typename T>
void cheb_smooth(Ctx &c, Level &L, int degree, bool from_zero) {
    using V = LvView<T>;
    T *x = V::x(L), *r = V::r(L), *d[2] = {V::e(L), V::e(L) + 3 * L.N};
    const LvOp<T> o = lv_op<T>(L);
    start_launch<T>(c, L, x, V::b(L), r, d[0], from_zero ? 1 : 0, 1);
    const int64_t th = L.N * L.lanes;
    for (int k = 1; k < degree; k++) {
        if (L.lanes == 32)
            AMG_LAUNCH(k_cheb_step<T, 32><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, r, d[(k - 1) & 1],
                                                                                     d[k & 1], k));
        else if (L.lanes == 8)
            AMG_LAUNCH(k_cheb_step<T, 8><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, r, d[(k - 1) & 1],
                                                                                    d[k & 1], k));
        else
            AMG_LAUNCH(k_cheb_step<T, 1><<<blocks_for(th, 128), 128, 0, c.stream>>>(o, x, r, d[(k - 1) & 1],
                                                                                    d[k & 1], k));
    }
    AMG_LAUNCH(k_axpy1<T><<<blocks_for(3 * L.N, 256), 256, 0, c.stream>>>(x, d[(degree - 1) & 1], 3 * L.N));
}

template <typename T>
void vcycle(Ctx &c, Amg &a, int l) {
    Level &L = a.lv[l];
    using V = LvView<T>;
    if (l + 1 == (int)a.lv.size()) {  // coarsest: dense inverse, or the smoother when coarsening stalled
        if (L.dinv32) {
            const int n = (int)(3 * L.N);
            AMG_LAUNCH(k_dense_apply<T><<<blocks_for(32 * (int64_t)n, 128), 128, 0, c.stream>>>(V::D(L), V::b(L),
                                                                                                 V::x(L), n));
        } else {
            cheb_smooth<T>(c, L, kCoarseDegree, true);
        }
        return;
    }
    Level &C = a.lv[l + 1];
    cheb_smooth<T>(c, L, kSmoothDegree, true);
    start_launch<T>(c, L, V::x(L), V::b(L), V::r(L), nullptr, 0, 0);
    const int64_t th = C.N * 32;
    AMG_LAUNCH(k_sa_restrict<T, 32><<<blocks_for(th, 128), 128, 0, c.stream>>>(L.pt_ptr, L.pt_row, L.pt_slot,
                                                                                 V::P(L), V::r(L), V::b(C), C.N));
    vcycle<T>(c, a, l + 1);
    AMG_LAUNCH(k_sa_prolong<T><<<blocks_for(L.N, 128), 128, 0, c.stream>>>(L.p_ptr, L.p_col, V::P(L), V::x(C),
                                                                             V::x(L), L.N));
    cheb_smooth<T>(c, L, kSmoothDegree, false);
}

// union of the ascending lists cols(row) over the given rows, ascending
struct Union {
    std::vector<int32_t> mark, out;
    explicit Union(int64_t ncols) : mark(ncols, -1) {}
    template <typename F>
    void row(int64_t tag, F &&each) {
        out.clear();
        each([&](int32_t v) {
            if (mark[v] != tag) {
                mark[v] = (int32_t)tag;
                out.push_back(v);
            }
        });
        std::sort(out.begin(), out.end());
    }
};

void check_int32(size_t n, const char *what) {
    if (n >= ((size_t)1 << 31) / 9) fail(HYEL_EINVAL, std::string("amg: too many entries in ") + what);
}

}  // namespace

// ---------------------------------------------------------------- host setup

void amg_free(Ctx &c) {
    delete c.amg;
    c.amg = nullptr;
}

static void amg_build(Ctx &c) {
    DeviceMesh &m = c.mesh;
    if ((int64_t)m.h_X.size() != 3 * m.N) fail(HYEL_ESTATE, "amg: the mesh coordinates are missing");
    Amg *a = new Amg();
    c.amg = a;
    int64_t N = m.N;  // block-nodes of the current level
    std::vector<int32_t> rp = m.h_row_ptr, cols = m.h_col;
    int bsup = 1;  // block-nodes per super-node (1 on level 0, 2 above)
    int64_t nsup = N;
    std::vector<double> pos = m.h_X;       // [nsup][3] super-node positions
    std::vector<double> ell(nsup, 1.0);    // super-node length scales (coarse levels)
    // super-node graph (ascending, with the node itself): the mesh pattern on
    // level 0, then the adjacency of the aggregates (not the wider pattern of
    // the smoothed Galerkin operator, which would make the aggregates too big)
    std::vector<int32_t> srp = rp, scol = cols;
    {
        Level L0;
        L0.N = N;
        L0.nslots = m.nslots;
        L0.slice_ptr = m.slice_ptr;
        L0.row_len = m.row_len;
        L0.col = m.col;
        L0.diag_slot = m.diag_slot;
        L0.col_slice = m.col_slice;
        L0.nnzb = m.nnzb;
        a->lv.push_back(L0);
    }
    while ((int)a->lv.size() < kMaxLevels && N > kDenseMax) {
        // greedy aggregation of the super-nodes
        std::vector<int32_t> agg(nsup, -1);
        int32_t nc = 0;
        for (int64_t i = 0; i < nsup; i++) {
            if (agg[i] >= 0) continue;
            bool free = true;
            for (int32_t p = srp[i]; p < srp[i + 1] && free; p++) free = agg[scol[p]] < 0;
            if (!free) continue;
            for (int32_t p = srp[i]; p < srp[i + 1]; p++) agg[scol[p]] = nc;
            nc++;
        }
        {
            const std::vector<int32_t> agg1 = agg;
            for (int64_t i = 0; i < nsup; i++)
                if (agg1[i] < 0)
                    for (int32_t p = srp[i]; p < srp[i + 1]; p++)
                        if (agg1[scol[p]] >= 0) {
                            agg[i] = agg1[scol[p]];
                            break;
                        }
        }
        for (int64_t i = 0; i < nsup; i++)
            if (agg[i] < 0) {
                for (int32_t p = srp[i]; p < srp[i + 1]; p++)
                    if (agg[scol[p]] < 0) agg[scol[p]] = nc;
                agg[i] = nc;
                nc++;
            }
        if (nc >= 0.6 * nsup || 2 * (int64_t)nc >= N) break;  // coarsening stalled
        // the next level's super-node graph: aggregates K ~ K' when members are adjacent
        std::vector<int32_t> nrp(nc + 1, 0), ncol;
        {
            std::vector<int32_t> mptr(nc + 1, 0), mlist(nsup);
            for (int64_t i = 0; i < nsup; i++) mptr[agg[i] + 1]++;
            for (int32_t K = 0; K < nc; K++) mptr[K + 1] += mptr[K];
            std::vector<int32_t> fill(mptr.begin(), mptr.end() - 1);
            for (int64_t i = 0; i < nsup; i++) mlist[fill[agg[i]]++] = (int32_t)i;
            Union u(nc);
            for (int32_t K = 0; K < nc; K++) {
                u.row(K, [&](auto add) {
                    for (int32_t e = mptr[K]; e < mptr[K + 1]; e++) {
                        const int32_t i = mlist[e];
                        for (int32_t p = srp[i]; p < srp[i + 1]; p++) add(agg[scol[p]]);
                    }
                });
                ncol.insert(ncol.end(), u.out.begin(), u.out.end());
                nrp[K + 1] = (int32_t)ncol.size();
            }
        }
        // centroids and length scales of the aggregates
        std::vector<double> cpos(3 * (size_t)nc, 0.0), cell(nc, 0.0), mell(nc, 0.0);
        std::vector<int32_t> cnt(nc, 0);
        for (int64_t s = 0; s < nsup; s++) {
            const int32_t K = agg[s];
            for (int d = 0; d < 3; d++) cpos[3 * K + d] += pos[3 * s + d];
            cnt[K]++;
            mell[K] = std::max(mell[K], ell[s]);
        }
        for (int32_t K = 0; K < nc; K++)
            for (int d = 0; d < 3; d++) cpos[3 * K + d] /= cnt[K];
        for (int64_t s = 0; s < nsup; s++) {
            const int32_t K = agg[s];
            for (int d = 0; d < 3; d++) {
                const double dx = pos[3 * s + d] - cpos[3 * K + d];
                cell[K] += dx * dx;
            }
        }
        for (int32_t K = 0; K < nc; K++) {
            cell[K] = std::sqrt(cell[K] / cnt[K]);
            if (!(cell[K] > 0.0)) cell[K] = bsup == 1 ? 1.0 : mell[K];
        }
        // P0 blocks per block-node: translation T, rotation R (row-major)
        std::vector<double> tent(18 * (size_t)N, 0.0);
        std::vector<int32_t> agg_bn(N);
        for (int64_t s = 0; s < nsup; s++) {
            const int32_t K = agg[s];
            const double il = 1.0 / cell[K];
            const double d0 = pos[3 * s] - cpos[3 * K], d1 = pos[3 * s + 1] - cpos[3 * K + 1],
                         d2 = pos[3 * s + 2] - cpos[3 * K + 2];
            // u = omega x d = -[d]_x omega, omega = R-variable / l_K
            const double Rm[9] = {0.0, d2 * il, -d1 * il, -d2 * il, 0.0, d0 * il, d1 * il, -d0 * il, 0.0};
            double *tb = tent.data() + 18 * (size_t)(s * bsup);
            tb[0] = tb[4] = tb[8] = 1.0;
            for (int k = 0; k < 9; k++) tb[9 + k] = Rm[k];
            agg_bn[s * bsup] = K;
            if (bsup == 2) {
                double *tr = tent.data() + 18 * (size_t)(2 * s + 1);
                tr[9] = tr[13] = tr[17] = ell[s] * il;
                agg_bn[2 * s + 1] = K;
            }
        }
        const int64_t Nc = 2 * (int64_t)nc;
        // P pattern: row b holds both block-nodes of every aggregate met in row b of A_l
        std::vector<int32_t> prp(N + 1, 0), pcol, prow;
        {
            Union u(Nc);
            for (int64_t b = 0; b < N; b++) {
                u.row(b, [&](auto add) {
                    for (int32_t q = rp[b]; q < rp[b + 1]; q++) {
                        const int32_t K = agg_bn[cols[q]];
                        add(2 * K);
                        add(2 * K + 1);
                    }
                });
                pcol.insert(pcol.end(), u.out.begin(), u.out.end());
                prow.insert(prow.end(), u.out.size(), (int32_t)b);
                prp[b + 1] = (int32_t)pcol.size();
                check_int32(pcol.size(), "P");
            }
        }
        // PT lists: per coarse block-node, the rows of P holding it, ascending
        std::vector<int32_t> ptp(Nc + 1, 0), ptrow(pcol.size()), ptslot(pcol.size());
        for (size_t p = 0; p < pcol.size(); p++) ptp[pcol[p] + 1]++;
        for (int64_t J = 0; J < Nc; J++) ptp[J + 1] += ptp[J];
        {
            std::vector<int32_t> fill(ptp.begin(), ptp.end() - 1);
            for (int64_t b = 0; b < N; b++)
                for (int32_t p = prp[b]; p < prp[b + 1]; p++) {
                    const int32_t f = fill[pcol[p]]++;
                    ptrow[f] = (int32_t)b;
                    ptslot[f] = p;
                }
        }
        // Q = A_l P pattern
        std::vector<int32_t> qrp(N + 1, 0), qcol, qrow;
        {
            Union u(Nc);
            for (int64_t b = 0; b < N; b++) {
                u.row(b, [&](auto add) {
                    for (int32_t q = rp[b]; q < rp[b + 1]; q++) {
                        const int32_t cb = cols[q];
                        for (int32_t p = prp[cb]; p < prp[cb + 1]; p++) add(pcol[p]);
                    }
                });
                qcol.insert(qcol.end(), u.out.begin(), u.out.end());
                qrow.insert(qrow.end(), u.out.size(), (int32_t)b);
                qrp[b + 1] = (int32_t)qcol.size();
                check_int32(qcol.size(), "Q");
            }
        }
        // A_{l+1} = P^T Q pattern
        std::vector<int32_t> crp(Nc + 1, 0), ccols;
        {
            Union u(Nc);
            for (int64_t J = 0; J < Nc; J++) {
                u.row(J, [&](auto add) {
                    for (int32_t e = ptp[J]; e < ptp[J + 1]; e++) {
                        const int32_t b = ptrow[e];
                        for (int32_t q = qrp[b]; q < qrp[b + 1]; q++) add(qcol[q]);
                    }
                });
                ccols.insert(ccols.end(), u.out.begin(), u.out.end());
                crp[J + 1] = (int32_t)ccols.size();
                check_int32(ccols.size(), "the coarse operator");
            }
        }
        SellHost cs = build_sell(Nc, crp, ccols);
        {
            Level &F = a->lv.back();
            F.nnzP = (int64_t)pcol.size();
            F.nnzQ = (int64_t)qcol.size();
            F.agg = up(c, agg_bn);
            F.tent = up(c, tent);
            F.p_ptr = up(c, prp);
            F.p_col = up(c, pcol);
            F.p_row = up(c, prow);
            F.P64 = dalloc_n<double>(c, 9 * (size_t)F.nnzP);
            F.P32 = dalloc_n<float>(c, 9 * (size_t)F.nnzP);
            F.pt_ptr = up(c, ptp);
            F.pt_row = up(c, ptrow);
            F.pt_slot = up(c, ptslot);
            F.q_ptr = up(c, qrp);
            F.q_col = up(c, qcol);
            F.q_row = up(c, qrow);
            F.Q64 = dalloc_n<double>(c, 9 * (size_t)F.nnzQ);
        }
        Level L;
        L.N = Nc;
        L.nslots = cs.nslots;
        L.slice_ptr = up(c, cs.slice_ptr);
        L.row_len = up(c, cs.row_len);
        L.col = up(c, cs.col);
        L.diag_slot = up(c, cs.diag_slot);
        L.col_slice = up(c, cs.col_slice);
        L.A64 = dalloc_n<double>(c, 9 * (size_t)cs.nslots);
        L.A32 = dalloc_n<float>(c, 9 * (size_t)cs.nslots);
        L.jac64 = dalloc_n<double>(c, 9 * (size_t)Nc);
        L.jac32 = dalloc_n<float>(c, 9 * (size_t)Nc);
        L.nnzb = (int64_t)ccols.size();
        L.lanes = Nc < kWarpRowsBelow ? 32 : 8;
        a->lv.push_back(L);
        // the next level's super-nodes are this level's aggregates
        N = Nc;
        rp = std::move(crp);
        cols = std::move(ccols);
        nsup = nc;
        bsup = 2;
        srp = std::move(nrp);
        scol = std::move(ncol);
        pos = std::move(cpos);
        ell = std::move(cell);
    }
    for (Level &L : a->lv) {
        L.x64 = dalloc_n<double>(c, 3 * (size_t)L.N);
        L.r64 = dalloc_n<double>(c, 3 * (size_t)L.N);
        L.b32 = dalloc_n<float>(c, 3 * (size_t)L.N);
        L.x32 = dalloc_n<float>(c, 3 * (size_t)L.N);
        L.r32 = dalloc_n<float>(c, 3 * (size_t)L.N);
        L.e32 = dalloc_n<float>(c, 6 * (size_t)L.N);
        L.lam = dalloc_n<double>(c, 1);
    }
    Level &Lc = a->lv.back();
    if (Lc.N <= kDenseMax) {
        const size_t n = 3 * (size_t)Lc.N;
        Lc.dense64 = dalloc_n<double>(c, n * n);
        Lc.dwork64 = dalloc_n<double>(c, n * n);
        Lc.dinv32 = dalloc_n<float>(c, n * n);
    }
    a->partial = dalloc_n<double>(c, (size_t)blocks_for(a->lv[0].N, 128));
    a->pscale = dalloc_n<double>(c, 1);
    HYEL_CK(cudaStreamSynchronize(c.stream));
}

// lambda of level L: kPowerSteps power steps on D^-1 A_l from the fixed start
static void power_estimate(Ctx &c, Amg &a, Level &L) {
    const int nb = blocks_for(L.N, 128);
    double *buf[2] = {L.x64, L.r64};
    AMG_LAUNCH(k_power_step<<<nb, 128, 0, c.stream>>>(L.slice_ptr, L.row_len, L.col, L.A64, L.jac64, nullptr,
                                                      a.pscale, buf[0], a.partial, L.N, 1));
    AMG_LAUNCH(k_power_fin<<<1, 256, 0, c.stream>>>(a.partial, nb, a.pscale, L.lam, 0));
    for (int k = 1; k <= kPowerSteps; k++) {
        AMG_LAUNCH(k_power_step<<<nb, 128, 0, c.stream>>>(L.slice_ptr, L.row_len, L.col, L.A64, L.jac64,
                                                          buf[(k - 1) & 1], a.pscale, buf[k & 1], a.partial, L.N, 0));
        AMG_LAUNCH(k_power_fin<<<1, 256, 0, c.stream>>>(a.partial, nb, a.pscale, L.lam, k == kPowerSteps));
    }
}

void amg_numeric(Ctx &c) {
    if (!c.mat.scaled) fail(HYEL_ESTATE, "amg: the scaled system is not set up");
    if (!c.amg) amg_build(c);
    Amg &a = *c.amg;
    Level &L0 = a.lv[0];
    L0.A64 = c.mat.As;
    L0.A32 = c.mat.Af;
    L0.jac64 = c.mat.jac64;
    L0.jac32 = c.mat.jac32;
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    const int nlev = (int)a.lv.size();
    for (int l = 0; l < nlev; l++) {
        Level &F = a.lv[l];
        if (l + 1 == nlev) {
            if (F.dinv32) {
                const int64_t n = 3 * F.N;
                HYEL_CK(cudaMemsetAsync(F.dense64, 0, (size_t)(n * n) * sizeof(double), c.stream));
                AMG_LAUNCH(k_dense_scatter<<<blocks_for(F.nslots, 128), 128, 0, c.stream>>>(
                    F.slice_ptr, F.row_len, F.col, F.col_slice, F.A64, F.dense64, F.N, F.nslots));
                AMG_LAUNCH(k_gauss_jordan<<<1, kGjThreads, 0, c.stream>>>(F.dense64, F.dwork64, F.dinv32,
                                                                         (int)n, c.err));
            } else {
                power_estimate(c, a, F);
            }
            break;
        }
        power_estimate(c, a, F);
        Level &C = a.lv[l + 1];
        SaArgs s;
        s.slice_ptr = F.slice_ptr;
        s.row_len = F.row_len;
        s.col = F.col;
        s.A = F.A64;
        s.jac = F.jac64;
        s.agg = F.agg;
        s.tent = F.tent;
        s.w = l == 0 ? c.mat.w : nullptr;
        s.dir = l == 0 ? c.mesh.dir : nullptr;
        s.lam = F.lam;
        s.p_ptr = F.p_ptr;
        s.p_col = F.p_col;
        s.p_row = F.p_row;
        s.P64 = F.P64;
        s.P32 = F.P32;
        s.q_ptr = F.q_ptr;
        s.q_col = F.q_col;
        s.q_row = F.q_row;
        s.Q64 = F.Q64;
        s.N = F.N;
        s.nnzP = F.nnzP;
        s.nnzQ = F.nnzQ;
        AMG_LAUNCH(k_sa_prolongator<<<blocks_for(F.nnzP, 128), 128, 0, c.stream>>>(s));
        AMG_LAUNCH(k_sa_q<<<blocks_for(F.nnzQ, 128), 128, 0, c.stream>>>(s));
        GalArgs g;
        g.pt_ptr = F.pt_ptr;
        g.pt_row = F.pt_row;
        g.pt_slot = F.pt_slot;
        g.P64 = F.P64;
        g.q_ptr = F.q_ptr;
        g.q_col = F.q_col;
        g.Q64 = F.Q64;
        g.slice_ptr = C.slice_ptr;
        g.row_len = C.row_len;
        g.col = C.col;
        g.col_slice = C.col_slice;
        g.Ac64 = C.A64;
        g.Ac32 = C.A32;
        g.Nc = C.N;
        g.nslots = C.nslots;
        AMG_LAUNCH(k_sa_galerkin<<<blocks_for(C.nslots, 128), 128, 0, c.stream>>>(g));
        AMG_LAUNCH(k_block_inverse<<<blocks_for(C.N, 128), 128, 0, c.stream>>>(C.diag_slot, C.A64, C.N, C.jac64,
                                                                             C.jac32, c.err));
    }
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & ERR_SINGULAR) fail(HYEL_ESINGULAR, "amg: a coarse operator is singular");
    a.numeric_ok = true;
}

int amg_levels(const Ctx &c, int64_t *sizes, int max) {
    if (!c.amg) return 0;
    const int n = (int)c.amg->lv.size();
    for (int l = 0; l < n && 2 * l + 1 < max; l++) {
        sizes[2 * l] = c.amg->lv[l].N;
        sizes[2 * l + 1] = c.amg->lv[l].nnzb;
    }
    return n;
}

// z = V-cycle(v) on [3N] vectors of precision T (stream-ordered; graph-safe).
// The cycle itself runs in FP32 for either level precision: it is a
// preconditioner of a flexible GMRES level, whose own products keep the
// level's precision, and in FP64 its block products would be bound by the
// FP64 pipe.
template <typename T>
void amg_apply(Ctx &c, const T *v, T *z) {
    Amg &a = *c.amg;
    Level &L0 = a.lv[0];
    const int64_t n = 3 * L0.N;
    AMG_LAUNCH(k_copy<T, float><<<blocks_for(n, 256), 256, 0, c.stream>>>(v, L0.b32, n));
    vcycle<float>(c, a, 0);
    AMG_LAUNCH(k_copy<float, T><<<blocks_for(n, 256), 256, 0, c.stream>>>(L0.x32, z, n));
}
template void amg_apply<double>(Ctx &, const double *, double *);
template void amg_apply<float>(Ctx &, const float *, float *);

}  // namespace hyel
