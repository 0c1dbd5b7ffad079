// Aggregation multigrid for the A-solves (the paper applies A^-1 through
// algebraic multigrid, §4.4 and §5). A GPU-native stand-in for BoomerAMG:
//
// * Setup of the hierarchy, once per mesh, on the host: greedy aggregation of
//   the block graph (a node and all its free neighbours form an aggregate;
//   leftovers join a neighbouring aggregate), coarse block patterns, and for
//   every coarse block the list of fine blocks that sum into it. Coarsening
//   stops at kCoarsest nodes or when a level shrinks by less than 40 %.
// * Numeric setup, after every scaling of a new assembly, on the GPU:
//   unsmoothed-aggregation Galerkin operators A_{l+1} = P^T A_l P with P the
//   aggregate indicator times I_3, so every level keeps 3x3 blocks in the
//   SELL-32 layout; each coarse block is the sum of its fine blocks in a fixed
//   order (bitwise reproducible). Then the inverses of the 3x3 diagonal
//   blocks of every level.
// * Application: one V-cycle with damped block-Jacobi smoothing (one pre- and
//   one post-sweep, omega = kOmega; kCoarseSweeps sweeps on the coarsest
//   level), a fixed linear operator, used as the right preconditioner of the
//   A-level (F)GMRES.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace hyel {

namespace {

constexpr int64_t kCoarsest = 256;
constexpr int kMaxLevels = 12;
constexpr double kOmega = 0.6;
constexpr int kCoarseSweeps = 6;

struct SellHost {
    std::vector<int32_t> slice_ptr, row_len, col, diag_slot;
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
    s.col.assign(s.nslots, 0);
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
    int64_t N = 0, nslots = 0;
    // SELL-32 pattern (device); level 0 borrows the mesh's arrays
    const int32_t *slice_ptr = nullptr, *row_len = nullptr, *col = nullptr, *diag_slot = nullptr;
    // values: level 0 borrows the scaled matrix and its block inverses
    double *A64 = nullptr, *jac64 = nullptr;
    float *A32 = nullptr, *jac32 = nullptr;
    // from the finer level: Galerkin lists (per coarse slot, fine slot ids),
    // aggregate members (per coarse node) and the fine node -> aggregate map
    int32_t *g_ptr = nullptr, *g_list = nullptr, *mem_ptr = nullptr, *mem_list = nullptr, *agg_of_fine = nullptr;
    int32_t *col_slice = nullptr;
    // work vectors [3N]: right-hand side, iterate, residual
    double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr;
    float *b32 = nullptr, *x32 = nullptr, *r32 = nullptr;
};

}  // namespace

struct Amg {
    std::vector<Level> lv;
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

// A_c(Q) = sum of the fine blocks listed for coarse slot Q (ascending fine slot)
__global__ void k_galerkin(const int32_t *__restrict__ g_ptr, const int32_t *__restrict__ g_list,
                           const double *__restrict__ Af, double *__restrict__ Ac, float *__restrict__ Ac32,
                           int64_t nslots_c) {
    const int64_t Q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (Q >= nslots_c) return;
    double acc[9];
#pragma unroll
    for (int k = 0; k < 9; k++) acc[k] = 0.0;
    for (int32_t p = g_ptr[Q]; p < g_ptr[Q + 1]; p++) {
        const int64_t q = g_list[p], b = q >> 5, t = q & 31;
#pragma unroll
        for (int k = 0; k < 9; k++) acc[k] += Af[(b * 9 + k) * 32 + t];
    }
    const int64_t B = Q >> 5, T = Q & 31;
#pragma unroll
    for (int k = 0; k < 9; k++) {
        Ac[(B * 9 + k) * 32 + T] = acc[k];
        Ac32[(B * 9 + k) * 32 + T] = (float)acc[k];
    }
}

// inverses of the 3x3 diagonal blocks, stored [9][N]
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

// x = omega J b (acc = 0) or x += omega J b (acc = 1), per node
template <typename T>
__global__ void k_jac_apply(const T *__restrict__ jac, const T *__restrict__ b, T *__restrict__ x, int64_t N,
                            T omega, int acc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T b0 = b[3 * i], b1 = b[3 * i + 1], b2 = b[3 * i + 2];
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const T v = omega * (jac[(3 * r) * N + i] * b0 + jac[(3 * r + 1) * N + i] * b1 + jac[(3 * r + 2) * N + i] * b2);
        x[3 * i + r] = acc ? x[3 * i + r] + v : v;
    }
}

// r = b - A x on a SELL-32 level
template <typename T>
__global__ void __launch_bounds__(128) k_residual_sell(const int32_t *__restrict__ slice_ptr,
                                                       const int32_t *__restrict__ row_len,
                                                       const int32_t *__restrict__ col, const T *__restrict__ A,
                                                       const T *__restrict__ x, const T *__restrict__ b,
                                                       T *__restrict__ r, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int t = (int)(i & 31);
    const int64_t b0 = slice_ptr[i >> 5];
    const int len = row_len[i];
    T a0 = 0, a1 = 0, a2 = 0;
    for (int j = 0; j < len; j++) {
        const int64_t bb = b0 + j;
        const int64_t c = __ldg(col + bb * 32 + t);
        const T *Ab = A + bb * 288 + t;
        const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
        a0 = fma(__ldg(Ab + 0), x0, fma(__ldg(Ab + 32), x1, fma(__ldg(Ab + 64), x2, a0)));
        a1 = fma(__ldg(Ab + 96), x0, fma(__ldg(Ab + 128), x1, fma(__ldg(Ab + 160), x2, a1)));
        a2 = fma(__ldg(Ab + 192), x0, fma(__ldg(Ab + 224), x1, fma(__ldg(Ab + 256), x2, a2)));
    }
    r[3 * i] = b[3 * i] - a0;
    r[3 * i + 1] = b[3 * i + 1] - a1;
    r[3 * i + 2] = b[3 * i + 2] - a2;
}

// b_c(I) = sum over the members of aggregate I of r (ascending fine node)
template <typename T>
__global__ void k_restrict(const int32_t *__restrict__ mem_ptr, const int32_t *__restrict__ mem_list,
                           const T *__restrict__ r, T *__restrict__ bc, int64_t Nc) {
    const int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= Nc) return;
    T s0 = 0, s1 = 0, s2 = 0;
    for (int32_t p = mem_ptr[I]; p < mem_ptr[I + 1]; p++) {
        const int64_t i = mem_list[p];
        s0 += r[3 * i];
        s1 += r[3 * i + 1];
        s2 += r[3 * i + 2];
    }
    bc[3 * I] = s0;
    bc[3 * I + 1] = s1;
    bc[3 * I + 2] = s2;
}

template <typename T>
__global__ void k_copy(const T *__restrict__ a, T *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// x(i) += x_c(agg(i))
template <typename T>
__global__ void k_prolong(const int32_t *__restrict__ agg, const T *__restrict__ xc, T *__restrict__ x, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t I = agg[i];
    x[3 * i] += xc[3 * I];
    x[3 * i + 1] += xc[3 * I + 1];
    x[3 * i + 2] += xc[3 * I + 2];
}

template <typename T>
struct LvView;
template <>
struct LvView<double> {
    static const double *A(const Level &l) { return l.A64; }
    static const double *J(const Level &l) { return l.jac64; }
    static double *b(Level &l) { return l.b64; }
    static double *x(Level &l) { return l.x64; }
    static double *r(Level &l) { return l.r64; }
};
template <>
struct LvView<float> {
    static const float *A(const Level &l) { return l.A32; }
    static const float *J(const Level &l) { return l.jac32; }
    static float *b(Level &l) { return l.b32; }
    static float *x(Level &l) { return l.x32; }
    static float *r(Level &l) { return l.r32; }
};

#define AMG_LAUNCH(...) ((__VA_ARGS__), ::hyel::count_launch())

template <typename T>
void vcycle(Ctx &c, Amg &a, int l) {
    Level &L = a.lv[l];
    using V = LvView<T>;
    const T om = (T)kOmega;
    const int nb = blocks_for(L.N, 128);
    if (l + 1 == (int)a.lv.size()) {  // coarsest: damped block-Jacobi sweeps
        AMG_LAUNCH(k_jac_apply<T><<<nb, 128, 0, c.stream>>>(V::J(L), V::b(L), V::x(L), L.N, om, 0));
        for (int s = 1; s < kCoarseSweeps; s++) {
            AMG_LAUNCH(k_residual_sell<T><<<nb, 128, 0, c.stream>>>(L.slice_ptr, L.row_len, L.col, V::A(L), V::x(L),
                                                                      V::b(L), V::r(L), L.N));
            AMG_LAUNCH(k_jac_apply<T><<<nb, 128, 0, c.stream>>>(V::J(L), V::r(L), V::x(L), L.N, om, 1));
        }
        return;
    }
    Level &C = a.lv[l + 1];
    // pre-smoothing from zero, residual, restriction
    AMG_LAUNCH(k_jac_apply<T><<<nb, 128, 0, c.stream>>>(V::J(L), V::b(L), V::x(L), L.N, om, 0));
    AMG_LAUNCH(k_residual_sell<T><<<nb, 128, 0, c.stream>>>(L.slice_ptr, L.row_len, L.col, V::A(L), V::x(L), V::b(L),
                                                              V::r(L), L.N));
    AMG_LAUNCH(k_restrict<T><<<blocks_for(C.N, 128), 128, 0, c.stream>>>(C.mem_ptr, C.mem_list, V::r(L), V::b(C), C.N));
    vcycle<T>(c, a, l + 1);
    // coarse correction, post-smoothing
    AMG_LAUNCH(k_prolong<T><<<nb, 128, 0, c.stream>>>(C.agg_of_fine, V::x(C), V::x(L), L.N));
    AMG_LAUNCH(k_residual_sell<T><<<nb, 128, 0, c.stream>>>(L.slice_ptr, L.row_len, L.col, V::A(L), V::x(L), V::b(L),
                                                              V::r(L), L.N));
    AMG_LAUNCH(k_jac_apply<T><<<nb, 128, 0, c.stream>>>(V::J(L), V::r(L), V::x(L), L.N, om, 1));
}

}  // namespace

// ---------------------------------------------------------------- host setup

void amg_free(Ctx &c) {
    delete c.amg;
    c.amg = nullptr;
}

static void amg_build(Ctx &c) {
    DeviceMesh &m = c.mesh;
    Amg *a = new Amg();
    c.amg = a;
    // level 0 on the host: the mesh's block pattern in the same SELL-32 layout
    int64_t N = m.N;
    std::vector<int32_t> rp = m.h_row_ptr, cols = m.h_col;
    SellHost fine = build_sell(N, rp, cols);
    {
        Level L0;
        L0.N = N;
        L0.nslots = m.nslots;
        L0.slice_ptr = m.slice_ptr;
        L0.row_len = m.row_len;
        L0.col = m.col;
        L0.diag_slot = m.diag_slot;
        a->lv.push_back(L0);
    }
    while ((int)a->lv.size() < kMaxLevels && N > kCoarsest) {
        // greedy aggregation
        std::vector<int32_t> agg(N, -1);
        int32_t nc = 0;
        for (int64_t i = 0; i < N; i++) {
            if (agg[i] >= 0) continue;
            bool free = true;
            for (int32_t p = rp[i]; p < rp[i + 1] && free; p++) free = agg[cols[p]] < 0;
            if (!free) continue;
            for (int32_t p = rp[i]; p < rp[i + 1]; p++) agg[cols[p]] = nc;
            nc++;
        }
        std::vector<int32_t> agg1 = agg;
        for (int64_t i = 0; i < N; i++)
            if (agg1[i] < 0)
                for (int32_t p = rp[i]; p < rp[i + 1]; p++)
                    if (agg1[cols[p]] >= 0) {
                        agg[i] = agg1[cols[p]];
                        break;
                    }
        for (int64_t i = 0; i < N; i++)
            if (agg[i] < 0) {
                for (int32_t p = rp[i]; p < rp[i + 1]; p++)
                    if (agg[cols[p]] < 0) agg[cols[p]] = nc;
                agg[i] = nc;
                nc++;
            }
        if (nc >= 0.6 * N) break;  // coarsening stalled
        // members of each aggregate, ascending fine node
        std::vector<int32_t> mem_ptr(nc + 1, 0), mem_list(N);
        for (int64_t i = 0; i < N; i++) mem_ptr[agg[i] + 1]++;
        for (int32_t I = 0; I < nc; I++) mem_ptr[I + 1] += mem_ptr[I];
        {
            std::vector<int32_t> fill(mem_ptr.begin(), mem_ptr.end() - 1);
            for (int64_t i = 0; i < N; i++) mem_list[fill[agg[i]]++] = (int32_t)i;
        }
        // coarse pattern (sorted columns, diagonal included)
        std::vector<int32_t> crp(nc + 1, 0), ccols;
        std::vector<int32_t> cand;
        for (int32_t I = 0; I < nc; I++) {
            cand.clear();
            for (int32_t p = mem_ptr[I]; p < mem_ptr[I + 1]; p++) {
                const int64_t i = mem_list[p];
                for (int32_t q = rp[i]; q < rp[i + 1]; q++) cand.push_back(agg[cols[q]]);
            }
            std::sort(cand.begin(), cand.end());
            cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
            ccols.insert(ccols.end(), cand.begin(), cand.end());
            crp[I + 1] = (int32_t)ccols.size();
        }
        SellHost cs = build_sell(nc, crp, ccols);
        // Galerkin lists: every fine (non-padding) slot adds into the slot of
        // (agg(row), agg(col)); lists in ascending fine slot order
        std::vector<int32_t> g_ptr(cs.nslots + 1, 0);
        std::vector<int32_t> target(fine.nslots, -1);
        for (int64_t r = 0; r < N; r++) {
            const int64_t I = agg[r];
            for (int32_t j = 0; j < fine.row_len[r]; j++) {
                const int64_t q = ((int64_t)fine.slice_ptr[r >> 5] + j) * 32 + (r & 31);
                const int32_t J = agg[fine.col[q]];
                const int32_t *b0 = ccols.data() + crp[I], *e0 = ccols.data() + crp[I + 1];
                const int32_t *f = std::lower_bound(b0, e0, J);
                if (f == e0 || *f != J) fail(HYEL_EINVAL, "amg: internal pattern error");
                const int64_t Q = ((int64_t)cs.slice_ptr[I >> 5] + (f - b0)) * 32 + (I & 31);
                target[q] = (int32_t)Q;
                g_ptr[Q + 1]++;
            }
        }
        for (int64_t Q = 0; Q < cs.nslots; Q++) g_ptr[Q + 1] += g_ptr[Q];
        std::vector<int32_t> g_list(g_ptr[cs.nslots]);
        {
            std::vector<int32_t> fill(g_ptr.begin(), g_ptr.end() - 1);
            for (int64_t q = 0; q < fine.nslots; q++)
                if (target[q] >= 0) g_list[fill[target[q]]++] = (int32_t)q;
        }
        Level L;
        L.N = nc;
        L.nslots = cs.nslots;
        L.slice_ptr = up(c, cs.slice_ptr);
        L.row_len = up(c, cs.row_len);
        L.col = up(c, cs.col);
        L.diag_slot = up(c, cs.diag_slot);
        L.g_ptr = up(c, g_ptr);
        L.g_list = up(c, g_list);
        L.mem_ptr = up(c, mem_ptr);
        L.mem_list = up(c, mem_list);
        L.agg_of_fine = up(c, agg);
        L.A64 = dalloc_n<double>(c, 9 * (size_t)cs.nslots);
        L.A32 = dalloc_n<float>(c, 9 * (size_t)cs.nslots);
        L.jac64 = dalloc_n<double>(c, 9 * (size_t)nc);
        L.jac32 = dalloc_n<float>(c, 9 * (size_t)nc);
        a->lv.push_back(L);
        // next level
        N = nc;
        rp = crp;
        cols = ccols;
        fine = cs;
    }
    for (Level &L : a->lv) {
        L.b64 = dalloc_n<double>(c, 3 * (size_t)L.N);
        L.x64 = dalloc_n<double>(c, 3 * (size_t)L.N);
        L.r64 = dalloc_n<double>(c, 3 * (size_t)L.N);
        L.b32 = dalloc_n<float>(c, 3 * (size_t)L.N);
        L.x32 = dalloc_n<float>(c, 3 * (size_t)L.N);
        L.r32 = dalloc_n<float>(c, 3 * (size_t)L.N);
    }
    HYEL_CK(cudaStreamSynchronize(c.stream));
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
    for (size_t l = 1; l < a.lv.size(); l++) {
        Level &F = a.lv[l - 1], &C = a.lv[l];
        AMG_LAUNCH(k_galerkin<<<blocks_for(C.nslots, 128), 128, 0, c.stream>>>(C.g_ptr, C.g_list, F.A64, C.A64, C.A32,
                                                                             C.nslots));
        AMG_LAUNCH(k_block_inverse<<<blocks_for(C.N, 128), 128, 0, c.stream>>>(C.diag_slot, C.A64, C.N, C.jac64,
                                                                             C.jac32, c.err));
    }
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & ERR_SINGULAR) fail(HYEL_ESINGULAR, "amg: a coarse diagonal block is singular");
    a.numeric_ok = true;
}

int amg_levels(const Ctx &c, int64_t *sizes, int max) {
    if (!c.amg) return 0;
    const int n = (int)c.amg->lv.size();
    for (int l = 0; l < n && l < max; l++) sizes[l] = c.amg->lv[l].N;
    return n;
}

// z = V-cycle(v) on [3N] vectors of precision T (stream-ordered; graph-safe)
template <typename T>
void amg_apply(Ctx &c, const T *v, T *z) {
    Amg &a = *c.amg;
    Level &L0 = a.lv[0];
    using V = LvView<T>;
    const int64_t n = 3 * L0.N;
    AMG_LAUNCH(k_copy<T><<<blocks_for(n, 256), 256, 0, c.stream>>>(v, V::b(L0), n));
    vcycle<T>(c, a, 0);
    AMG_LAUNCH(k_copy<T><<<blocks_for(n, 256), 256, 0, c.stream>>>(V::x(L0), z, n));
}
template void amg_apply<double>(Ctx &, const double *, double *);
template void amg_apply<float>(Ctx &, const float *, float *);

}  // namespace hyel
