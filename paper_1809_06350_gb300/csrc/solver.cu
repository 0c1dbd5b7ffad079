// Krylov solvers and the nested block preconditioner (§4).
//
// * Right-preconditioned GMRES(m) and FGMRES(m) (§4, ref. Saad), zero initial
//   guess, classical Gram-Schmidt with one full reorthogonalization (CGS2),
//   Givens rotations on the device; stop when the rotated residual
//   ||r|| <= max(rtol ||b||, atol) or at maxit.
// * Outer FGMRES on the symmetrically scaled system (§4.1) with the SCR
//   preconditioner of Algorithm 1; the Schur product of Algorithm 2 is
//   matrix-free with an inner A-solve; S-solves are right-preconditioned by
//   point-Jacobi on diag(S^), S^ = D - C diag(A)^-1 B (§4.2: the paper applies
//   S^^-1 by algebraic multigrid); A-solves by the inverses of the 3x3 node
//   diagonal blocks of A (the paper uses algebraic multigrid).
// * Precision: the intermediate and inner levels (A-, S- and inner solves,
//   their SpMVs and Gram-Schmidt) run in T = double or float; the outer
//   FGMRES, its Gram-Schmidt and Givens stay FP64 and the flexible basis Z is
//   FP64, so the outer iteration acts as iterative refinement.
//
// Every reduction has a fixed grid and a fixed summation order (per-block
// partials, then the last block to finish sums them in block order), so all
// results are bitwise reproducible.
//
// Each iteration's kernels read the level's device state and return at once
// when it is marked done, so the host may launch several iterations between
// convergence checks (``check_every``) without changing the result.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>

#include "internal.h"

namespace hyel {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 512;   // largest restart supported by the shared-memory coefficient buffers
constexpr int KC = 8;        // columns per multi-dot chunk

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Mark this block done; returns true in the last block to finish (all other
// blocks' partials are then visible to it).
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

enum { MD_STORE = 0, MD_INIT_FIRST = 1, MD_INIT_RESTART = 2, MD_DOT = 3 };

// h[k] = sum_i V[k*ld + i] w[i], k < nk. Modes:
//   MD_STORE: out[k] = h[k].
//   MD_INIT_FIRST / MD_INIT_RESTART (nk = 1, w = V): beta = ||V_0||, cycle start.
//   MD_DOT: out[0] = h[0] (no state).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_multidot(const T *__restrict__ V, int64_t ld, int nk,
                                                       const T *__restrict__ w, int64_t n, double *partial,
                                                       unsigned *counter, double *out, GmState *st, int mode,
                                                       double *g, int m, double rtol, double atol) {
    if (st && mode == MD_STORE && st->done) return;
    __shared__ double red[kThreads / 32][KC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int k0 = 0; k0 < nk; k0 += KC) {
        const int kc = min(KC, nk - k0);
        T acc[KC];
#pragma unroll
        for (int c = 0; c < KC; c++) acc[c] = 0;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const T wi = w[i];
#pragma unroll
            for (int c = 0; c < KC; c++)
                if (c < kc) acc[c] = fma(V[(int64_t)(k0 + c) * ld + i], wi, acc[c]);
        }
#pragma unroll
        for (int c = 0; c < KC; c++) {
            const T s = warp_sum(acc[c]);
            if (lane == 0) red[warp][c] = (double)s;
        }
        __syncthreads();
        if (threadIdx.x < kc) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < kThreads / 32; q++) s += red[q][threadIdx.x];
            partial[(int64_t)blockIdx.x * nk + k0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
    if (!last_block(counter)) return;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) s += ((volatile double *)partial)[(int64_t)b * nk + k];
        if (mode == MD_STORE || mode == MD_DOT) out[k] = s;
        if (mode == MD_INIT_FIRST || mode == MD_INIT_RESTART) {
            const double beta = sqrt(s);
            if (mode == MD_INIT_FIRST) {
                st->bnorm = beta;
                st->tol = fmax(rtol * beta, atol);
            }
            st->beta = beta;
            st->k = 0;
            st->res = beta;
            st->inv_scale = beta > 0.0 ? 1.0 / beta : 0.0;
            st->converged = (beta <= st->tol) ? 1 : 0;
            st->flags = isfinite(beta) ? 0 : 1;
            st->done = (st->converged || st->flags) ? 1 : 0;
            g[0] = beta;
            for (int l = 1; l <= m; l++) g[l] = 0.0;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// w -= sum_k V_k h[k]
template <typename T>
__global__ void __launch_bounds__(kThreads) k_multiaxpy(const T *__restrict__ V, int64_t ld, int nk,
                                                        const double *__restrict__ h, T *__restrict__ w, int64_t n,
                                                        const GmState *st) {
    if (st->done) return;
    __shared__ T hs[kMaxK];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = (T)h[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T acc = w[i];
        int k = 0;
        for (; k + 4 <= nk; k += 4) {
            acc = fma(-V[(int64_t)k * ld + i], hs[k], acc);
            acc = fma(-V[(int64_t)(k + 1) * ld + i], hs[k + 1], acc);
            acc = fma(-V[(int64_t)(k + 2) * ld + i], hs[k + 2], acc);
            acc = fma(-V[(int64_t)(k + 3) * ld + i], hs[k + 3], acc);
        }
        for (; k < nk; k++) acc = fma(-V[(int64_t)k * ld + i], hs[k], acc);
        w[i] = acc;
    }
}

// Second CGS pass update, norm of the new basis vector and the Givens step on
// Hessenberg column j (done by the last block).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_axpy_norm_givens(const T *__restrict__ V, int64_t ld, int j,
                                                               const double *__restrict__ h2, T *__restrict__ w,
                                                               int64_t n, double *partial, unsigned *counter,
                                                               double *H, double *cs, double *sn, double *g,
                                                               GmState *st, int m) {
    if (st->done) return;
    const int nk = j + 1;
    __shared__ T hs[kMaxK];
    __shared__ double red[kThreads / 32];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = (T)h2[k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    T ss = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T acc = w[i];
        int k = 0;
        for (; k + 4 <= nk; k += 4) {
            acc = fma(-V[(int64_t)k * ld + i], hs[k], acc);
            acc = fma(-V[(int64_t)(k + 1) * ld + i], hs[k + 1], acc);
            acc = fma(-V[(int64_t)(k + 2) * ld + i], hs[k + 2], acc);
            acc = fma(-V[(int64_t)(k + 3) * ld + i], hs[k + 3], acc);
        }
        for (; k < nk; k++) acc = fma(-V[(int64_t)k * ld + i], hs[k], acc);
        w[i] = acc;
        ss = fma(acc, acc, ss);
    }
    const T s = warp_sum(ss);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kThreads / 32; q++) t += red[q];
        partial[blockIdx.x] = t;
    }
    if (!last_block(counter)) return;
    double *Hc = H + (int64_t)j * (m + 1);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) Hc[k] += h2[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) t += ((volatile double *)partial)[b];
        const double hn = sqrt(t);
        Hc[j + 1] = hn;
        for (int l = 0; l < j; l++) {
            const double a0 = Hc[l], a1 = Hc[l + 1];
            Hc[l] = cs[l] * a0 + sn[l] * a1;
            Hc[l + 1] = -sn[l] * a0 + cs[l] * a1;
        }
        const double a = Hc[j];
        double c, s2, r;
        if (hn == 0.0) {
            c = 1.0;
            s2 = 0.0;
            r = a;
        } else {
            r = sqrt(a * a + hn * hn);
            c = a / r;
            s2 = hn / r;
        }
        cs[j] = c;
        sn[j] = s2;
        Hc[j] = r;
        Hc[j + 1] = 0.0;
        const double gj = g[j];
        g[j] = c * gj;
        g[j + 1] = -s2 * gj;
        const double res = fabs(g[j + 1]);
        st->k = j + 1;
        st->res = res;
        st->inv_scale = hn > 0.0 ? 1.0 / hn : 0.0;
        int done = 0;
        if (!isfinite(res) || !isfinite(hn)) {
            st->flags |= 1;
            done = 1;
        } else if (res <= st->tol) {
            st->converged = 1;
            done = 1;
        } else if (r == 0.0 || hn == 0.0) {
            st->flags |= 2;  // breakdown without convergence
            done = 1;
        }
        if (j + 1 == m) done = 1;
        st->done = done;
        *counter = 0u;
    }
}

// y = R^-1 g over the first k = st->k columns (one warp).
__global__ void k_backsolve(const double *H, const double *g, double *y, const GmState *st, int m) {
    const int k = st->k;
    const int lane = threadIdx.x;
    for (int i = k - 1; i >= 0; i--) {
        double s = 0.0;
        for (int l = i + 1 + lane; l < k; l += 32) s += H[(int64_t)l * (m + 1) + i] * y[l];
        s = warp_sum_d(s);
        if (lane == 0) y[i] = (g[i] - s) / H[(int64_t)i * (m + 1) + i];
        __syncwarp();
    }
}

// x (+)= jac * (sum_l V_l y_l) per node (GMRES on A with block-Jacobi).
template <typename T>
__global__ void k_update_bjac(const T *__restrict__ V, int64_t ld, const double *__restrict__ y,
                              const T *__restrict__ jac, T *__restrict__ x, int64_t N, const GmState *st, int accumulate) {
    __shared__ T ys[kMaxK];
    const int k = st->k;
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = (T)y[l];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    T u0 = 0, u1 = 0, u2 = 0;
    for (int l = 0; l < k; l++) {
        const T *Vl = V + (int64_t)l * ld + 3 * i;
        u0 = fma(Vl[0], ys[l], u0);
        u1 = fma(Vl[1], ys[l], u1);
        u2 = fma(Vl[2], ys[l], u2);
    }
    T z[3];
#pragma unroll
    for (int r = 0; r < 3; r++) z[r] = jac[(3 * r) * N + i] * u0 + jac[(3 * r + 1) * N + i] * u1 + jac[(3 * r + 2) * N + i] * u2;
#pragma unroll
    for (int r = 0; r < 3; r++) x[3 * i + r] = (accumulate ? x[3 * i + r] : (T)0) + z[r];
}

// x (+)= diag * (sum_l V_l y_l) (point Jacobi) or x (+)= sum_l Z_l y_l (diag == nullptr).
template <typename T>
__global__ void k_update_diag(const T *__restrict__ V, int64_t ld, const double *__restrict__ y,
                              const T *__restrict__ diag, T *__restrict__ x, int64_t n, const GmState *st, int accumulate) {
    __shared__ T ys[kMaxK];
    const int k = st->k;
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = (T)y[l];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T u = 0;
    for (int l = 0; l < k; l++) u = fma(V[(int64_t)l * ld + i], ys[l], u);
    if (diag) u *= diag[i];
    x[i] = (accumulate ? x[i] : (T)0) + u;
}

// v_j *= inv_scale; z = jac v_j  (block-Jacobi, per node)
template <typename T>
__global__ void k_scale_bjac(T *__restrict__ v, T *__restrict__ z, const T *__restrict__ jac, int64_t N, const GmState *st) {
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const T s = (T)st->inv_scale;
    const T v0 = v[3 * i] * s, v1 = v[3 * i + 1] * s, v2 = v[3 * i + 2] * s;
    v[3 * i] = v0;
    v[3 * i + 1] = v1;
    v[3 * i + 2] = v2;
#pragma unroll
    for (int r = 0; r < 3; r++) z[3 * i + r] = jac[(3 * r) * N + i] * v0 + jac[(3 * r + 1) * N + i] * v1 + jac[(3 * r + 2) * N + i] * v2;
}

// v_j *= inv_scale; z = diag .* v_j (diag == nullptr: scale only)
template <typename T>
__global__ void k_scale_diag(T *__restrict__ v, T *__restrict__ z, const T *__restrict__ diag, int64_t n, const GmState *st) {
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T s = (T)st->inv_scale;
    const T vi = v[i] * s;
    v[i] = vi;
    if (diag) z[i] = diag[i] * vi;
}

template <typename T>
__global__ void k_sub(const T *__restrict__ b, T *__restrict__ r, int64_t n) {  // r = b - r
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - r[i];
}

template <typename Tin, typename Tout>
__global__ void k_cast(const Tin *__restrict__ a, Tout *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (Tout)a[i];
}

__global__ void k_mul(const double *__restrict__ a, const double *__restrict__ w, double *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] * w[i];
}

// ------------------------------------------------------------ host driver

struct Level {
    int64_t its = 0;
    int32_t solves = 0;
};

template <typename T>
struct Gmres {
    Ctx *c = nullptr;
    int64_t n = 0;
    int m = 0;
    bool flexible = false;
    T *V = nullptr, *Z = nullptr, *z = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h2 = nullptr;
    double *partial = nullptr;
    unsigned *counter = nullptr;
    GmState *st = nullptr;
    GmState *hst = nullptr;
    int grid = 0;
    std::vector<void *> mem;

    void *alloc(size_t bytes) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            fail(HYEL_ENOMEM, "solver workspace: cudaMalloc failed");
        }
        mem.push_back(p);
        c->bytes_held += bytes;
        return p;
    }
    void init(Ctx *ctx, int64_t n_, int m_, bool flex) {
        c = ctx;
        n = n_;
        m = m_;
        flexible = flex;
        grid = (int)std::max<int64_t>(1, std::min<int64_t>(2 * c->num_sms, (n + 4 * kThreads - 1) / (4 * kThreads)));
        V = (T *)alloc(sizeof(T) * (size_t)(m + 1) * n);
        if (flexible)
            Z = (T *)alloc(sizeof(T) * (size_t)m * n);
        else
            z = (T *)alloc(sizeof(T) * (size_t)n);
        H = (double *)alloc(sizeof(double) * (size_t)(m + 1) * m);
        cs = (double *)alloc(sizeof(double) * m);
        sn = (double *)alloc(sizeof(double) * m);
        g = (double *)alloc(sizeof(double) * (m + 1));
        y = (double *)alloc(sizeof(double) * m);
        h2 = (double *)alloc(sizeof(double) * (m + 1));
        partial = (double *)alloc(sizeof(double) * (size_t)grid * (m + 1));
        counter = (unsigned *)alloc(sizeof(unsigned) * 4);
        st = (GmState *)alloc(sizeof(GmState));
        HYEL_CK(cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, c->stream));
        HYEL_CK(cudaMemsetAsync(st, 0, sizeof(GmState), c->stream));
        HYEL_CK(cudaMallocHost(&hst, sizeof(GmState)));
    }
    void release() {
        for (void *p : mem) cudaFree(p);
        mem.clear();
        if (hst) cudaFreeHost(hst);
        hst = nullptr;
    }
    void read_state() {
        HYEL_CK(cudaMemcpyAsync(hst, st, sizeof(GmState), cudaMemcpyDeviceToHost, c->stream));
        HYEL_CK(cudaStreamSynchronize(c->stream));
    }
    T *Vcol(int j) { return V + (size_t)j * n; }

    // Solve Op M^-1 u = b, x = M^-1 u (or FGMRES with Z). kind: 0 = block-Jacobi
    // (n = 3N), 1 = point-diagonal, 2 = flexible (prec callback).
    // Returns status; its accumulates iterations.
    int solve(const T *b, T *x, const hyel_krylov_level &L, int kind, const T *pdata,
              const std::function<void(const T *, T *, const int *)> &op,
              const std::function<void(const T *, T *)> &prec, int check_every, int64_t &its) {
        if (L.restart > m) fail(HYEL_EINVAL, "gmres: restart larger than workspace");
        const int mm = std::min(L.restart, m);
        const int64_t N3 = n / 3;
        HYEL_CK(cudaMemcpyAsync(Vcol(0), b, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->stream));
        (k_multidot<T><<<grid, kThreads, 0, c->stream>>>(V, n, 1, Vcol(0), n, partial, counter, nullptr, st,
                                                        MD_INIT_FIRST, g, mm, L.rtol, L.atol), ::hyel::count_launch());
        HYEL_CK(cudaGetLastError());
        int64_t total = 0;
        bool first = true;
        int status = HYEL_OK;
        for (;;) {
            read_state();
            if (hst->done) {
                if (hst->flags & 1) return HYEL_ENAN;
                if (first) HYEL_CK(cudaMemsetAsync(x, 0, sizeof(T) * n, c->stream));
                break;
            }
            int j = 0;
            for (; j < mm && total + j < L.maxit; j++) {
                T *vj = Vcol(j);
                T *w = Vcol(j + 1);
                T *zj = flexible ? Z + (size_t)j * n : z;
                if (kind == 0) {
                    (k_scale_bjac<T><<<blocks_for(N3, 128), 128, 0, c->stream>>>(vj, zj, pdata, N3, st), ::hyel::count_launch());
                } else if (kind == 1) {
                    (k_scale_diag<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(vj, zj, pdata, n, st), ::hyel::count_launch());
                } else {
                    (k_scale_diag<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(vj, zj, (const T *)nullptr, n, st), ::hyel::count_launch());
                    prec(vj, zj);
                }
                op(zj, w, &st->done);
                (k_multidot<T><<<grid, kThreads, 0, c->stream>>>(V, n, j + 1, w, n, partial, counter,
                                                                H + (size_t)j * (mm + 1), st, MD_STORE, g, mm, 0, 0), ::hyel::count_launch());
                (k_multiaxpy<T><<<grid, kThreads, 0, c->stream>>>(V, n, j + 1, H + (size_t)j * (mm + 1), w, n, st), ::hyel::count_launch());
                (k_multidot<T><<<grid, kThreads, 0, c->stream>>>(V, n, j + 1, w, n, partial, counter, h2, st, MD_STORE,
                                                                g, mm, 0, 0), ::hyel::count_launch());
                (k_axpy_norm_givens<T><<<grid, kThreads, 0, c->stream>>>(V, n, j, h2, w, n, partial, counter, H, cs, sn,
                                                                        g, st, mm), ::hyel::count_launch());
                HYEL_CK(cudaGetLastError());
                const bool last_it = (j + 1 == mm) || (total + j + 1 >= L.maxit);
                if (kind == 2 || last_it || ((j + 1) % std::max(1, check_every)) == 0) {
                    read_state();
                    if (hst->done) break;
                }
            }
            read_state();
            const int k = hst->k;
            if (k > 0) {
                (k_backsolve<<<1, 32, 0, c->stream>>>(H, g, y, st, mm), ::hyel::count_launch());
                const int acc = first ? 0 : 1;
                if (kind == 0)
                    (k_update_bjac<T><<<blocks_for(N3, 128), 128, 0, c->stream>>>(V, n, y, pdata, x, N3, st, acc), ::hyel::count_launch());
                else if (kind == 1)
                    (k_update_diag<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(V, n, y, pdata, x, n, st, acc), ::hyel::count_launch());
                else
                    (k_update_diag<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(Z, n, y, (const T *)nullptr, x, n, st,
                                                                               acc), ::hyel::count_launch());
                HYEL_CK(cudaGetLastError());
            } else if (first) {
                HYEL_CK(cudaMemsetAsync(x, 0, sizeof(T) * n, c->stream));
            }
            first = false;
            total += k;
            if (hst->flags & 1) {
                status = HYEL_ENAN;
                break;
            }
            if (hst->converged) break;
            if (hst->flags & 2) {
                status = HYEL_EBREAKDOWN;
                break;
            }
            if (total >= L.maxit) {
                status = HYEL_ENOCONV;
                break;
            }
            // restart: r = b - Op(x)
            op(x, Vcol(0), nullptr);
            (k_sub<T><<<blocks_for(n, 256), 256, 0, c->stream>>>(b, Vcol(0), n), ::hyel::count_launch());
            (k_multidot<T><<<grid, kThreads, 0, c->stream>>>(V, n, 1, Vcol(0), n, partial, counter, nullptr, st,
                                                            MD_INIT_RESTART, g, mm, 0, 0), ::hyel::count_launch());
            HYEL_CK(cudaGetLastError());
            if (kind == 0 || kind == 1) {
                // the non-flexible update needs x only after the cycle; nothing else to do
            }
        }
        its += total;
        return status;
    }
};

}  // namespace

// ------------------------------------------------------------ workspace

struct Workspace {
    int m_outer = 0, m_a = 0, m_s = 0, prec = -1;
    Gmres<double> outer;
    Gmres<double> a64, s64;
    Gmres<float> a32, s32;
    // vectors (sized 4N each), typed views
    double *d = nullptr;  // 12 x 4N doubles
    float *f = nullptr;   // 12 x 4N floats
    std::vector<void *> mem;
    void release() {
        outer.release();
        a64.release();
        s64.release();
        a32.release();
        s32.release();
        for (void *p : mem) cudaFree(p);
        mem.clear();
    }
};

void free_workspace(Ctx &c) {
    if (c.ws) {
        c.ws->release();
        delete c.ws;
        c.ws = nullptr;
    }
}

namespace {

Workspace &workspace(Ctx &c, const hyel_solver_params &p) {
    const int mo = p.outer.restart, ma = std::max(p.a.restart, p.inner.restart), ms = p.s.restart;
    Workspace *w = c.ws;
    if (w && w->m_outer >= mo && w->m_a >= ma && w->m_s >= ms && w->prec == p.precision) return *w;
    free_workspace(c);
    w = new Workspace();
    c.ws = w;
    const int64_t N = c.mesh.N;
    w->m_outer = mo;
    w->m_a = ma;
    w->m_s = ms;
    w->prec = p.precision;
    w->outer.init(&c, 4 * N, mo, true);
    if (p.precision == HYEL_PREC_FP64) {
        w->a64.init(&c, 3 * N, ma, false);
        w->s64.init(&c, N, ms, false);
    } else {
        w->a32.init(&c, 3 * N, ma, false);
        w->s32.init(&c, N, ms, false);
    }
    void *pd = nullptr, *pf = nullptr;
    if (cudaMalloc(&pd, sizeof(double) * 12 * 4 * (size_t)N) != cudaSuccess ||
        cudaMalloc(&pf, sizeof(float) * 12 * 4 * (size_t)N) != cudaSuccess) {
        (void)cudaGetLastError();
        fail(HYEL_ENOMEM, "solver workspace: cudaMalloc failed");
    }
    w->mem.push_back(pd);
    w->mem.push_back(pf);
    w->d = (double *)pd;
    w->f = (float *)pf;
    return *w;
}

void check_params(const hyel_solver_params &p) {
    const hyel_krylov_level *lv[4] = {&p.outer, &p.a, &p.s, &p.inner};
    for (auto *l : lv) {
        if (l->restart < 1 || l->restart > kMaxK) fail(HYEL_EINVAL, "solver params: restart must be in [1, 512]");
        if (l->maxit < 1) fail(HYEL_EINVAL, "solver params: maxit must be >= 1");
        if (!(l->rtol >= 0) || !(l->atol >= 0)) fail(HYEL_EINVAL, "solver params: tolerances must be >= 0");
    }
    if (p.precision != HYEL_PREC_FP64 && p.precision != HYEL_PREC_FP32) fail(HYEL_EINVAL, "solver params: bad precision");
}

// Typed view of the scaled matrix and the level solvers for precision T.
template <typename T>
struct Sys;
template <>
struct Sys<double> {
    static const double *A(Ctx &c) { return c.mat.As; }
    static const double *B(Ctx &c) { return c.mat.Bs; }
    static const double *C(Ctx &c) { return c.mat.Cs; }
    static const double *D(Ctx &c) { return c.mat.Ds; }
    static const double *jac(Ctx &c) { return c.mat.jac64; }
    static const double *shat(Ctx &c) { return c.mat.shat64; }
    static Gmres<double> &ga(Workspace &w) { return w.a64; }
    static Gmres<double> &gs(Workspace &w) { return w.s64; }
    static double *vec(Workspace &w, int k, int64_t N) { return w.d + (size_t)k * 4 * N; }
};
template <>
struct Sys<float> {
    static const float *A(Ctx &c) { return c.mat.Af; }
    static const float *B(Ctx &c) { return c.mat.Bf; }
    static const float *C(Ctx &c) { return c.mat.Cf; }
    static const float *D(Ctx &c) { return c.mat.Df; }
    static const float *jac(Ctx &c) { return c.mat.jac32; }
    static const float *shat(Ctx &c) { return c.mat.shat32; }
    static Gmres<float> &ga(Workspace &w) { return w.a32; }
    static Gmres<float> &gs(Workspace &w) { return w.s32; }
    static float *vec(Workspace &w, int k, int64_t N) { return w.f + (size_t)k * 4 * N; }
};

struct Counters {
    Level a, s, inner;
    int status = HYEL_OK;
    void note(int st) {
        if (status == HYEL_OK && st != HYEL_OK && st != HYEL_ENOCONV) status = st;
    }
};

// A-solve: x = A^-1 b with the given level controls.
template <typename T>
void a_solve(Ctx &c, Workspace &w, const hyel_solver_params &p, const hyel_krylov_level &L, const T *b, T *x,
             Level &lv, Counters &cnt) {
    Gmres<T> &g = Sys<T>::ga(w);
    auto op = [&c](const T *in, T *out, const int *done) { spmv_A<T>(c, Sys<T>::A(c), in, out, done); };
    int st = g.solve(b, x, L, 0, Sys<T>::jac(c), op, nullptr, p.check_every, lv.its);
    lv.solves++;
    cnt.note(st);
}

// Algorithm 2: y = D x - C A^-1 (B x)
template <typename T>
void schur_op(Ctx &c, Workspace &w, const hyel_solver_params &p, const T *x, T *y, Counters &cnt) {
    const int64_t N = c.mesh.N;
    T *xbar = Sys<T>::vec(w, 4, N);
    T *xtil = Sys<T>::vec(w, 5, N);
    spmv_B<T>(c, Sys<T>::B(c), x, xbar, nullptr, nullptr);
    a_solve<T>(c, w, p, p.inner, xbar, xtil, cnt.inner, cnt);
    spmv_DC<T>(c, Sys<T>::D(c), Sys<T>::C(c), x, xtil, y, nullptr);
}

// Algorithm 1 (SCR) as the preconditioner: (rv, rp) -> (xv, xp)
template <typename T>
void pscr(Ctx &c, Workspace &w, const hyel_solver_params &p, const T *rv, const T *rp, T *xv, T *xp, Counters &cnt) {
    const int64_t N = c.mesh.N;
    T *xhat = Sys<T>::vec(w, 0, N);
    T *rp2 = Sys<T>::vec(w, 1, N);
    T *rv2 = Sys<T>::vec(w, 2, N);
    // 1: A xhat = r_v
    a_solve<T>(c, w, p, p.a, rv, xhat, cnt.a, cnt);
    // 2: r_p <- r_p - C xhat
    spmv_C<T>(c, Sys<T>::C(c), xhat, rp2, rp, nullptr);
    // 3: S x_p = r_p, right-preconditioned by diag(S^)^-1
    Gmres<T> &gs = Sys<T>::gs(w);
    auto sop = [&](const T *in, T *out, const int *) { schur_op<T>(c, w, p, in, out, cnt); };
    int st = gs.solve(rp2, xp, p.s, 1, Sys<T>::shat(c), sop, nullptr, 1, cnt.s.its);
    cnt.s.solves++;
    cnt.note(st);
    // 4: r_v <- r_v - B x_p
    spmv_B<T>(c, Sys<T>::B(c), xp, rv2, rv, nullptr);
    // 5: A x_v = r_v
    a_solve<T>(c, w, p, p.a, rv2, xv, cnt.a, cnt);
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

void solve_nested(Ctx &c, const hyel_solver_params &p, const double *rhs, double *x, hyel_solve_stats *out) {
    check_params(p);
    if (!c.mat.assembled) fail(HYEL_ESTATE, "solve: nothing assembled");
    auto t0 = std::chrono::steady_clock::now();
    solve_setup(c);
    Workspace &w = workspace(c, p);
    HYEL_CK(cudaStreamSynchronize(c.stream));
    const double ms_setup = 1e3 * seconds_since(t0);
    auto t1 = std::chrono::steady_clock::now();
    const int64_t N = c.mesh.N, n = 4 * N;
    double *b = Sys<double>::vec(w, 8, N);
    double *xs = Sys<double>::vec(w, 9, N);
    double *r = Sys<double>::vec(w, 10, N);
    // r* = W r
    (k_mul<<<blocks_for(n, 256), 256, 0, c.stream>>>(rhs, c.mat.w, b, n), ::hyel::count_launch());
    Counters cnt;
    auto op = [&c](const double *in, double *o, const int *done) {
        spmv_full64(c, c.mat.As, c.mat.Bs, c.mat.Cs, c.mat.Ds, in, o, done);
    };
    std::function<void(const double *, double *)> prec;
    if (p.precision == HYEL_PREC_FP64) {
        prec = [&](const double *v, double *z) { pscr<double>(c, w, p, v, v + 3 * N, z, z + 3 * N, cnt); };
    } else {
        prec = [&](const double *v, double *z) {
            float *vf = Sys<float>::vec(w, 6, N), *zf = Sys<float>::vec(w, 7, N);
            (k_cast<double, float><<<blocks_for(n, 256), 256, 0, c.stream>>>(v, vf, n), ::hyel::count_launch());
            pscr<float>(c, w, p, vf, vf + 3 * N, zf, zf + 3 * N, cnt);
            (k_cast<float, double><<<blocks_for(n, 256), 256, 0, c.stream>>>(zf, z, n), ::hyel::count_launch());
        };
    }
    int64_t outer_its = 0;
    int st = w.outer.solve(b, xs, p.outer, 2, nullptr, op, prec, 1, outer_its);
    // true residual of the scaled system and unscaling x = W x*
    op(xs, r, nullptr);
    (k_sub<double><<<blocks_for(n, 256), 256, 0, c.stream>>>(b, r, n), ::hyel::count_launch());
    (k_multidot<double><<<w.outer.grid, kThreads, 0, c.stream>>>(r, n, 1, r, n, w.outer.partial, w.outer.counter,
                                                                c.red + 8, nullptr, MD_DOT, nullptr, 0, 0, 0), ::hyel::count_launch());
    (k_mul<<<blocks_for(n, 256), 256, 0, c.stream>>>(xs, c.mat.w, x, n), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_red + 8, c.red + 8, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    w.outer.read_state();
    const double bn = w.outer.hst->bnorm;
    const double rel = bn > 0 ? std::sqrt(c.h_red[8]) / bn : std::sqrt(c.h_red[8]);
    if (out) {
        out->status = st;
        out->outer_its = (int32_t)outer_its;
        out->a_its = cnt.a.its;
        out->s_its = cnt.s.its;
        out->inner_its = cnt.inner.its;
        out->a_solves = cnt.a.solves;
        out->s_solves = cnt.s.solves;
        out->inner_solves = cnt.inner.solves;
        out->rel_residual = rel;
        out->ms_setup = ms_setup;
        out->ms_solve = 1e3 * seconds_since(t1);
    }
    if (cnt.status != HYEL_OK && st == HYEL_OK) st = cnt.status;
    if (!std::isfinite(rel)) st = HYEL_ENAN;
    if (st != HYEL_OK) {
        const char *what = st == HYEL_ENOCONV ? "outer FGMRES reached its iteration cap"
                           : st == HYEL_ENAN  ? "NaN or Inf in the solve"
                           : st == HYEL_EBREAKDOWN ? "GMRES breakdown without convergence"
                                                   : "solve failed";
        fail(st, std::string("solve_nested: ") + what);
    }
}

void schur_apply(Ctx &c, const hyel_solver_params &p, const double *x, double *y, hyel_solve_stats *out) {
    check_params(p);
    if (!c.mat.assembled) fail(HYEL_ESTATE, "schur_apply: nothing assembled");
    solve_setup(c);
    Workspace &w = workspace(c, p);
    const int64_t N = c.mesh.N;
    Counters cnt;
    if (p.precision == HYEL_PREC_FP64) {
        schur_op<double>(c, w, p, x, y, cnt);
    } else {
        float *xf = Sys<float>::vec(w, 6, N), *yf = Sys<float>::vec(w, 7, N);
        (k_cast<double, float><<<blocks_for(N, 256), 256, 0, c.stream>>>(x, xf, N), ::hyel::count_launch());
        schur_op<float>(c, w, p, xf, yf, cnt);
        (k_cast<float, double><<<blocks_for(N, 256), 256, 0, c.stream>>>(yf, y, N), ::hyel::count_launch());
    }
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (out) {
        *out = hyel_solve_stats{};
        out->status = cnt.status;
        out->inner_its = cnt.inner.its;
        out->inner_solves = cnt.inner.solves;
    }
}

}  // namespace hyel
