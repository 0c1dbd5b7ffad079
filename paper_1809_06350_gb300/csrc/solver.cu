// Krylov solvers and the nested block preconditioner (§4).
//
// * Right-preconditioned GMRES(m) and FGMRES(m) (ref. Saad), zero initial
//   guess, classical Gram-Schmidt with one full reorthogonalization (CGS2;
//   loose A- and S-solves keep a single pass when a test in the manner of
//   Daniel-Gragg-Kaufman-Stewart allows), Givens rotations and
//   back-substitution on the device; stop when the rotated residual
//   ||r|| <= max(rtol ||b||, atol) or after maxit iterations. A restart takes
//   the new starting vector from the Arnoldi relation,
//   r = V_{k+1} Q^T (g_k e_k), so no extra operator application is needed.
// * Outer FGMRES on the symmetrically scaled system (§4.1) with the SCR
//   preconditioner of Algorithm 1; the Schur product of Algorithm 2 is
//   matrix-free with an inner A-solve. S-solves are right-preconditioned by
//   point-Jacobi on diag(S^), S^ = D - C diag(A)^-1 B (§4.2; the paper applies
//   S^^-1 by algebraic multigrid), A-solves by the inverses of the 3x3 node
//   diagonal blocks of A (the paper uses algebraic multigrid).
// * Precision: the intermediate and inner levels (A-, S- and inner solves,
//   their SpMVs and Gram-Schmidt) run in T = double or float; the outer
//   FGMRES, its Gram-Schmidt and Givens stay FP64 and its flexible basis Z is
//   FP64, so the outer iteration acts as iterative refinement. The BF16S
//   variant runs the float levels with A read from its BF16-with-block-scale
//   copy in the A-solves.
//
// Control flow: every Krylov level keeps its state (iteration index, norms,
// flags) in device memory. The intermediate A-solves (k_gmres_a) and the
// S-solve with its inner A-solves (k_gmres_s) are persistent cooperative
// kernels: one launch runs a whole solve, its phases separated by grid
// barriers. The outer FGMRES (and, with multigrid A-solves, the S-level) runs
// as a sequence of kernels per iteration. The whole nested solve is recorded
// once into a CUDA graph in which each kernel-per-step loop is a `while`
// conditional node; the last kernel of an iteration sets the loop condition.
// One graph launch performs the entire solve; the host reads the level states
// once at the end. The same kernels can instead be replayed by a host loop
// (params.graph = 0).
//
// Every reduction has a fixed grid and a fixed summation order (per-block
// partials summed in block order), so all results are bitwise reproducible.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <type_traits>

#include "internal.h"

namespace hyel {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxK = 512;  // largest restart supported by the shared-memory coefficient buffers
constexpr int kChebMaxDegree = 16;  // largest degree of the Chebyshev S-preconditioner
constexpr int KC = 8;       // columns per multi-dot chunk

struct LevelState {
    int k;          // basis vectors completed in the current cycle (iteration index j of the next one)
    int done;       // current cycle finished
    int stop;       // solve finished
    int converged;  // res <= tol
    int flags;      // 1 = NaN/Inf, 2 = breakdown without convergence
    int total;      // iterations of this solve
    int maxit, m;
    int cycles;
    int solves;        // completed solves since reset (statistics)
    long long its;     // iterations since reset (statistics)
    int status_any;    // OR of flags over solves since reset (1 nan, 2 breakdown, 4 cap reached)
    int yok;           // y = R^-1 g was formed for the finished cycle
    double beta, bnorm, tol, res, inv_scale;
    double alg_bytes;  // algorithmic bytes of the persistent A-solve iterations since reset
};

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
// blocks' writes are then visible to it).
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (last) __threadfence();
    return last;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, unsigned v) {
    if (h) cudaGraphSetConditional(h, v);
}

// Sum over the grid's per-block partials p[b*stride + k] for k < nk, by the
// last block: warp w handles columns w, w + nwarps, ...; its lanes stride over
// the blocks; the order is fixed, so the sum is reproducible.
__device__ __forceinline__ void sum_partials(const double *p, int stride, int nk, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int k = warp; k < nk; k += nw) {
        double s = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) s += ((volatile const double *)p)[(int64_t)b * stride + k];
        s = warp_sum_d(s);
        if (lane == 0) out[k] = s;
    }
}

// Block-wide sum of one double (all threads get the result in thread 0).
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum_d(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q];
    __syncthreads();
    return t;
}

// Start of a solve: V0 = b, x = 0, beta = ||b||, state, loop condition.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_init(const T *__restrict__ b, T *__restrict__ V0, T *__restrict__ x,
                                                   int64_t n, double *partial, unsigned *counter, LevelState *st,
                                                   double *g, int m, double rtol, double atol, int maxit,
                                                   cudaGraphConditionalHandle h) {
    __shared__ double red[kThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    T ss = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const T v = b[i];
        V0[i] = v;
        x[i] = 0;
        ss = fma(v, v, ss);
    }
    const double t = block_sum((double)ss, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    if (!last_block(counter)) return;
    __shared__ double tot;
    sum_partials(partial, 1, 1, &tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double beta = sqrt(tot);
        st->k = 0;
        st->total = 0;
        st->cycles = 0;
        st->maxit = maxit;
        st->m = m;
        st->beta = beta;
        st->bnorm = beta;
        st->tol = fmax(rtol * beta, atol);
        st->res = beta;
        st->inv_scale = beta > 0.0 ? 1.0 / beta : 0.0;
        const int nan = isfinite(beta) ? 0 : 1;
        st->flags = nan;
        st->converged = (!nan && beta <= st->tol) ? 1 : 0;
        st->stop = (st->converged || nan) ? 1 : 0;
        st->done = st->stop;
        if (st->stop) {
            st->solves += 1;
            st->status_any |= nan;
        }
        g[0] = beta;
        for (int l = 1; l <= m; l++) g[l] = 0.0;
        set_cond(h, st->stop ? 0u : 1u);
        *counter = 0u;
    }
}

// h[l] = V_l . w, l <= k (w = V_{k+1}); pass 1 stores into Hessenberg column k,
// pass 2 into h2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_multidot(const T *__restrict__ V, int64_t n, double *partial,
                                                       unsigned *counter, double *H, double *h2,
                                                       const LevelState *st, int pass) {
    if (st->done) return;
    const int j = st->k, nk = j + 1, m = st->m;
    const T *w = V + (int64_t)(j + 1) * n;
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
                if (c < kc) acc[c] = fma(V[(int64_t)(k0 + c) * n + i], wi, acc[c]);
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
            partial[(int64_t)blockIdx.x * (m + 1) + k0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
    if (!last_block(counter)) return;
    double *out = pass == 1 ? H + (int64_t)j * (m + 1) : h2;
    sum_partials(partial, m + 1, nk, out);
    if (threadIdx.x == 0) *counter = 0u;
}

// w -= sum_l V_l h_l with h the Hessenberg column k (first CGS pass).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_multiaxpy(T *__restrict__ V, int64_t n, const double *__restrict__ H,
                                                        const LevelState *st) {
    if (st->done) return;
    const int j = st->k, nk = j + 1, m = st->m;
    T *w = V + (int64_t)(j + 1) * n;
    __shared__ T hs[kMaxK];
    for (int k = threadIdx.x; k < nk; k += blockDim.x) hs[k] = (T)H[(int64_t)j * (m + 1) + k];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        T acc = w[i];
        int k = 0;
        for (; k + 4 <= nk; k += 4) {
            acc = fma(-V[(int64_t)k * n + i], hs[k], acc);
            acc = fma(-V[(int64_t)(k + 1) * n + i], hs[k + 1], acc);
            acc = fma(-V[(int64_t)(k + 2) * n + i], hs[k + 2], acc);
            acc = fma(-V[(int64_t)(k + 3) * n + i], hs[k + 3], acc);
        }
        for (; k < nk; k++) acc = fma(-V[(int64_t)k * n + i], hs[k], acc);
        w[i] = acc;
    }
}

// Second CGS pass, norm of the new basis vector, Givens step on column j, the
// stopping decision, and (when the cycle ends) y = R^-1 g.
// single != 0: one classical pass (h2 holds the only coefficients, which
// become the Hessenberg column); otherwise the second CGS2 pass (added to it).
template <typename T>
__global__ void __launch_bounds__(kThreads) k_axpy_norm_givens(T *__restrict__ V, int64_t n,
                                                               const double *__restrict__ h2, double *partial,
                                                               unsigned *counter, double *H, double *cs, double *sn,
                                                               double *g, double *y, LevelState *st, int single) {
    if (st->done) return;
    const int j = st->k, nk = j + 1, m = st->m;
    T *w = V + (int64_t)(j + 1) * n;
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
            acc = fma(-V[(int64_t)k * n + i], hs[k], acc);
            acc = fma(-V[(int64_t)(k + 1) * n + i], hs[k + 1], acc);
            acc = fma(-V[(int64_t)(k + 2) * n + i], hs[k + 2], acc);
            acc = fma(-V[(int64_t)(k + 3) * n + i], hs[k + 3], acc);
        }
        for (; k < nk; k++) acc = fma(-V[(int64_t)k * n + i], hs[k], acc);
        w[i] = acc;
        ss = fma(acc, acc, ss);
    }
    const double tb = block_sum((double)ss, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = tb;
    if (!last_block(counter)) return;
    double *Hc = H + (int64_t)j * (m + 1);
    for (int k = threadIdx.x; k < nk; k += blockDim.x) Hc[k] = single ? h2[k] : Hc[k] + h2[k];
    __shared__ int s_done;
    __shared__ double tot;
    sum_partials(partial, 1, 1, &tot);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double hn = sqrt(tot);
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
        st->total += 1;
        st->res = res;
        st->inv_scale = hn > 0.0 ? 1.0 / hn : 0.0;
        int done = 0, stop = 0;
        if (!isfinite(res) || !isfinite(hn)) {
            st->flags |= 1;
            done = stop = 1;
        } else if (r == 0.0) {  // singular Hessenberg: no least-squares solution this cycle
            st->flags |= 2;
            done = stop = 1;
        } else if (res <= st->tol) {
            st->converged = 1;
            done = stop = 1;
        } else if (hn == 0.0) {  // invariant subspace without convergence
            st->flags |= 2;
            done = stop = 1;
        } else if (st->total >= st->maxit) {
            done = stop = 1;
        } else if (j + 1 == m) {
            done = 1;
        }
        st->done = done;
        st->stop = stop;
        s_done = done && isfinite(res) && isfinite(hn) && r != 0.0;
        st->yok = s_done;
        *counter = 0u;
    }
    __syncthreads();
    if (s_done && threadIdx.x < 32) {  // y = R^-1 g over the k = j+1 columns (warp 0)
        const int k = j + 1, lane = threadIdx.x;
        for (int i = k - 1; i >= 0; i--) {
            double s = 0.0;
            for (int l = i + 1 + lane; l < k; l += 32) s += H[(int64_t)l * (m + 1) + i] * y[l];
            s = warp_sum_d(s);
            if (lane == 0) y[i] = (g[i] - s) / H[(int64_t)i * (m + 1) + i];
            __syncwarp();
        }
    }
}

// End of an iteration: when the cycle is done, x += M^-1 V y (KIND 1:
// diagonal M^-1) or x += Z y (KIND 2); if the solve
// continues (restart), V_0 = V Q^T (g_k e_k) and a new cycle starts. Sets the
// loop condition.
template <typename T, int KIND>
__global__ void __launch_bounds__(kThreads) k_cycle_end(T *__restrict__ V, const T *__restrict__ Z, T *__restrict__ x,
                                                        const T *__restrict__ prec, int64_t n, const double *y,
                                                        const double *cs, const double *sn, double *g,
                                                        unsigned *counter, LevelState *st,
                                                        cudaGraphConditionalHandle h) {
    if (!st->done) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(h, 1u);
        return;
    }
    if (st->stop == 2) return;  // already finalized (host-driven replays)
    const int k = st->k, stop = st->stop;
    __shared__ T ys[kMaxK];
    __shared__ T cr[kMaxK + 1];
    const bool usable = st->yok && k > 0;
    for (int l = threadIdx.x; l < k; l += blockDim.x) ys[l] = usable ? (T)y[l] : (T)0;
    if (!stop && threadIdx.x == 0) {
        // c = G_0^T G_1^T ... G_{k-1}^T (g_k e_k); G_i^T maps (a_i, a_{i+1}) to
        // (cs a_i - sn a_{i+1}, sn a_i + cs a_{i+1}), and a_i = 0 when it is applied
        double carry = g[k];
        for (int i = k - 1; i >= 0; i--) {
            cr[i + 1] = (T)(cs[i] * carry);
            carry = -sn[i] * carry;
        }
        cr[0] = (T)carry;
        // V_k still holds w = h_{k,k-1} v_k (its scaling is applied lazily)
        cr[k] = (T)(cs[k - 1] * g[k] * st->inv_scale);
    }
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if (usable) {
        const T *B = KIND == 2 ? Z : V;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            T u = 0;
            for (int l = 0; l < k; l++) u = fma(B[(int64_t)l * n + i], ys[l], u);
            if (KIND == 1) u *= prec[i];
            x[i] += u;
        }
    }
    if (!stop) {
        // restart vector (unnormalised) into V_0; element-wise, in place
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            T r = 0;
            for (int l = 0; l <= k; l++) r = fma(V[(int64_t)l * n + i], cr[l], r);
            V[i] = r;
        }
    }
    if (!last_block(counter)) return;
    if (threadIdx.x == 0) {
        if (stop) {
            st->its += st->total;
            st->solves += 1;
            st->status_any |= st->flags | ((!st->converged && !st->flags) ? 4 : 0);
            st->stop = 2;
            set_cond(h, 0u);
        } else {
            const double beta = fabs(g[k]);
            st->k = 0;
            st->done = 0;
            st->cycles += 1;
            st->beta = beta;
            st->res = beta;
            st->inv_scale = beta > 0.0 ? 1.0 / beta : 0.0;
            g[0] = beta;
            for (int l = 1; l <= st->m; l++) g[l] = 0.0;
            set_cond(h, 1u);
        }
        *counter = 0u;
    }
}

// v_k *= inv_scale; z = diag .* v_k (diag == nullptr: scale only, z unused)
template <typename T>
__global__ void k_scale_diag(T *__restrict__ V, T *__restrict__ z, const T *__restrict__ diag, int64_t n,
                             const LevelState *st) {
    if (st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T *v = V + (int64_t)st->k * n;
    const T vi = v[i] * (T)st->inv_scale;
    v[i] = vi;
    if (diag) z[i] = diag[i] * vi;
}

// dst = (Tout) src with src/dst offset by (k + ofs) * stride when indexed by a level state
template <typename Tin, typename Tout>
__global__ void k_copy_ind(const Tin *__restrict__ src, Tout *__restrict__ dst, int64_t n, const LevelState *st,
                           int64_t src_stride, int64_t dst_stride) {
    if (st && st->done) return;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = st ? st->k : 0;
    dst[(int64_t)k * dst_stride + i] = (Tout)src[(int64_t)k * src_stride + i];
}

template <typename T>
__global__ void k_sub(const T *__restrict__ b, T *__restrict__ r, int64_t n) {  // r = b - r
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - r[i];
}

__global__ void k_mul(const double *__restrict__ a, const double *__restrict__ w, double *__restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] * w[i];
}

// sum of squares into out (fixed grid, last block sums)
__global__ void __launch_bounds__(kThreads) k_sumsq(const double *__restrict__ r, int64_t n, double *partial,
                                                    unsigned *counter, double *out) {
    __shared__ double red[kThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double ss = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) ss = fma(r[i], r[i], ss);
    const double t = block_sum(ss, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
    if (!last_block(counter)) return;
    sum_partials(partial, 1, 1, out);
    if (threadIdx.x == 0) *counter = 0u;
}

// ------------------------------------------------------------ persistent A-solve
//
// One A-solve (GMRES(m) on A~ = A M^-1, M the 3x3 block diagonal of A, then
// x = M^-1 V y) as a single cooperative kernel: every block owns the nodes
// gid, gid + G*B, ... for the whole solve and the phases of an iteration are
// separated by grid barriers instead of kernel boundaries. Per iteration j:
//   P1  v_j = s u (s = 1/||u||, applied lazily), w = s A~ u (SELL-32 SpMV,
//       gathering u), partial dots V_l . w and w . w  -> barrier, h1, ||w||
//   test in the manner of Daniel, Gragg, Kaufman and Stewart: when
//   ||w - V h1||, from Pythagoras, is at least eta ||w|| (eta^2 = kPgEta2
//   for loose solves, 1/2 otherwise), one classical Gram-Schmidt pass is kept:
//   P2  w -= V h1; Givens and stopping test        -> barrier (w complete)
//   otherwise the second pass follows (CGS2):
//   P2  w -= V h1, partial dots V_l . w            -> barrier, h2
//   P3  w -= V h2, partial ||w||^2                 -> barrier; Givens, test
//   At the end of a cycle: y = R^-1 g, x += M^-1 V y and the restart
//   combination.
// After each barrier every block sums the per-block partials itself, in
// block order, and keeps its own copy of the Givens rotations, g and the
// current Hessenberg column: all blocks compute bitwise-identical values and
// take the same decisions, and no block waits on another's reduction. Block 0
// alone writes the Hessenberg columns (read back at the end of a cycle) and
// the level state. Partials are double-buffered by barrier parity, so a block
// never overwrites sums another block is still reading. Row-local vectors (V,
// w, x) are only touched by the thread that owns the node; values written by
// other blocks are read after a barrier.
// Every barrier wait is bounded (1 s): a block that runs out of time sets the
// abort word, every block then leaves, and the level state reports flag 8.

constexpr int kPgThreads = 512;
// eta^2 of the single-pass test for loose solves: 1e-6 in FP64 (norm to
// ~4e-10, orthogonality to ~2e-13), 1e-2 in FP32 (norm to ~1e-5,
// orthogonality to ~1e-6). Solves asked for rtol below kPgLoose<T> use the
// classical 1/2 (eta = 1/sqrt(2)), where the basis stays orthogonal to
// working precision.
template <typename T>
constexpr double kPgEta2 = sizeof(T) == 8 ? 1e-6 : 1e-2;
template <typename T>
constexpr double kPgLoose = sizeof(T) == 8 ? 1e-6 : 1e-3;
constexpr unsigned long long kBarrierNs = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One persistent GMRES level: vectors of NC values per node
template <typename T>
struct GmArgs {
    int64_t N;                 // nodes
    const T *b;
    T *x, *V, *U0, *U1;
    // flexible form: the operator stores P^-1 v_j in column j of Zb and the
    // solution update reads Zb instead of V (x += Z y); nullptr: x += P^-1 (V y)
    T *Zb = nullptr;
    double *H;                 // rotated Hessenberg columns (written by block 0)
    double *partial;           // 2 x [m + 1][grid], by barrier parity
    unsigned *bar;             // barrier words (arrivals, release, abort), shared by nested levels
    LevelState *st;
    int m, maxit;
    double rtol, atol;
    double it_fixed, it_unit;  // algorithmic bytes per iteration: fixed + passes x unit
    double eta2;               // single Gram-Schmidt pass when ||w - V h||^2 >= eta2 ||w||^2
};

// Chebyshev polynomial preconditioner of the A-solves (HYEL_APREC_CHEB):
// z = p(M^-1 A) M^-1 v, M the 3x3 block diagonal of A
template <typename T>
struct AChArgs {
    const float *Af;       // FP32 scaled A: the polynomial's products
    const T *A;            // scaled A of precision T: the A-solve's product
    const double *bounds;  // device [2]: estimated lmin, lmax
    int degree;
    T *zc, *r;             // [3N]
    float *d0, *d1;        // [3N]
};

// The A-solve: GMRES on A M^-1 (3 values per node), or on A p(M^-1 A) M^-1
template <typename T>
struct PgArgs {
    const int32_t *slice_ptr, *row_len, *col;
    const T *Am;                              // A~ values (nullptr: BF16 records)
    const uint4 *Am8;
    const uint16_t *Am1;
    const float *Ams;
    const T *jac;                             // [9][N] M^-1
    AChArgs<T> ac;                            // HYEL_APREC_CHEB only
    GmArgs<T> g;
};

// Arguments of the CG inner solve on A_sym (pg_cg_a below)
template <typename T>
struct CgArgs {
    const int32_t *slice_ptr, *row_len, *col;
    const T *Av;   // A_sym values
    const T *jac;  // [9][N] inverses of A_sym's diagonal blocks
    const T *b;
    T *x, *r, *u, *p, *s, *w;  // [3N]
    double *partial;           // 2 x [3][grid]
    unsigned *bar;
    LevelState *st;
    int64_t N;
    int maxit;
    double rtol, atol;
    double it_bytes;  // algorithmic bytes of one iteration
};

// Chebyshev polynomial preconditioner on the explicit S^: z = p(M^-1 S^) M^-1 v,
// M = diag(S^), the interval [lmax / ratio, lmax]
template <typename T, typename V = float>
struct ChebArgs {
    const int32_t *slice_ptr, *row_len, *col;  // S^ pattern (SELL-32)
    const V *val;                              // S^ values (FP32 in the solver: a preconditioner)
    const T *dinv;                             // [N] 1 / diag(S^)
    const double *bounds;                      // device [2]: estimated lmin, lmax
    double ratio;                              // > 0: lmin = lmax / ratio; 0: the estimate, clamped
    int degree;
    T *r;                                      // [N] residual, precision T
    V *d0, *d1;                                // [N] directions, precision V (the S^ product runs in V)
};

// The S-solve: GMRES on S P^-1 (1 value per node), S z = D z - C A^-1 B z,
// P^-1 = diag(S^)^-1 or the Chebyshev polynomial in S^
template <typename T>
struct SgArgs {
    const int32_t *slice_ptr, *row_len, *col;
    const T *B, *C, *D, *shat;
    T *xbar, *xtil;  // [3N] right-hand side and solution of the inner A-solve
    T *zc;           // [N] P^-1 v (Chebyshev only)
    ChebArgs<T> ch;
    CgArgs<T> cg;    // the inner A-solve by CG on A_sym (HYEL_INNER_CG_SYM only)
    GmArgs<T> g;
};

// Barrier words, each on its own 128-byte line: arrivals (they only grow
// within a launch), release (the number of completed barriers), abort. The
// fourth line (kBarCtl, copied from the context's control line before every
// launch, see bar_reset) holds the wait limit in ns (64-bit; 0 = kBarrierNs),
// the injected fault (a value b + 1 makes block b skip one arrival; the block
// clears it in the context's line, whose address is the 64-bit word at
// kBarCtl + 4, so one launch takes it) (hyel_inject_fault).

// Grid barrier number `phase` (then phase + 1). The last block to arrive
// releases the others; a wait is bounded by the limit of the control line
// (kBarrierNs by default). false: the wait ran out of time or a block gave up
// (every block then leaves). The fences around the wait make writes issued
// before the barrier by any block visible to ordinary loads of every thread
// of the block after it.
__device__ bool pg_barrier(unsigned *bw, unsigned &phase) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        volatile unsigned *vb = bw;
        int ok = 1;
        const unsigned me = blockIdx.x + 1u;
        unsigned *src = reinterpret_cast<unsigned *>(
            (uintptr_t)*reinterpret_cast<volatile unsigned long long *>(bw + kBarCtl + 4));
        if (vb[kBarCtl + 2] == me && src && atomicCAS(src + 2, me, 0u) == me) {
            // injected fault, withdrawn at its source so that one launch takes
            // it: this block leaves the barrier without arriving, and every
            // other block's wait runs into its limit
            vb[kBarCtl + 2] = 0u;
        } else {
        const unsigned target = (phase + 1u) * gridDim.x;
        const unsigned prev = atomicAdd(&bw[kBarArrive], 1u);
        unsigned long long limit = *reinterpret_cast<volatile unsigned long long *>(bw + kBarCtl);
        if (limit == 0ull) limit = kBarrierNs;
        if (prev + 1u == target) {
            __threadfence();
            atomicExch(&bw[kBarRelease], phase + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (vb[kBarRelease] < phase + 1u) {
                __nanosleep(32);
                if (vb[kBarAbort] != 0u || global_ns() - t0 > limit) {
                    atomicExch(&bw[kBarAbort], 1u);
                    ok = 0;
                    break;
                }
            }
        }
        }
        if (vb[kBarAbort] != 0u) ok = 0;
        s_ok = ok;
        __threadfence();
    }
    __syncthreads();
    phase += 1u;
    return s_ok != 0;
}

// Sums over the grid's partials p[k * G + block] (k < nk) in block order,
// one warp per column, lanes striding over the blocks (coalesced).
__device__ __forceinline__ void pg_sum(const double *p, int nk, double *out) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int G = gridDim.x;
    for (int k = warp; k < nk; k += nw) {
        double s = 0.0;
        for (int b = lane; b < G; b += 32) s += p[(int64_t)k * G + b];
        s = warp_sum_d(s);
        if (lane == 0) out[k] = s;
    }
}

// Nodes owned by the calling thread: block b holds the contiguous 32-row
// slices [S b / G, S (b+1) / G) (S slices, G blocks), its warps take them in
// turn and lane t the row 32 s + t. Every phase uses this map, so row-local
// data never cross threads, and with G a multiple of the SM count every SM
// gets the same number of slices to within one per block.
#define PG_FOR_OWN_NODES(N, i)                                                                   \
    for (int64_t pg_s = ((((N) + 31) >> 5) * blockIdx.x) / gridDim.x + (threadIdx.x >> 5),       \
                 pg_e = ((((N) + 31) >> 5) * (blockIdx.x + 1)) / gridDim.x;                      \
         pg_s < pg_e; pg_s += (blockDim.x >> 5))                                                 \
        for (int64_t i = pg_s * 32 + (threadIdx.x & 31); i < (N); i = (N))

// Warp sums of eight values per lane by reduce-scatter (9 adds, 9 shuffles):
// afterwards lane l holds, in v[0], the warp total of value (l >> 2) & 7.
template <typename T>
__device__ __forceinline__ void warp_reduce8(T v[8]) {
    const int lane = threadIdx.x & 31;
    const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const T keep = h16 ? v[4 + k] : v[k], send = h16 ? v[k] : v[4 + k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const T keep = h8 ? v[2 + k] : v[k], send = h8 ? v[k] : v[2 + k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    {
        const T keep = h4 ? v[1] : v[0], send = h4 ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Block sum of one value per thread: warp sums in T, then the warps' sums in
// double (thread 0 gets the result).
template <typename T>
__device__ __forceinline__ double pg_block_sum(T v, double *red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q];
    __syncthreads();
    return t;
}

// Partial dots V_l . w (l < nv), and w . w as column nv when self, of this
// block's nodes into partial[l][block]; sums within a warp in T, across the
// block's warps in double.
template <typename T, int NC>
__device__ void pg_dots(const T *V, const T *w, int64_t N, int nv, bool self, double *partial) {
    __shared__ double red[kPgThreads / 32][KC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = NC * N;
    const int nk = nv + (self ? 1 : 0);
    for (int k0 = 0; k0 < nk; k0 += KC) {
        const int kc = min(KC, nk - k0);
        T acc[KC];
#pragma unroll
        for (int c = 0; c < KC; c++) acc[c] = 0;
        PG_FOR_OWN_NODES(N, i) {
            T wi[NC];
#pragma unroll
            for (int r = 0; r < NC; r++) wi[r] = w[NC * i + r];
#pragma unroll
            for (int c = 0; c < KC; c++)
                if (c < kc) {
                    const T *v = k0 + c < nv ? V + (int64_t)(k0 + c) * n + NC * i : w + NC * i;
#pragma unroll
                    for (int r = NC - 1; r >= 0; r--) acc[c] = fma(v[r], wi[r], acc[c]);
                }
        }
        if (kc == 1) {
            const T s = warp_sum(acc[0]);
            if (lane == 0) red[warp][0] = (double)s;
        } else {
            warp_reduce8<T>(acc);
            if ((lane & 3) == 0) red[warp][lane >> 2] = (double)acc[0];
        }
        __syncthreads();
        if (threadIdx.x < kc) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < kPgThreads / 32; q++) s += red[q][threadIdx.x];
            partial[(int64_t)(k0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
        }
        __syncthreads();
    }
}

// w -= V h (h in shared memory, l < nk) on this block's nodes; returns sum w^2
// (accumulated in T per thread)
template <typename T, int NC>
__device__ T pg_axpy(const T *V, T *w, int64_t N, int nk, const T *h) {
    const int64_t n = NC * N;
    T ss = 0;
    PG_FOR_OWN_NODES(N, i) {
        T wi[NC];
#pragma unroll
        for (int r = 0; r < NC; r++) wi[r] = w[NC * i + r];
        for (int l = 0; l < nk; l++) {
            const T *v = V + (int64_t)l * n + NC * i;
            const T hl = h[l];
#pragma unroll
            for (int r = 0; r < NC; r++) wi[r] = fma(-v[r], hl, wi[r]);
        }
#pragma unroll
        for (int r = NC - 1; r >= 0; r--) {
            w[NC * i + r] = wi[r];
            ss = fma(wi[r], wi[r], ss);
        }
    }
    return ss;
}

template <typename T, bool H16>
__device__ __forceinline__ void pg_row(const PgArgs<T> &a, int64_t i, const T *u, T &y0, T &y1, T &y2) {
    const int t = (int)(i & 31);
    const int64_t b0 = a.slice_ptr[i >> 5];
    const int len = a.row_len[i];
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 4
    for (int jb = 0; jb < len; jb++) {
        const int64_t q = (b0 + jb) * 32 + t;
        const int64_t c = __ldg(a.col + q);
        const T x0 = u[3 * c], x1 = u[3 * c + 1], x2 = u[3 * c + 2];
        if constexpr (H16) {
            const uint4 w = __ldg(a.Am8 + q);
            const unsigned e8 = __ldg(a.Am1 + q);
            const float s = __ldg(a.Ams + q);
            float t0 = __uint_as_float(w.x << 16) * x0;
            t0 = fmaf(__uint_as_float(w.x & 0xffff0000u), x1, t0);
            t0 = fmaf(__uint_as_float(w.y << 16), x2, t0);
            float t1 = __uint_as_float(w.y & 0xffff0000u) * x0;
            t1 = fmaf(__uint_as_float(w.z << 16), x1, t1);
            t1 = fmaf(__uint_as_float(w.z & 0xffff0000u), x2, t1);
            float t2 = __uint_as_float(w.w << 16) * x0;
            t2 = fmaf(__uint_as_float(w.w & 0xffff0000u), x1, t2);
            t2 = fmaf(__uint_as_float(e8 << 16), x2, t2);
            a0 = fmaf(s, t0, a0);
            a1 = fmaf(s, t1, a1);
            a2 = fmaf(s, t2, a2);
        } else {
            const T *Ab = a.Am + (q >> 5) * 288 + t;
            a0 = fma(__ldg(Ab + 0), x0, a0);
            a0 = fma(__ldg(Ab + 32), x1, a0);
            a0 = fma(__ldg(Ab + 64), x2, a0);
            a1 = fma(__ldg(Ab + 96), x0, a1);
            a1 = fma(__ldg(Ab + 128), x1, a1);
            a1 = fma(__ldg(Ab + 160), x2, a1);
            a2 = fma(__ldg(Ab + 192), x0, a2);
            a2 = fma(__ldg(Ab + 224), x1, a2);
            a2 = fma(__ldg(Ab + 256), x2, a2);
        }
    }
    y0 = a0;
    y1 = a1;
    y2 = a2;
}

// One GMRES solve on the calling grid (all blocks of a cooperative launch),
// NC values per node. op(u, s, w, phase) sets w = Op(s u) on the block's
// nodes (it may run grid barriers of its own, in every block alike);
// xupd(i, u) adds the preconditioned u = (V y)_i to x_i. phase counts the grid
// barriers passed so far. false: a barrier gave up.
constexpr double kChebMaxRatio = 1000.0, kChebMinRatio = 1.5;  // clamp of the estimated lmax / lmin

// z = p(M^-1 S^) M^-1 (vs v) over the grid: `degree` steps of the Chebyshev
// iteration for S^ z = vs v from z = 0, Jacobi-preconditioned, on
// [lmin, lmax] (theta, delta the interval's centre and half-width,
// sigma = theta / delta):
//   r = vs v, d = M^-1 r / theta, rho = 1 / sigma; then degree - 1 times
//   z += d; r -= S^ d; rho' = 1 / (2 sigma - rho);
//   d = rho' rho d + (2 rho' / delta) M^-1 r; and a last z += d.
// add: z += instead of z =. v may alias ch.r (each thread reads its own rows
// before writing them). The directions d and the S^ d product are kept in the
// value type V (FP32 in the solver: on this GPU an FP64 operation, a
// conversion included, costs tens of FP32 ones), r and z in T; a fixed
// operator up to V's rounding, which a preconditioner tolerates. Ends with a
// grid barrier, so z and the scratch are complete for every block.
template <typename T, typename V>
__device__ bool pg_cheb(const ChebArgs<T, V> &ch, int64_t N, const T *v, T vs, T *z, bool add, unsigned *bar,
                        unsigned &phase) {
    const double lmax = ch.bounds[1];
    const double lmin = ch.ratio > 0.0 ? lmax / ch.ratio
                                       : fmin(fmax(ch.bounds[0], lmax / kChebMaxRatio), lmax / kChebMinRatio);
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    {
        const T it = (T)(1.0 / theta);
        PG_FOR_OWN_NODES(N, i) {
            const T r = v[i] * vs;
            ch.r[i] = r;
            const V d = (V)(__ldg(ch.dinv + i) * r * it);
            ch.d0[i] = d;
            z[i] = add ? z[i] + (T)d : (T)d;
        }
    }
    if (!pg_barrier(bar, phase)) return false;
    V *dc = ch.d0, *dn = ch.d1;
    for (int k = 1; k < ch.degree; k++) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        const T a1 = (T)(rho_n * rho), a2 = (T)(2.0 * rho_n / delta);
        PG_FOR_OWN_NODES(N, i) {
            const int t = (int)(i & 31);
            const int64_t b0 = __ldg(ch.slice_ptr + (i >> 5));
            const int len = __ldg(ch.row_len + i);
            V sd = 0;
            for (int p = 0; p < len; p++) {
                const int64_t q = (b0 + p) * 32 + t;
                sd = fma(__ldg(ch.val + q), dc[__ldg(ch.col + q)], sd);
            }
            const T r = ch.r[i] - (T)sd;
            ch.r[i] = r;
            const V d = (V)(a1 * (T)dc[i] + a2 * (__ldg(ch.dinv + i) * r));
            dn[i] = d;
            z[i] += (T)d;
        }
        rho = rho_n;
        if (!pg_barrier(bar, phase)) return false;
        V *tmp = dc;
        dc = dn;
        dn = tmp;
    }
    return true;
}

// A no-op end-of-cycle step
struct PgNoEnd {
    __device__ bool operator()(unsigned &) const { return true; }
};

template <typename T, int NC, typename Op, typename XUpd, typename XEnd = PgNoEnd>
__device__ bool pg_gmres(const GmArgs<T> &a, unsigned &phase, Op &&op, XUpd &&xupd, XEnd &&xend = XEnd()) {
    // per-block copies of the small GMRES state (identical in every block)
    __shared__ double s_cs[kMaxK], s_sn[kMaxK], s_g[kMaxK + 1], s_col[kMaxK + 2], s_tmp[kMaxK + 2];
    __shared__ T hs[kMaxK + 2];
    __shared__ double s_sc[4];  // 0: squared norm, 1: next scale, 2: 1 / h_{j+1,j}, 3: tol
    __shared__ int s_fl[5];     // 0: done, 1: stop, 2: y usable, 3: total iterations, 4: second pass
    const int64_t N = a.N, n = NC * N;
    const int m = a.m;
    const int G = gridDim.x;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;  // writes the level state and H
    LevelState *st = a.st;
    auto pbuf = [&](unsigned ph) { return a.partial + (size_t)(ph & 1u) * G * (m + 1); };

    auto abort_out = [&]() {
        if (threadIdx.x == 0) {
            atomicOr(&st->flags, 8);
            atomicOr(&st->status_any, 8);
            st->stop = 1;
        }
        return false;
    };

    // ---- start: x = 0, beta = ||b||
    {
        T ss = 0;
        PG_FOR_OWN_NODES(N, i)
#pragma unroll
            for (int r = 0; r < NC; r++) {
                const T v = a.b[NC * i + r];
                a.x[NC * i + r] = 0;
                ss = fma(v, v, ss);
            }
        __shared__ double red1[kPgThreads / 32];
        const double tb = pg_block_sum<T>(ss, red1);
        if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
    }
    if (!pg_barrier(a.bar, phase)) return abort_out();
    pg_sum(pbuf(phase - 1), 1, s_sc);
    __syncthreads();
    if (threadIdx.x == 0) {
        const double beta = sqrt(s_sc[0]);
        const double tol = fmax(a.rtol * beta, a.atol);
        const int nan = isfinite(beta) ? 0 : 1;
        const int conv = (!nan && beta <= tol) ? 1 : 0;
        s_sc[1] = beta > 0.0 ? 1.0 / beta : 0.0;
        s_sc[3] = tol;
        s_fl[1] = (conv || nan) ? 1 : 0;
        s_fl[3] = 0;
        s_g[0] = beta;
        for (int l = 1; l <= m; l++) s_g[l] = 0.0;
        if (lead) {
            st->k = 0;
            st->total = 0;
            st->cycles = 0;
            st->maxit = a.maxit;
            st->m = m;
            st->beta = beta;
            st->bnorm = beta;
            st->tol = tol;
            st->res = beta;
            st->inv_scale = s_sc[1];
            st->flags = nan;
            st->converged = conv;
            st->stop = s_fl[1];
            st->done = s_fl[1];
            st->yok = 0;
            if (s_fl[1]) {
                st->solves += 1;
                st->status_any |= nan;
                st->stop = 2;
            }
        }
    }
    __syncthreads();
    if (s_fl[1]) return true;

    const T *uin = a.b;
    T *uout = a.U0;
    T s = (T)s_sc[1];
    int j = 0;
    for (;;) {
        // ---- P1: v_j = s u; w = s A~ u; dots with V_0..V_j
        T *Vj = a.V + (int64_t)j * n;
        PG_FOR_OWN_NODES(N, i)
#pragma unroll
            for (int r = 0; r < NC; r++) Vj[NC * i + r] = uin[NC * i + r] * s;
        if (!op(uin, s, uout, phase, j)) return abort_out();
        pg_dots<T, NC>(a.V, uout, N, j + 1, true, pbuf(phase));
        if (!pg_barrier(a.bar, phase)) return abort_out();
        pg_sum(pbuf(phase - 1), j + 2, s_col);  // h1, and ||w||^2 in s_col[j + 1]
        __syncthreads();
        // DGKS-type test: one Gram-Schmidt pass suffices when it keeps at
        // least eta of ||w|| (the norm after the pass by Pythagoras, accurate
        // to about eps / eta^2; orthogonality to about eps / eta)
        if (threadIdx.x == 0) {
            const double ww = s_col[j + 1];
            double hh = 0.0;
            for (int l = 0; l <= j; l++) hh += s_col[l] * s_col[l];
            const double w2 = ww - hh;
            s_fl[4] = (w2 >= a.eta2 * ww) ? 0 : 1;
            s_sc[0] = w2;
        }
        __syncthreads();
        for (int l = threadIdx.x; l <= j; l += blockDim.x) hs[l] = (T)s_col[l];
        __syncthreads();
        const bool reorth = s_fl[4] != 0;
        if (!reorth) {
            // ---- P2: w -= V h1, the new direction (norm from the test above)
            pg_axpy<T, NC>(a.V, uout, N, j + 1, hs);
        } else {
            // ---- P2: w -= V h1; dots again (second Gram-Schmidt pass)
            pg_axpy<T, NC>(a.V, uout, N, j + 1, hs);
            pg_dots<T, NC>(a.V, uout, N, j + 1, false, pbuf(phase));
            if (!pg_barrier(a.bar, phase)) return abort_out();
            pg_sum(pbuf(phase - 1), j + 1, s_tmp);  // h2
            __syncthreads();
            for (int l = threadIdx.x; l <= j; l += blockDim.x) {
                hs[l] = (T)s_tmp[l];
                s_col[l] += s_tmp[l];
            }
            __syncthreads();
            // ---- P3: w -= V h2; ||w||
            {
                __shared__ double red1[kPgThreads / 32];
                const double tb = pg_block_sum<T>(pg_axpy<T, NC>(a.V, uout, N, j + 1, hs), red1);
                if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
            }
            if (!pg_barrier(a.bar, phase)) return abort_out();
            pg_sum(pbuf(phase - 1), 1, s_sc);
            __syncthreads();
        }
        // ---- Givens step and stopping test, redundantly in every block
        if (threadIdx.x == 0) {
            const double hn = sqrt(fmax(s_sc[0], 0.0));
            for (int l = 0; l < j; l++) {
                const double a0 = s_col[l], a1 = s_col[l + 1];
                s_col[l] = s_cs[l] * a0 + s_sn[l] * a1;
                s_col[l + 1] = -s_sn[l] * a0 + s_cs[l] * a1;
            }
            const double al = s_col[j];
            double c, s2, r;
            if (hn == 0.0) {
                c = 1.0;
                s2 = 0.0;
                r = al;
            } else {
                r = sqrt(al * al + hn * hn);
                c = al / r;
                s2 = hn / r;
            }
            s_cs[j] = c;
            s_sn[j] = s2;
            s_col[j] = r;
            s_col[j + 1] = 0.0;
            const double gj = s_g[j];
            s_g[j] = c * gj;
            s_g[j + 1] = -s2 * gj;
            const double res = fabs(s_g[j + 1]);
            const int total = s_fl[3] + 1;
            s_fl[3] = total;
            int done = 0, stop = 0, flags = 0, conv = 0;
            if (!isfinite(res) || !isfinite(hn)) {
                flags = 1;
                done = stop = 1;
            } else if (r == 0.0) {
                flags = 2;
                done = stop = 1;
            } else if (res <= s_sc[3]) {
                conv = 1;
                done = stop = 1;
            } else if (hn == 0.0) {
                flags = 2;
                done = stop = 1;
            } else if (total >= a.maxit) {
                done = stop = 1;
            } else if (j + 1 == m) {
                done = 1;
            }
            s_fl[0] = done;
            s_fl[1] = stop;
            s_fl[2] = done && isfinite(res) && isfinite(hn) && r != 0.0;
            s_sc[1] = hn > 0.0 ? 1.0 / hn : 0.0;
            s_sc[2] = s_sc[1];
            if (lead) {
                for (int l = 0; l <= j + 1; l++) a.H[(int64_t)j * (m + 1) + l] = s_col[l];
                st->k = j + 1;
                st->total = total;
                st->res = res;
                st->inv_scale = s_sc[1];
                // one Gram-Schmidt pass: 2 (j+1) + 6 vector passes; two: 4 (j+1) + 10
                st->alg_bytes += a.it_fixed + (reorth ? 4.0 * (j + 1) + 10.0 : 2.0 * (j + 1) + 6.0) * a.it_unit;
                st->flags |= flags;
                if (conv) st->converged = 1;
                st->done = done;
                st->stop = stop;
                st->yok = s_fl[2];
            }
        }
        __syncthreads();
        if (!s_fl[0]) {
            // next iteration: u = w, scaled lazily by 1 / h_{j+1,j}; after a
            // single pass w was finished after the last barrier
            if (!reorth && !pg_barrier(a.bar, phase)) return abort_out();
            s = (T)s_sc[1];
            uin = uout;
            uout = (uout == a.U0) ? a.U1 : a.U0;
            j += 1;
            continue;
        }
        // ---- end of a cycle: y = R^-1 g over the k = j+1 columns (columns
        // < j from H, written by block 0 before earlier barriers; column j here)
        const int k = j + 1;
        if (s_fl[2]) {
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                for (int i = k - 1; i >= 0; i--) {
                    double sacc = 0.0;
                    for (int l = i + 1 + lane; l < k; l += 32)
                        sacc += (l == j ? s_col[i] : a.H[(int64_t)l * (m + 1) + i]) * s_tmp[l];
                    sacc = warp_sum_d(sacc);
                    if (lane == 0) s_tmp[i] = (s_g[i] - sacc) / (i == j ? s_col[i] : a.H[(int64_t)i * (m + 1) + i]);
                    __syncwarp();
                }
            }
            __syncthreads();
            for (int l = threadIdx.x; l < k; l += blockDim.x) hs[l] = (T)s_tmp[l];
            __syncthreads();
            // x += M^-1 V y (or x += Z y in the flexible form)
            const T *XB = a.Zb ? a.Zb : a.V;
            PG_FOR_OWN_NODES(N, i) {
                T u[NC];
#pragma unroll
                for (int r = 0; r < NC; r++) u[r] = 0;
                for (int l = 0; l < k; l++) {
                    const T *v = XB + (int64_t)l * n + NC * i;
#pragma unroll
                    for (int r = 0; r < NC; r++) u[r] = fma(v[r], hs[l], u[r]);
                }
                xupd(i, u);
            }
            __syncthreads();
            // a preconditioner that is not row-local finishes x here (every
            // block takes this branch: s_fl is the same in all of them)
            if (!xend(phase)) return abort_out();
        }
        if (s_fl[1]) {
            if (lead) {
                st->its += s_fl[3];
                st->solves += 1;
                st->status_any |= st->flags | ((!st->converged && !st->flags) ? 4 : 0);
                st->stop = 2;
            }
            return true;
        }
        // ---- restart: c = G_0^T ... G_{k-1}^T (g_k e_k), residual norm |g_k|;
        // r = sum_{l<k} c_l V_l + c_k (w / h_{k,k-1}), unnormalised
        if (threadIdx.x == 0) {
            double carry = s_g[k];
            for (int i = k - 1; i >= 0; i--) {
                s_tmp[i + 1] = s_cs[i] * carry;
                carry = -s_sn[i] * carry;
            }
            s_tmp[0] = carry;
            const double beta = fabs(s_g[k]);
            s_sc[1] = beta > 0.0 ? 1.0 / beta : 0.0;
            s_g[0] = beta;
            for (int l = 1; l <= m; l++) s_g[l] = 0.0;
            if (lead) {
                st->k = 0;
                st->done = 0;
                st->cycles += 1;
                st->beta = beta;
                st->res = beta;
                st->inv_scale = s_sc[1];
            }
        }
        __syncthreads();
        for (int l = threadIdx.x; l <= k; l += blockDim.x) hs[l] = (T)s_tmp[l];
        __syncthreads();
        const T hinv = (T)s_sc[2];
        T *unew = (uout == a.U0) ? a.U1 : a.U0;
        PG_FOR_OWN_NODES(N, i) {
            T rr[NC];
#pragma unroll
            for (int r = 0; r < NC; r++) rr[r] = uout[NC * i + r] * hinv * hs[k];
            for (int l = 0; l < k; l++) {
                const T *v = a.V + (int64_t)l * n + NC * i;
#pragma unroll
                for (int r = 0; r < NC; r++) rr[r] = fma(v[r], hs[l], rr[r]);
            }
#pragma unroll
            for (int r = 0; r < NC; r++) unew[NC * i + r] = rr[r];
        }
        if (!pg_barrier(a.bar, phase)) return abort_out();
        s = (T)s_sc[1];
        uin = unew;
        uout = (unew == a.U0) ? a.U1 : a.U0;
        j = 0;
    }
}

// Row i of V-valued 3x3 blocks (SELL-32 layout of As) times u: y = (Av u)_i
template <typename V, typename X, typename Y>
__device__ __forceinline__ void block_row(const int32_t *slice_ptr, const int32_t *row_len, const int32_t *col,
                                          const V *Av, int64_t i, const X *u, Y &y0, Y &y1, Y &y2) {
    const int t = (int)(i & 31);
    const int64_t b0 = __ldg(slice_ptr + (i >> 5));
    const int len = __ldg(row_len + i);
    Y a0 = 0, a1 = 0, a2 = 0;
    for (int jb = 0; jb < len; jb++) {
        const int64_t b = b0 + jb;
        const int64_t c = __ldg(col + b * 32 + t);
        const Y x0 = (Y)u[3 * c], x1 = (Y)u[3 * c + 1], x2 = (Y)u[3 * c + 2];
        const V *Ab = Av + (b * 9) * 32 + t;
        a0 = fma((Y)__ldg(Ab), x0, fma((Y)__ldg(Ab + 32), x1, fma((Y)__ldg(Ab + 64), x2, a0)));
        a1 = fma((Y)__ldg(Ab + 96), x0, fma((Y)__ldg(Ab + 128), x1, fma((Y)__ldg(Ab + 160), x2, a1)));
        a2 = fma((Y)__ldg(Ab + 192), x0, fma((Y)__ldg(Ab + 224), x1, fma((Y)__ldg(Ab + 256), x2, a2)));
    }
    y0 = a0;
    y1 = a1;
    y2 = a2;
}

// z = p(M^-1 A) M^-1 v over the grid (the recurrence of pg_cheb with the 3x3
// block-Jacobi M): the directions and the A d products in FP32 with the FP32
// copy of A, r and z in T. v may alias a.ac.r. Ends with a grid barrier.
template <typename T>
__device__ bool pg_cheb3(const PgArgs<T> &a, const T *v, T *z, bool add, unsigned &phase) {
    const AChArgs<T> &ch = a.ac;
    const int64_t N = a.g.N;
    const double lmax = ch.bounds[1];
    const double lmin = fmin(fmax(ch.bounds[0], lmax / kChebMaxRatio), lmax / kChebMinRatio);
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
    double rho = 1.0 / sigma;
    auto minv = [&](int64_t i, const T (&r)[3], T (&m)[3]) {
#pragma unroll
        for (int k = 0; k < 3; k++)
            m[k] = __ldg(a.jac + (3 * k) * N + i) * r[0] + __ldg(a.jac + (3 * k + 1) * N + i) * r[1] +
                   __ldg(a.jac + (3 * k + 2) * N + i) * r[2];
    };
    {
        const T it = (T)(1.0 / theta);
        PG_FOR_OWN_NODES(N, i) {
            T r[3], m[3];
#pragma unroll
            for (int k = 0; k < 3; k++) r[k] = v[3 * i + k];
            minv(i, r, m);
#pragma unroll
            for (int k = 0; k < 3; k++) {
                ch.r[3 * i + k] = r[k];
                const float d = (float)(m[k] * it);
                ch.d0[3 * i + k] = d;
                z[3 * i + k] = add ? z[3 * i + k] + (T)d : (T)d;
            }
        }
    }
    if (!pg_barrier(a.g.bar, phase)) return false;
    float *dc = ch.d0, *dn = ch.d1;
    for (int k = 1; k < ch.degree; k++) {
        const double rho_n = 1.0 / (2.0 * sigma - rho);
        const T a1 = (T)(rho_n * rho), a2 = (T)(2.0 * rho_n / delta);
        PG_FOR_OWN_NODES(N, i) {
            float s0, s1, s2;
            block_row<float, float, float>(a.slice_ptr, a.row_len, a.col, ch.Af, i, dc, s0, s1, s2);
            T r[3], m[3];
            r[0] = ch.r[3 * i] - (T)s0;
            r[1] = ch.r[3 * i + 1] - (T)s1;
            r[2] = ch.r[3 * i + 2] - (T)s2;
            minv(i, r, m);
#pragma unroll
            for (int q = 0; q < 3; q++) {
                ch.r[3 * i + q] = r[q];
                const float d = (float)(a1 * (T)dc[3 * i + q] + a2 * m[q]);
                dn[3 * i + q] = d;
                z[3 * i + q] += (T)d;
            }
        }
        rho = rho_n;
        if (!pg_barrier(a.g.bar, phase)) return false;
        float *tmp = dc;
        dc = dn;
        dn = tmp;
    }
    return true;
}

// The A-solve on the calling grid: operator A M^-1 (phase 1 of an iteration is
// the SELL-32 SpMV, gathering u), x += M^-1 V y; with ACH the operator is
// A p(M^-1 A) M^-1 (the polynomial's grid phases, then the SpMV with the
// unfolded A on z) and x += p(M^-1 A) M^-1 V y.
template <typename T, bool H16, bool ACH = false>
__device__ bool pg_gmres_a(const PgArgs<T> &a, unsigned &phase) {
    const int64_t N = a.g.N;
    auto op = [&](const T *u, T sc, T *w, unsigned &ph, int) {
        if constexpr (ACH) {
            if (!pg_cheb3<T>(a, u, a.ac.zc, false, ph)) return false;
            PG_FOR_OWN_NODES(N, i) {
                T y0, y1, y2;
                block_row<T, T, T>(a.slice_ptr, a.row_len, a.col, a.ac.A, i, a.ac.zc, y0, y1, y2);
                w[3 * i] = y0 * sc;
                w[3 * i + 1] = y1 * sc;
                w[3 * i + 2] = y2 * sc;
            }
        } else {
            PG_FOR_OWN_NODES(N, i) {
                T y0, y1, y2;
                pg_row<T, H16>(a, i, u, y0, y1, y2);
                w[3 * i] = y0 * sc;
                w[3 * i + 1] = y1 * sc;
                w[3 * i + 2] = y2 * sc;
            }
        }
        return true;
    };
    if constexpr (ACH) {
        auto xupd = [&](int64_t i, const T (&u)[3]) {
#pragma unroll
            for (int r = 0; r < 3; r++) a.ac.r[3 * i + r] = u[r];
        };
        auto xend = [&](unsigned &ph) { return pg_cheb3<T>(a, a.ac.r, a.g.x, true, ph); };
        return pg_gmres<T, 3>(a.g, phase, op, xupd, xend);
    } else {
        auto xupd = [&](int64_t i, const T (&u)[3]) {
#pragma unroll
            for (int r = 0; r < 3; r++)
                a.g.x[3 * i + r] += __ldg(a.jac + (3 * r) * N + i) * u[0] + __ldg(a.jac + (3 * r + 1) * N + i) * u[1] +
                                    __ldg(a.jac + (3 * r + 2) * N + i) * u[2];
        };
        return pg_gmres<T, 3>(a.g, phase, op, xupd);
    }
}

template <typename T, bool H16, bool ACH>
__global__ void __launch_bounds__(kPgThreads, 2) k_gmres_a(PgArgs<T> a) {
    unsigned phase = 0u;  // the barrier words are cleared before every launch
    pg_gmres_a<T, H16, ACH>(a, phase);
}

// The inner A-solve on the symmetrized block (row-major 3x3 blocks of
// A_sym = (A + A^T)/2 in the SELL-32 layout): preconditioned CG with the
// block-Jacobi M = diag blocks of A_sym, in the single-reduction form of
// Chronopoulos and Gear (1989): per iteration u = M^-1 r (row-local), a grid
// barrier, w = A_sym u with the three dots (r, u), (w, u), (r, r) reduced
// together, a grid barrier; then
//   beta = g' / g, alpha = g' / (d - beta g' / alpha),
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// Stops at ||r|| <= max(rtol ||b||, atol) or maxit. Every block computes the
// scalars from the same sums, so all take the same decisions.
template <typename T>
__device__ __forceinline__ void cg_minv(const CgArgs<T> &a, int64_t i) {
    const int64_t N = a.N;
    const T r0 = a.r[3 * i], r1 = a.r[3 * i + 1], r2 = a.r[3 * i + 2];
#pragma unroll
    for (int k = 0; k < 3; k++)
        a.u[3 * i + k] = __ldg(a.jac + (3 * k) * N + i) * r0 + __ldg(a.jac + (3 * k + 1) * N + i) * r1 +
                         __ldg(a.jac + (3 * k + 2) * N + i) * r2;
}

// w_i = (A_sym u)_i; returns the row's contributions to (r, u), (w, u), (r, r)
template <typename T>
__device__ __forceinline__ void cg_row(const CgArgs<T> &a, int64_t i, T &g, T &d, T &q) {
    const int t = (int)(i & 31);
    const int64_t b0 = __ldg(a.slice_ptr + (i >> 5));
    const int len = __ldg(a.row_len + i);
    T y0 = 0, y1 = 0, y2 = 0;
    for (int jb = 0; jb < len; jb++) {
        const int64_t b = b0 + jb;
        const int64_t c = __ldg(a.col + b * 32 + t);
        const T u0 = a.u[3 * c], u1 = a.u[3 * c + 1], u2 = a.u[3 * c + 2];
        const T *Ab = a.Av + (b * 9) * 32 + t;
        y0 = fma(__ldg(Ab), u0, fma(__ldg(Ab + 32), u1, fma(__ldg(Ab + 64), u2, y0)));
        y1 = fma(__ldg(Ab + 96), u0, fma(__ldg(Ab + 128), u1, fma(__ldg(Ab + 160), u2, y1)));
        y2 = fma(__ldg(Ab + 192), u0, fma(__ldg(Ab + 224), u1, fma(__ldg(Ab + 256), u2, y2)));
    }
    a.w[3 * i] = y0;
    a.w[3 * i + 1] = y1;
    a.w[3 * i + 2] = y2;
    const T r0 = a.r[3 * i], r1 = a.r[3 * i + 1], r2 = a.r[3 * i + 2];
    const T v0 = a.u[3 * i], v1 = a.u[3 * i + 1], v2 = a.u[3 * i + 2];
    g = fma(r0, v0, fma(r1, v1, fma(r2, v2, g)));
    d = fma(y0, v0, fma(y1, v1, fma(y2, v2, d)));
    q = fma(r0, r0, fma(r1, r1, fma(r2, r2, q)));
}

template <typename T>
__device__ bool pg_cg_a(const CgArgs<T> &a, unsigned &phase) {
    __shared__ double red1[kPgThreads / 32];
    __shared__ double s_red[3];
    const int64_t N = a.N;
    const int G = gridDim.x;
    LevelState *st = a.st;
    auto pbuf = [&](unsigned ph) { return a.partial + (size_t)(ph & 1u) * 3 * G; };
    auto abort_out = [&]() {
        if (threadIdx.x == 0) {
            atomicOr(&st->flags, 8);
            atomicOr(&st->status_any, 8);
            st->stop = 1;
        }
        return false;
    };
    // one grid reduction of three values (then every block holds the sums in s_red)
    auto reduce3 = [&](T v0, T v1, T v2) {
        const double t0 = pg_block_sum<T>(v0, red1);
        if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = t0;
        const double t1 = pg_block_sum<T>(v1, red1);
        if (threadIdx.x == 0) pbuf(phase)[G + blockIdx.x] = t1;
        const double t2 = pg_block_sum<T>(v2, red1);
        if (threadIdx.x == 0) pbuf(phase)[2 * G + blockIdx.x] = t2;
        if (!pg_barrier(a.bar, phase)) return false;
        pg_sum(pbuf(phase - 1), 3, s_red);
        __syncthreads();
        return true;
    };
    // x = 0, r = b, u = M^-1 r
    PG_FOR_OWN_NODES(N, i) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            a.x[3 * i + k] = 0;
            a.r[3 * i + k] = a.b[3 * i + k];
        }
        cg_minv(a, i);
    }
    if (!pg_barrier(a.bar, phase)) return abort_out();
    {
        T g = 0, d = 0, q = 0;
        PG_FOR_OWN_NODES(N, i) cg_row(a, i, g, d, q);
        if (!reduce3(g, d, q)) return abort_out();
    }
    double gam = s_red[0], del = s_red[1];
    const double bnorm = sqrt(s_red[2]);
    const double tol = fmax(a.rtol * bnorm, a.atol);
    int k = 0, flags = 0, conv = 0;
    double alpha = 0.0, beta = 0.0;
    if (!isfinite(bnorm) || !isfinite(gam) || !isfinite(del))
        flags = 1;
    else if (bnorm <= tol)
        conv = 1;
    else if (!(del != 0.0))
        flags = 2;
    else
        alpha = gam / del;
    while (!flags && !conv) {
        const T ta = (T)alpha, tb = (T)beta;
        const bool first = k == 0;
        PG_FOR_OWN_NODES(N, i) {
#pragma unroll
            for (int q = 0; q < 3; q++) {
                const int64_t o = 3 * i + q;
                const T pv = first ? a.u[o] : fma(tb, a.p[o], a.u[o]);
                const T sv = first ? a.w[o] : fma(tb, a.s[o], a.w[o]);
                a.p[o] = pv;
                a.s[o] = sv;
                a.x[o] = fma(ta, pv, a.x[o]);
                a.r[o] = fma(-ta, sv, a.r[o]);
            }
            cg_minv(a, i);
        }
        k += 1;
        if (!pg_barrier(a.bar, phase)) return abort_out();  // u complete before it is gathered
        T g = 0, d = 0, q = 0;
        PG_FOR_OWN_NODES(N, i) cg_row(a, i, g, d, q);
        if (!reduce3(g, d, q)) return abort_out();
        const double gn = s_red[0], res = sqrt(s_red[2]);
        del = s_red[1];
        if (!isfinite(res) || !isfinite(gn) || !isfinite(del)) {
            flags = 1;
            break;
        }
        if (res <= tol) {
            conv = 1;
            break;
        }
        if (k >= a.maxit) break;
        beta = gn / gam;
        const double den = del - beta * gn / alpha;
        if (!(den != 0.0) || !(gn != 0.0)) {
            flags = 2;
            break;
        }
        alpha = gn / den;
        gam = gn;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->its += k;
        st->solves += 1;
        st->total = k;
        st->converged = conv;
        st->flags = flags;
        st->status_any |= flags | ((!conv && !flags) ? 4 : 0);
        st->alg_bytes += (k + 1) * a.it_bytes;
        st->stop = 2;
    }
    return true;
}

template <typename T>
__global__ void __launch_bounds__(kPgThreads, 2) k_cg_a(CgArgs<T> a) {
    unsigned phase = 0u;  // the barrier words are cleared before every launch
    pg_cg_a<T>(a, phase);
}

// The S-solve of Algorithm 1 (step 3) as one cooperative kernel: GMRES on
// S P^-1 with the matrix-free product of Algorithm 2 inside,
//   z = P^-1 v (diag(S^)^-1: applied while gathering; Chebyshev in S^: a few
//   grid phases of its own), xbar = B z,
//   xtil = A^-1 xbar (the A-solve above, or CG on A_sym, on the same grid),
//   barrier, w = D z - C xtil;
// x = P^-1 V y.
template <typename T, bool H16, bool CHEB, bool ICG, bool ACH>
__global__ void __launch_bounds__(kPgThreads, 2) k_gmres_s(SgArgs<T> s, PgArgs<T> a) {
    unsigned phase = 0u;  // the barrier words are cleared before every launch
    const int64_t N = s.g.N;
    auto zval = [&](const T *u, int64_t c) -> T {
        if constexpr (CHEB)
            return s.zc[c];
        else
            return __ldg(s.shat + c) * u[c];
    };
    auto op = [&](const T *u, T sc, T *w, unsigned &ph, int j) {
        if constexpr (CHEB) {
            if (!pg_cheb(s.ch, N, u, (T)1, s.zc, false, s.g.bar, ph)) return false;
            if (s.g.Zb) {
                // Z_j = P^-1 v_j = sc P^-1 u (row-local; x = Z y at the end of a cycle)
                T *Zj = s.g.Zb + (int64_t)j * N;
                PG_FOR_OWN_NODES(N, i) Zj[i] = s.zc[i] * sc;
            }
        }
        PG_FOR_OWN_NODES(N, i) {
            const int t = (int)(i & 31);
            const int64_t b0 = s.slice_ptr[i >> 5];
            const int len = s.row_len[i];
            T a0 = 0, a1 = 0, a2 = 0;
            for (int jb = 0; jb < len; jb++) {
                const int64_t q = (b0 + jb) * 32 + t;
                const int64_t c = __ldg(s.col + q);
                const T zc = zval(u, c);
                const T *Bb = s.B + (q >> 5) * 96 + t;
                a0 = fma(__ldg(Bb), zc, a0);
                a1 = fma(__ldg(Bb + 32), zc, a1);
                a2 = fma(__ldg(Bb + 64), zc, a2);
            }
            s.xbar[3 * i] = a0 * sc;
            s.xbar[3 * i + 1] = a1 * sc;
            s.xbar[3 * i + 2] = a2 * sc;
        }
        if constexpr (ICG) {
            if (!pg_cg_a<T>(s.cg, ph)) return false;
        } else {
            if (!pg_gmres_a<T, H16, ACH>(a, ph)) return false;
        }
        if (!pg_barrier(s.g.bar, ph)) return false;  // xtil complete before it is gathered
        PG_FOR_OWN_NODES(N, i) {
            const int t = (int)(i & 31);
            const int64_t b0 = s.slice_ptr[i >> 5];
            const int len = s.row_len[i];
            T d = 0, m = 0;
            for (int jb = 0; jb < len; jb++) {
                const int64_t q = (b0 + jb) * 32 + t;
                const int64_t c = __ldg(s.col + q);
                d = fma(__ldg(s.D + (q >> 5) * 32 + t), zval(u, c), d);
                const T *Cb = s.C + (q >> 5) * 96 + t;
                m = fma(__ldg(Cb), s.xtil[3 * c], fma(__ldg(Cb + 32), s.xtil[3 * c + 1], fma(__ldg(Cb + 64), s.xtil[3 * c + 2], m)));
            }
            w[i] = d * sc - m;
        }
        return true;
    };
    if constexpr (CHEB) {
        if (s.g.Zb) {
            // flexible form: x += Z y
            auto xupd = [&](int64_t i, const T (&u)[1]) { s.g.x[i] += u[0]; };
            pg_gmres<T, 1>(s.g, phase, op, xupd);
        } else {
            // V y goes to the Chebyshev residual buffer, then x += P^-1 (V y)
            auto xupd = [&](int64_t i, const T (&u)[1]) { s.ch.r[i] = u[0]; };
            auto xend = [&](unsigned &ph) { return pg_cheb(s.ch, N, s.ch.r, (T)1, s.g.x, true, s.g.bar, ph); };
            pg_gmres<T, 1>(s.g, phase, op, xupd, xend);
        }
    } else {
        auto xupd = [&](int64_t i, const T (&u)[1]) { s.g.x[i] += __ldg(s.shat + i) * u[0]; };
        pg_gmres<T, 1>(s.g, phase, op, xupd);
    }
}

// GMRES on the explicit S^ (the S^-solve of the SIMPLE preconditioner) as one
// cooperative launch: operator S^ P^-1 with P^-1 = diag(S^)^-1 (applied while
// gathering) or the Chebyshev polynomial in S^ (grid phases of its own);
// x = P^-1 V y. S^ values of the level's precision.
template <typename T>
struct ShArgs {
    const int32_t *slice_ptr, *row_len, *col;  // S^ pattern (SELL-32)
    const T *val;
    const T *dinv;  // [N] 1 / diag(S^)
    T *zc;          // [N] P^-1 v (Chebyshev only)
    ChebArgs<T> ch;
    GmArgs<T> g;
};

template <typename T, bool CHEB>
__global__ void __launch_bounds__(kPgThreads, 2) k_gmres_shat(ShArgs<T> s) {
    unsigned phase = 0u;  // the barrier words are cleared before every launch
    const int64_t N = s.g.N;
    auto op = [&](const T *u, T sc, T *w, unsigned &ph, int) {
        if constexpr (CHEB) {
            if (!pg_cheb(s.ch, N, u, (T)1, s.zc, false, s.g.bar, ph)) return false;
        }
        PG_FOR_OWN_NODES(N, i) {
            const int t = (int)(i & 31);
            const int64_t b0 = __ldg(s.slice_ptr + (i >> 5));
            const int len = __ldg(s.row_len + i);
            T acc = 0;
            for (int p = 0; p < len; p++) {
                const int64_t q = (b0 + p) * 32 + t;
                const int64_t c = __ldg(s.col + q);
                T zc;
                if constexpr (CHEB)
                    zc = s.zc[c];
                else
                    zc = __ldg(s.dinv + c) * u[c];
                acc = fma(__ldg(s.val + q), zc, acc);
            }
            w[i] = acc * sc;
        }
        return true;
    };
    if constexpr (CHEB) {
        auto xupd = [&](int64_t i, const T (&u)[1]) { s.ch.r[i] = u[0]; };
        auto xend = [&](unsigned &ph) { return pg_cheb(s.ch, N, s.ch.r, (T)1, s.g.x, true, s.g.bar, ph); };
        pg_gmres<T, 1>(s.g, phase, op, xupd, xend);
    } else {
        auto xupd = [&](int64_t i, const T (&u)[1]) { s.g.x[i] += __ldg(s.dinv + i) * u[0]; };
        pg_gmres<T, 1>(s.g, phase, op, xupd);
    }
}

// SIMPLE's last step: x_v = xhat - diag(A)^-1 (B x_p), diag(A) the scalar
// diagonal of the scaled A (Av in the SELL-32 block layout)
template <typename T>
__global__ void k_simple_update(const int32_t *__restrict__ diag_slot, const T *__restrict__ Av,
                                const T *__restrict__ xhat, const T *__restrict__ bx, T *__restrict__ xv, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t dq = diag_slot[i], db = dq >> 5, dt = dq & 31;
#pragma unroll
    for (int r = 0; r < 3; r++) xv[3 * i + r] = xhat[3 * i + r] - bx[3 * i + r] / Av[(db * 9 + 4 * r) * 32 + dt];
}

// Ritz values for the Chebyshev interval: kRitzSteps steps of Arnoldi on
// T = |M|^-1/2 S^ |M|^-1/2 (M = diag(S^); T is similar to M^-1 S^ when
// diag(S^) > 0), in FP32 (an estimate; sums across blocks in FP64), one
// cooperative launch. The start vector comes from
// SplitMix64 (Steele, Lea and Flood 2014): output i of the generator seeded
// with 0 gives x0[i] = 2 u - 1, u its top 53 bits over 2^53. Each new
// direction is orthogonalised twice against the basis (classical
// Gram-Schmidt); block 0 writes the Hessenberg columns H[j * (k + 1) + i].
// The host takes the eigenvalues of the symmetric part of the leading k x k
// block. V: [(k + 1) N]; U: [2N] (the unnormalised new direction, double-
// buffered: a step gathers the previous one while writing the next); Sq: [N].
constexpr int kRitzSteps = 12;
constexpr double kRitzSafety = 1.05, kRitzLow = 2.0;  // lmax = 1.05 theta_max, lmin = theta_min / 2

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long k) {
    unsigned long long z = (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct ArnArgs {
    const int32_t *slice_ptr, *row_len, *col;
    const float *val;
    const double *dinv;
    float *V, *U, *Sq;  // U: [2N]; Sq: [N] |diag(S^)|^-1/2
    double *H, *partial;
    unsigned *bar;
    int64_t N;
};

__global__ void __launch_bounds__(kPgThreads) k_shat_arnoldi(ArnArgs a) {
    __shared__ double red1[kPgThreads / 32];
    __shared__ double s_sum[kRitzSteps + 2], s_h[kRitzSteps + 2];
    __shared__ float hs[kRitzSteps + 2];
    unsigned phase = 0u;
    const int64_t N = a.N;
    const int G = gridDim.x, K1 = kRitzSteps + 1;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    auto pbuf = [&](unsigned ph) { return a.partial + (size_t)(ph & 1u) * G * K1; };
    auto fail_out = [&]() {
        if (lead) a.H[0] = nan("");
    };
    float ss = 0.0f;
    PG_FOR_OWN_NODES(N, i) {
        const float x = (float)(2.0 * ((double)(splitmix64_at((unsigned long long)i) >> 11) * 0x1p-53) - 1.0);
        a.U[i] = x;
        a.Sq[i] = (float)sqrt(fabs(__ldg(a.dinv + i)));
        ss = fmaf(x, x, ss);
    }
    double tb = pg_block_sum<float>(ss, red1);
    if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
    if (!pg_barrier(a.bar, phase)) return fail_out();
    pg_sum(pbuf(phase - 1), 1, s_sum);
    __syncthreads();
    float sc = (float)(1.0 / sqrt(s_sum[0]));
    for (int j = 0; j < kRitzSteps; j++) {
        const float *u = a.U + (size_t)(j & 1) * N;
        float *w = a.U + (size_t)((j + 1) & 1) * N;
        float *Vj = a.V + (size_t)j * N;
        // v_j = sc u; w = T v_j
        PG_FOR_OWN_NODES(N, i) {
            Vj[i] = u[i] * sc;
            const int t = (int)(i & 31);
            const int64_t b0 = __ldg(a.slice_ptr + (i >> 5));
            const int len = __ldg(a.row_len + i);
            float acc = 0.0f;
            for (int p = 0; p < len; p++) {
                const int64_t q = (b0 + p) * 32 + t;
                const int64_t c = __ldg(a.col + q);
                acc = fmaf(__ldg(a.val + q), a.Sq[c] * u[c], acc);
            }
            w[i] = a.Sq[i] * acc * sc;
        }
        // two classical Gram-Schmidt passes, then ||w||
        for (int l = threadIdx.x; l <= j; l += blockDim.x) s_h[l] = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            pg_dots<float, 1>(a.V, w, N, j + 1, false, pbuf(phase));
            if (!pg_barrier(a.bar, phase)) return fail_out();
            pg_sum(pbuf(phase - 1), j + 1, s_sum);
            __syncthreads();
            for (int l = threadIdx.x; l <= j; l += blockDim.x) {
                hs[l] = (float)s_sum[l];
                s_h[l] += s_sum[l];
            }
            __syncthreads();
            const float part = pg_axpy<float, 1>(a.V, w, N, j + 1, hs);
            if (pass == 1) {
                tb = pg_block_sum<float>(part, red1);
                if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
            }
        }
        if (!pg_barrier(a.bar, phase)) return fail_out();
        pg_sum(pbuf(phase - 1), 1, s_sum);
        __syncthreads();
        const double hn = sqrt(s_sum[0]);
        if (lead) {
            for (int l = 0; l <= j; l++) a.H[(size_t)j * K1 + l] = s_h[l];
            a.H[(size_t)j * K1 + j + 1] = hn;
        }
        if (!(hn > 0.0)) return;  // invariant subspace (or NaN): the host reads the leading block
        sc = (float)(1.0 / hn);
    }
}

// Ritz values for the A-Chebyshev interval: kRitzSteps steps of Arnoldi on
// M^-1 A in the M-inner product <x, y> = x^T M y (M the 3x3 block diagonal of
// A; M^-1 A is self-adjoint there when A is symmetric, so H is then
// symmetric), in FP32 with the FP32 copy of A (sums across blocks in FP64),
// one cooperative launch. Start vector: x0[k] = 2 u_k - 1 from output k of
// SplitMix64 (k = 3 i + component). Each new direction is orthogonalised
// twice (classical Gram-Schmidt); block 0 writes H[j * (k + 1) + i].
struct AArnArgs {
    const int32_t *slice_ptr, *row_len, *col, *diag_slot;
    const float *Af, *jac;  // FP32 scaled A and M^-1 [9][N]
    float *V, *U;           // V: [(k + 1) 3N]; U: [3 x 3N] two directions and M w
    double *H, *partial;
    unsigned *bar;
    int64_t N;
};

// y = M_i x_i with M_i the diagonal block of row i
__device__ __forceinline__ void diag_block_apply(const AArnArgs &a, int64_t i, const float *x, float *y) {
    const int64_t q = __ldg(a.diag_slot + i), b = q >> 5, t = q & 31;
    const float x0 = x[3 * i], x1 = x[3 * i + 1], x2 = x[3 * i + 2];
#pragma unroll
    for (int r = 0; r < 3; r++)
        y[3 * i + r] = __ldg(a.Af + (b * 9 + 3 * r) * 32 + t) * x0 + __ldg(a.Af + (b * 9 + 3 * r + 1) * 32 + t) * x1 +
                       __ldg(a.Af + (b * 9 + 3 * r + 2) * 32 + t) * x2;
}

__global__ void __launch_bounds__(kPgThreads) k_a_arnoldi(AArnArgs a) {
    __shared__ double red1[kPgThreads / 32];
    __shared__ double s_sum[kRitzSteps + 2], s_h[kRitzSteps + 2];
    __shared__ float hs[kRitzSteps + 2];
    unsigned phase = 0u;
    const int64_t N = a.N, n = 3 * N;
    const int G = gridDim.x, K1 = kRitzSteps + 1;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    float *Mw = a.U + 2 * n;
    auto pbuf = [&](unsigned ph) { return a.partial + (size_t)(ph & 1u) * G * K1; };
    auto fail_out = [&]() {
        if (lead) a.H[0] = nan("");
    };
    float ss = 0.0f;
    PG_FOR_OWN_NODES(N, i) {
#pragma unroll
        for (int k = 0; k < 3; k++)
            a.U[3 * i + k] =
                (float)(2.0 * ((double)(splitmix64_at((unsigned long long)(3 * i + k)) >> 11) * 0x1p-53) - 1.0);
        diag_block_apply(a, i, a.U, Mw);
#pragma unroll
        for (int k = 0; k < 3; k++) ss = fmaf(a.U[3 * i + k], Mw[3 * i + k], ss);
    }
    double tb = pg_block_sum<float>(ss, red1);
    if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
    if (!pg_barrier(a.bar, phase)) return fail_out();
    pg_sum(pbuf(phase - 1), 1, s_sum);
    __syncthreads();
    float sc = (float)(1.0 / sqrt(s_sum[0]));
    for (int j = 0; j < kRitzSteps; j++) {
        const float *u = a.U + (size_t)(j & 1) * n;
        float *w = a.U + (size_t)((j + 1) & 1) * n;
        float *Vj = a.V + (size_t)j * n;
        // v_j = sc u; w = M^-1 A v_j
        PG_FOR_OWN_NODES(N, i) {
            float y0, y1, y2;
            block_row<float, float, float>(a.slice_ptr, a.row_len, a.col, a.Af, i, u, y0, y1, y2);
#pragma unroll
            for (int k = 0; k < 3; k++) Vj[3 * i + k] = u[3 * i + k] * sc;
#pragma unroll
            for (int k = 0; k < 3; k++)
                w[3 * i + k] = (__ldg(a.jac + (3 * k) * N + i) * y0 + __ldg(a.jac + (3 * k + 1) * N + i) * y1 +
                                __ldg(a.jac + (3 * k + 2) * N + i) * y2) * sc;
        }
        for (int l = threadIdx.x; l <= j; l += blockDim.x) s_h[l] = 0.0;
        for (int pass = 0; pass < 2; pass++) {
            // h = V^T (M w), then w -= V h
            PG_FOR_OWN_NODES(N, i) diag_block_apply(a, i, w, Mw);
            pg_dots<float, 3>(a.V, Mw, N, j + 1, false, pbuf(phase));
            if (!pg_barrier(a.bar, phase)) return fail_out();
            pg_sum(pbuf(phase - 1), j + 1, s_sum);
            __syncthreads();
            for (int l = threadIdx.x; l <= j; l += blockDim.x) {
                hs[l] = (float)s_sum[l];
                s_h[l] += s_sum[l];
            }
            __syncthreads();
            pg_axpy<float, 3>(a.V, w, N, j + 1, hs);
        }
        // ||w||_M^2 = w . M w
        ss = 0.0f;
        PG_FOR_OWN_NODES(N, i) {
            diag_block_apply(a, i, w, Mw);
#pragma unroll
            for (int k = 0; k < 3; k++) ss = fmaf(w[3 * i + k], Mw[3 * i + k], ss);
        }
        tb = pg_block_sum<float>(ss, red1);
        if (threadIdx.x == 0) pbuf(phase)[blockIdx.x] = tb;
        if (!pg_barrier(a.bar, phase)) return fail_out();
        pg_sum(pbuf(phase - 1), 1, s_sum);
        __syncthreads();
        const double hn = sqrt(fmax(s_sum[0], 0.0));
        if (lead) {
            for (int l = 0; l <= j; l++) a.H[(size_t)j * K1 + l] = s_h[l];
            a.H[(size_t)j * K1 + j + 1] = hn;
        }
        if (!(hn > 0.0)) return;
        sc = (float)(1.0 / hn);
    }
}

// y = p(M^-1 A) M^-1 x (FP64 vectors, FP32 A and directions), one cooperative launch
__global__ void __launch_bounds__(kPgThreads) k_acheb_apply(PgArgs<double> a, const double *x, double *y,
                                                            unsigned *status) {
    unsigned phase = 0u;
    if (!pg_cheb3<double>(a, x, y, false, phase) && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, 8u);
}

// y = p(M^-1 S^) M^-1 x (FP64, one cooperative launch); status 8 on a barrier timeout
template <typename V>
__global__ void __launch_bounds__(kPgThreads) k_cheb_apply(ChebArgs<double, V> ch, const double *x, double *y,
                                                           int64_t N, unsigned *bar, unsigned *status) {
    unsigned phase = 0u;
    if (!pg_cheb(ch, N, x, 1.0, y, false, bar, phase) && blockIdx.x == 0 && threadIdx.x == 0)
        atomicOr(status, 8u);
}

// ------------------------------------------------------------ recording

// Records kernel sequences either as direct launches driven by a host loop or
// into a CUDA graph with while-conditional nodes.
struct Rec {
    Ctx *c = nullptr;
    bool graph = false;
    int check_every = 1;
    std::vector<cudaStream_t> *streams = nullptr;  // capture streams by depth
    int depth = 0;
    // kernel-node bookkeeping for launch counting: per level state, kernels
    // per iteration and per solve
    struct Site {
        LevelState *st;
        int body_nodes;
        int init_nodes;
    };
    std::vector<Site> *sites = nullptr;
    int *capture_count = nullptr;

    // run body() while the level is not stopped; init(h) starts the solve
    void loop(LevelState *st, int every, const std::function<void(cudaGraphConditionalHandle)> &init,
              const std::function<void(cudaGraphConditionalHandle)> &body) {
        if (!graph) {
            LevelState hs;
            init(0);
            for (;;) {
                HYEL_CK(cudaMemcpyAsync(&hs, st, sizeof(LevelState), cudaMemcpyDeviceToHost, c->stream));
                HYEL_CK(cudaStreamSynchronize(c->stream));
                if (hs.stop) break;
                for (int r = 0; r < every; r++) body(0);
            }
            return;
        }
        cudaStream_t s = c->stream;
        cudaStreamCaptureStatus cst;
        cudaGraph_t g;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        HYEL_CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd));
        cudaGraphConditionalHandle h;
        HYEL_CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        const int before_init = *capture_count;
        init(h);
        const int init_nodes = *capture_count - before_init;
        HYEL_CK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd));
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        HYEL_CK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
        HYEL_CK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        cudaGraph_t bodyg = p.conditional.phGraph_out[0];
        if ((int)streams->size() <= depth + 1) {
            cudaStream_t ns;
            HYEL_CK(cudaStreamCreateWithFlags(&ns, cudaStreamNonBlocking));
            streams->push_back(ns);
        }
        cudaStream_t bs = (*streams)[depth + 1];
        HYEL_CK(cudaStreamBeginCaptureToGraph(bs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        c->stream = bs;
        depth++;
        const int before_body = *capture_count;
        const size_t nsites = sites->size();
        body(h);
        // nodes of nested loops are accounted to their own sites
        int nested = 0;
        for (size_t q = nsites; q < sites->size(); q++) nested += (*sites)[q].body_nodes + (*sites)[q].init_nodes;
        const int body_nodes = *capture_count - before_body - nested;
        depth--;
        c->stream = s;
        cudaGraph_t outg;
        HYEL_CK(cudaStreamEndCapture(bs, &outg));
        sites->push_back({st, body_nodes, init_nodes});
    }
};

}  // namespace

// ------------------------------------------------------------ workspace

namespace {

template <typename T>
struct Level {
    int64_t n = 0;
    int m = 0;
    int kind = 0;
    T *V = nullptr, *Z = nullptr, *z = nullptr;
    double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr, *h2 = nullptr;
    double *partial = nullptr;
    unsigned *counter = nullptr;
    int grid = 0;
    // persistent A-solve (kind 0): second work vector, per-block partials,
    // barrier words, cooperative grid sizes
    T *z2 = nullptr;
    double *pg_partial = nullptr;
    unsigned *bar = nullptr;
    int pg_grid = 0, pg_grid16 = 0;
    int pg_gridc = 0, pg_grid16c = 0;  // S-level with the Chebyshev preconditioner
    int pg_grid_sh = 0, pg_grid_shc = 0;  // GMRES on the explicit S^ (SIMPLE), diag / Chebyshev
    // A-level (kind 0): the A-Chebyshev polynomial's buffers, zc and r [3N] of
    // T, then d0 and d1 [3N] of float
    unsigned char *ach = nullptr;
};

}  // namespace

struct Workspace {
    int m_outer = 0, m_a = 0, m_s = 0, prec = -1, a_amg = 0;
    int a_cheb = 0;  // degree of the A-Chebyshev polynomial of the current solve (0: block-Jacobi)
    Level<double> outer;
    Level<double> a64, s64;
    Level<float> a32, s32;
    Level<double> am64;  // FGMRES A-level with the multigrid preconditioner
    Level<float> am32;
    LevelState *states = nullptr;  // [5]: outer, a1, a2, s, inner
    LevelState *h_states = nullptr;
    double *d = nullptr;  // 12 x 4N doubles
    float *f = nullptr;   // 12 x 4N floats
    std::vector<void *> mem;
    // cached graph
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    hyel_solver_params key;
    bool have_key = false;
    std::vector<cudaStream_t> streams;
    std::vector<Rec::Site> sites;
    int top_nodes = 0;

    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
        for (cudaStream_t s : streams) cudaStreamDestroy(s);
        streams.clear();
        for (void *p : mem) cudaFree(p);
        mem.clear();
        if (h_states) cudaFreeHost(h_states);
        h_states = nullptr;
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

void *walloc(Ctx &c, Workspace &w, size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        fail(HYEL_ENOMEM, "solver workspace: cudaMalloc failed");
    }
    w.mem.push_back(p);
    c.bytes_held += bytes;
    return p;
}

template <typename T>
void level_init(Ctx &c, Workspace &w, Level<T> &L, int64_t n, int m, int kind) {
    L.n = n;
    L.m = m;
    L.kind = kind;
    L.grid = (int)std::max<int64_t>(1, std::min<int64_t>(2 * c.num_sms, (n + 4 * kThreads - 1) / (4 * kThreads)));
    L.V = (T *)walloc(c, w, sizeof(T) * (size_t)(m + 1) * n);
    if (kind == 2 || kind == 1) L.Z = (T *)walloc(c, w, sizeof(T) * (size_t)m * n);  // kind 1: the flexible S-level
    L.z = (T *)walloc(c, w, sizeof(T) * (size_t)n);
    L.H = (double *)walloc(c, w, sizeof(double) * (size_t)(m + 1) * m);
    L.cs = (double *)walloc(c, w, sizeof(double) * m);
    L.sn = (double *)walloc(c, w, sizeof(double) * m);
    L.g = (double *)walloc(c, w, sizeof(double) * (m + 1));
    L.y = (double *)walloc(c, w, sizeof(double) * m);
    L.h2 = (double *)walloc(c, w, sizeof(double) * (m + 1));
    L.partial = (double *)walloc(c, w, sizeof(double) * (size_t)L.grid * (m + 1));
    L.counter = (unsigned *)walloc(c, w, sizeof(unsigned) * 4);
    HYEL_CK(cudaMemsetAsync(L.counter, 0, sizeof(unsigned) * 4, c.stream));
    if (kind == 0 || kind == 1) {
        // the persistent A- and S-solves: cooperative grids of co-resident
        // blocks (at most one thread per node); an A-level's partials serve
        // every grid that can run it (its own and the S-solve's)
        const int64_t nodes = kind == 0 ? n / 3 : n;
        L.z2 = (T *)walloc(c, w, sizeof(T) * (size_t)n);
        if (kind == 0) L.ach = (unsigned char *)walloc(c, w, (size_t)n * (2 * sizeof(T) + 2 * sizeof(float)));
        L.bar = (unsigned *)walloc(c, w, sizeof(unsigned) * kBarAlloc);
        const int64_t need = std::max<int64_t>(1, (nodes + 31) / 32);  // no block without a slice
        int occ = 0, occ16 = 0;
        if (kind == 0)
            HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gmres_a<T, false, false>, kPgThreads, 0));
        else
            HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_gmres_s<T, false, false, false, false>, kPgThreads, 0));
        occ16 = occ;
        if constexpr (std::is_same<T, float>::value) {
            if (kind == 0)
                HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ16, k_gmres_a<float, true, false>, kPgThreads, 0));
            else
                HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ16, k_gmres_s<float, true, false, false, false>, kPgThreads, 0));
        }
        int occc = occ, occ16c = occ16;
        if (kind == 1) {
            HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occc, k_gmres_s<T, false, true, false, false>, kPgThreads, 0));
            occ16c = occc;
            if constexpr (std::is_same<T, float>::value)
                HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ16c, k_gmres_s<float, true, true, false, false>, kPgThreads, 0));
        }
        if (occ < 1 || occ16 < 1 || occc < 1 || occ16c < 1) fail(HYEL_ECUDA, "persistent solve kernel does not fit on an SM");
        L.pg_grid = (int)std::min<int64_t>((int64_t)occ * c.num_sms, need);
        L.pg_grid16 = (int)std::min<int64_t>((int64_t)occ16 * c.num_sms, need);
        L.pg_gridc = (int)std::min<int64_t>((int64_t)occc * c.num_sms, need);
        L.pg_grid16c = (int)std::min<int64_t>((int64_t)occ16c * c.num_sms, need);
        if (kind == 1) {
            int o1 = 0, o2 = 0;
            HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_gmres_shat<T, false>, kPgThreads, 0));
            HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_gmres_shat<T, true>, kPgThreads, 0));
            if (o1 < 1 || o2 < 1) fail(HYEL_ECUDA, "persistent S^ solve kernel does not fit on an SM");
            L.pg_grid_sh = (int)std::min<int64_t>((int64_t)o1 * c.num_sms, need);
            L.pg_grid_shc = (int)std::min<int64_t>((int64_t)o2 * c.num_sms, need);
        }
        const int64_t gmax = (int64_t)(2048 / kPgThreads) * c.num_sms;  // any co-resident grid
        L.pg_partial = (double *)walloc(c, w, sizeof(double) * 2 * (size_t)gmax * (m + 1));
    }
}

Workspace &workspace(Ctx &c, const hyel_solver_params &p) {
    const int mo = p.outer.restart, ma = std::max(p.a.restart, p.inner.restart), ms = p.s.restart;
    Workspace *w = c.ws;
    if (w && w->m_outer >= mo && w->m_a >= ma && w->m_s >= ms && w->prec == p.precision &&
        w->a_amg == (p.a_precond == HYEL_APREC_AMG))
        return *w;
    free_workspace(c);
    w = new Workspace();
    c.ws = w;
    const int64_t N = c.mesh.N;
    w->m_outer = mo;
    w->m_a = ma;
    w->m_s = ms;
    w->prec = p.precision;
    w->a_amg = p.a_precond == HYEL_APREC_AMG;
    level_init(c, *w, w->outer, 4 * N, mo, 2);
    if (p.precision == HYEL_PREC_FP64) {
        if (w->a_amg)
            level_init(c, *w, w->am64, 3 * N, ma, 2);
        else
            level_init(c, *w, w->a64, 3 * N, ma, 0);
        level_init(c, *w, w->s64, N, ms, 1);
    } else {
        if (w->a_amg)
            level_init(c, *w, w->am32, 3 * N, ma, 2);
        else
            level_init(c, *w, w->a32, 3 * N, ma, 0);
        level_init(c, *w, w->s32, N, ms, 1);
    }
    w->states = (LevelState *)walloc(c, *w, sizeof(LevelState) * 5);
    HYEL_CK(cudaMemsetAsync(w->states, 0, sizeof(LevelState) * 5, c.stream));
    HYEL_CK(cudaMallocHost(&w->h_states, sizeof(LevelState) * 5));
    w->d = (double *)walloc(c, *w, sizeof(double) * 12 * 4 * (size_t)N);
    w->f = (float *)walloc(c, *w, sizeof(float) * 12 * 4 * (size_t)N);
    return *w;
}

void check_cheb(int degree, double ratio) {
    if (degree < 1 || degree > kChebMaxDegree) fail(HYEL_EINVAL, "solver params: s_cheb_degree must be in [1, 16]");
    if (!(ratio == 0.0 || ratio > 1.0) || !std::isfinite(ratio))
        fail(HYEL_EINVAL, "solver params: s_cheb_ratio must be 0 (estimated) or finite and > 1");
}

void check_params(const hyel_solver_params &p) {
    const hyel_krylov_level *lv[4] = {&p.outer, &p.a, &p.s, &p.inner};
    for (auto *l : lv) {
        if (l->restart < 1 || l->restart > kMaxK) fail(HYEL_EINVAL, "solver params: restart must be in [1, 512]");
        if (l->maxit < 1) fail(HYEL_EINVAL, "solver params: maxit must be >= 1");
        if (!(l->rtol >= 0) || !(l->atol >= 0)) fail(HYEL_EINVAL, "solver params: tolerances must be >= 0");
    }
    if (p.precision != HYEL_PREC_FP64 && p.precision != HYEL_PREC_FP32 && p.precision != HYEL_PREC_BF16S)
        fail(HYEL_EINVAL, "solver params: bad precision");
    if (p.check_every < 1) fail(HYEL_EINVAL, "solver params: check_every must be >= 1");
    if (p.a_precond != HYEL_APREC_BJACOBI && p.a_precond != HYEL_APREC_AMG && p.a_precond != HYEL_APREC_CHEB)
        fail(HYEL_EINVAL, "solver params: bad a_precond");
    if (p.a_precond == HYEL_APREC_CHEB && (p.a_cheb_degree < 1 || p.a_cheb_degree > kChebMaxDegree))
        fail(HYEL_EINVAL, "solver params: a_cheb_degree must be in [1, 16]");
    if (p.s_precond != HYEL_SPREC_JACOBI && p.s_precond != HYEL_SPREC_CHEB)
        fail(HYEL_EINVAL, "solver params: bad s_precond");
    if (p.block_precond < HYEL_BLOCK_LDU || p.block_precond > HYEL_BLOCK_SIMPLE)
        fail(HYEL_EINVAL, "solver params: bad block_precond");
    if (p.inner_solver != HYEL_INNER_GMRES && p.inner_solver != HYEL_INNER_CG_SYM)
        fail(HYEL_EINVAL, "solver params: bad inner_solver");
    if (p.inner_solver == HYEL_INNER_CG_SYM) {
        if (p.a_precond != HYEL_APREC_BJACOBI)
            fail(HYEL_EINVAL, "solver params: the CG inner solve needs block-Jacobi A-solves");
        if (std::max(p.a.restart, p.inner.restart) < 2)
            fail(HYEL_EINVAL, "solver params: the CG inner solve needs an A-level restart of at least 2");
    }
    if (p.s_precond == HYEL_SPREC_CHEB) {
        if (p.a_precond == HYEL_APREC_AMG)
            fail(HYEL_EINVAL, "solver params: the Chebyshev S-preconditioner needs persistent A-solves (not multigrid)");
        check_cheb(p.s_cheb_degree, p.s_cheb_ratio);
    }
}

bool same_params(const hyel_solver_params &a, const hyel_solver_params &b) {
    return std::memcmp(&a, &b, sizeof a) == 0;
}

// Typed view of the scaled matrix and the levels for precision T.
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
    static Level<double> &la(Workspace &w) { return w.a64; }
    static Level<double> &lam(Workspace &w) { return w.am64; }
    static Level<double> &ls(Workspace &w) { return w.s64; }
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
    static Level<float> &la(Workspace &w) { return w.a32; }
    static Level<float> &lam(Workspace &w) { return w.am32; }
    static Level<float> &ls(Workspace &w) { return w.s32; }
    static float *vec(Workspace &w, int k, int64_t N) { return w.f + (size_t)k * 4 * N; }
};

enum { ST_OUTER = 0, ST_A1 = 1, ST_A2 = 2, ST_S = 3, ST_INNER = 4 };

#define LAUNCH(...) ((__VA_ARGS__), ::hyel::count_launch())

// One GMRES/FGMRES solve of level L: the init kernel, then the iteration
// loop. prec_flex (KIND 2) maps V_k to Z_k; op maps the preconditioned vector
// (z, or Z_k for KIND 2) to V_{k+1}.
template <typename T, int KIND>
void gm_solve(Rec &R, Level<T> &L, LevelState *st, const hyel_krylov_level &P, const T *b, T *x, const T *prec,
              const std::function<void()> &prec_flex, const std::function<void()> &op, bool loose_single) {
    Ctx &c = *R.c;
    const int m = std::min(P.restart, L.m);
    // S-level and multigrid A-level solves as loose as the paper's (rtol >=
    // kPgLoose) keep one classical Gram-Schmidt pass, as PETSc's default GMRES
    // does; the outer FGMRES and tighter solves run CGS2
    const int single = (loose_single && P.rtol >= kPgLoose<T>) ? 1 : 0;
    // the operator of both looped levels is itself a solve: the host-driven
    // mode checks them every iteration
    R.loop(
        st, 1,
        [&](cudaGraphConditionalHandle h) {
            LAUNCH(k_init<T><<<L.grid, kThreads, 0, c.stream>>>(b, L.V, x, L.n, L.partial, L.counter, st, L.g, m,
                                                               P.rtol, P.atol, P.maxit, h));
        },
        [&](cudaGraphConditionalHandle h) {
            if (KIND == 1)
                LAUNCH(k_scale_diag<T><<<blocks_for(L.n, 256), 256, 0, c.stream>>>(L.V, L.z, prec, L.n, st));
            else {
                LAUNCH(k_scale_diag<T><<<blocks_for(L.n, 256), 256, 0, c.stream>>>(L.V, (T *)nullptr, (const T *)nullptr,
                                                                                  L.n, st));
                prec_flex();
            }
            op();
            if (single) {
                LAUNCH(k_multidot<T><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.n, L.partial, L.counter, L.H, L.h2, st,
                                                                         2));
            } else {
                LAUNCH(k_multidot<T><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.n, L.partial, L.counter, L.H, L.h2, st,
                                                                         1));
                LAUNCH(k_multiaxpy<T><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.n, L.H, st));
                LAUNCH(k_multidot<T><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.n, L.partial, L.counter, L.H, L.h2, st,
                                                                         2));
            }
            LAUNCH(k_axpy_norm_givens<T><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.n, L.h2, L.partial, L.counter, L.H,
                                                                            L.cs, L.sn, L.g, L.y, st, single));
            LAUNCH(k_cycle_end<T, KIND><<<L.grid, kThreads, 0, c.stream>>>(L.V, L.Z, x, prec, L.n, L.y, L.cs, L.sn, L.g,
                                                                          L.counter, st, h));
        });
}

// Arguments of the persistent A-solve for precision T (h16: the BF16 operator)
template <typename T>
PgArgs<T> pg_args(Ctx &c, Workspace &w, LevelState *st, const hyel_krylov_level &P, const T *b, T *x, bool &h16) {
    Level<T> &L = Sys<T>::la(w);
    const DeviceMesh &msh = c.mesh;
    const DeviceMatrix &M = c.mat;
    PgArgs<T> a;
    a.slice_ptr = msh.slice_ptr;
    a.row_len = msh.row_len;
    a.col = msh.col;
    a.Am = nullptr;
    a.Am8 = M.Amh8;
    a.Am1 = M.Amh1;
    a.Ams = M.Amhs;
    a.jac = Sys<T>::jac(c);
    GmArgs<T> &g = a.g;
    g.N = msh.N;
    g.b = b;
    g.x = x;
    g.V = L.V;
    g.U0 = L.z;
    g.U1 = L.z2;
    g.H = L.H;
    g.partial = L.pg_partial;
    g.bar = L.bar;
    g.st = st;
    g.m = std::min(P.restart, L.m);
    g.maxit = P.maxit;
    g.rtol = P.rtol;
    g.atol = P.atol;
    g.eta2 = P.rtol >= kPgLoose<T> ? kPgEta2<T> : 0.5;
    h16 = false;
    if constexpr (std::is_same<T, float>::value) {
        h16 = w.prec == HYEL_PREC_BF16S && w.a_cheb == 0;
        a.Am = h16 ? nullptr : M.Amf;
    } else {
        a.Am = M.Ams;
    }
    // algorithmic bytes of one iteration (matrix once, each vector pass once):
    // A~ values + column indices + row metadata, and the passes over 3N-vectors
    g.it_fixed = (double)msh.nnzb * ((h16 ? 22.0 : 9.0 * sizeof(T)) + 4.0) + 4.0 * (msh.N + 1);
    g.it_unit = 3.0 * msh.N * sizeof(T);
    a.ac = AChArgs<T>{};
    if (w.a_cheb > 0) {
        const int64_t n = 3 * msh.N;
        a.ac.Af = M.Af;
        if constexpr (std::is_same<T, double>::value)
            a.ac.A = M.As;
        else
            a.ac.A = M.Af;
        a.ac.bounds = c.ach->bounds;
        a.ac.degree = w.a_cheb;
        a.ac.zc = reinterpret_cast<T *>(L.ach);
        a.ac.r = a.ac.zc + n;
        a.ac.d0 = reinterpret_cast<float *>(L.ach + 2 * n * sizeof(T));
        a.ac.d1 = a.ac.d0 + n;
        // per application: degree - 1 FP32 A products, M^-1 and the passes
        const int d = w.a_cheb;
        g.it_fixed += (d - 1) * ((double)msh.nnzb * 40.0 + 4.0 * (msh.N + 1) + 9.0 * msh.N * sizeof(T)) +
                      (3.0 + 7.0 * (d - 1)) * n * sizeof(T);
    }
    return a;
}

// Co-resident grid of a persistent kernel (512-thread blocks), at most one
// block per 32-row slice
int resident_grid(Ctx &c, const void *kernel) {
    int occ = 0;
    HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kPgThreads, 0));
    if (occ < 1) fail(HYEL_ECUDA, "persistent solve kernel does not fit on an SM");
    const int64_t need = std::max<int64_t>(1, (c.mesh.N + 31) / 32);
    return (int)std::min<int64_t>((int64_t)occ * c.num_sms, need);
}

cudaLaunchConfig_t coop_config(Ctx &c, int grid) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kPgThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c.stream;
    return cfg;
}

// A-solve x = A^-1 b: one cooperative launch of the persistent GMRES kernel
// (its barrier words cleared just before), in host-driven mode and in the graph
template <typename T>
void a_solve(Rec &R, Workspace &w, LevelState *st, const hyel_krylov_level &P, const T *b, T *x) {
    Ctx &c = *R.c;
    if (w.a_amg) {
        // FGMRES on A with one multigrid V-cycle as the right preconditioner:
        // V_k -> (V-cycle) -> Z_k, A Z_k -> V_{k+1}, x = Z y
        Level<T> &L = Sys<T>::lam(w);
        const int64_t N = c.mesh.N, n = 3 * N;
        T *vin = Sys<T>::vec(w, 3, N), *zout = Sys<T>::vec(w, 11, N);
        gm_solve<T, 2>(
            R, L, st, P, b, x, nullptr,
            [&]() {
                LAUNCH(k_copy_ind<T, T><<<blocks_for(n, 256), 256, 0, c.stream>>>(L.V, vin, n, st, n, 0));
                amg_apply<T>(c, vin, zout);
                LAUNCH(k_copy_ind<T, T><<<blocks_for(n, 256), 256, 0, c.stream>>>(zout, L.Z, n, st, 0, n));
            },
            [&]() { spmv_A_ind<T>(c, Sys<T>::A(c), zout, L.V, L.n, &st->k); }, true);
        return;
    }
    bool h16 = false;
    Level<T> &L = Sys<T>::la(w);
    PgArgs<T> a = pg_args<T>(c, w, st, P, b, x, h16);
    bar_reset(c, L.bar);
    cudaLaunchConfig_t cfg = coop_config(c, h16 ? L.pg_grid16 : L.pg_grid);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_GMRES_A, &ev);
    bool launched = false;
    if (w.a_cheb > 0) {
        cfg.gridDim = dim3((unsigned)resident_grid(c, (const void *)k_gmres_a<T, false, true>));
        HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_a<T, false, true>, a));
        launched = true;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (h16 && !launched) {
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_a<float, true, false>, a));
            launched = true;
        }
    }
    if (!launched) HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_a<T, false, false>, a));
    count_launch();
    prof_end(c, HYEL_K_GMRES_A, ev, 0.0);  // bytes are added from the level states after the solve
}

// CG arguments of the inner A-solve on A_sym (built by asym_setup), on the
// A-level buffers: r, p, s in the first three basis columns, u and w in the
// two direction buffers
template <typename T>
CgArgs<T> cg_args(Ctx &c, Workspace &w, const hyel_solver_params &p, const T *b, T *x) {
    Level<T> &L = Sys<T>::la(w);
    const DeviceMesh &msh = c.mesh;
    const int64_t n = 3 * msh.N;
    CgArgs<T> a;
    a.slice_ptr = msh.slice_ptr;
    a.row_len = msh.row_len;
    a.col = msh.col;
    if constexpr (std::is_same<T, double>::value) {
        a.Av = c.mat.Asym64;
        a.jac = c.mat.jsym64;
    } else {
        a.Av = c.mat.Asym32;
        a.jac = c.mat.jsym32;
    }
    a.b = b;
    a.x = x;
    a.r = L.V;
    a.p = L.V + n;
    a.s = L.V + 2 * n;
    a.u = L.z;
    a.w = L.z2;
    a.partial = L.pg_partial;
    a.bar = L.bar;
    a.st = w.states + ST_INNER;
    a.N = msh.N;
    a.maxit = p.inner.maxit;
    a.rtol = p.inner.rtol;
    a.atol = p.inner.atol;
    // A_sym values + column indices + row data, M^-1, and the [3N] passes
    // (u, w written; r, u read twice; p, s, x, r updated)
    a.it_bytes = (double)msh.nnzb * (9.0 * sizeof(T) + 4.0) + 4.0 * (msh.N + 1) + 9.0 * msh.N * sizeof(T) +
                 16.0 * n * sizeof(T);
    return a;
}

// Chebyshev arguments on the explicit S^ (built by shat_setup): vectors of
// precision T, values V (FP32 in the solver, either in the stand-alone apply)
template <typename T, typename V = float>
ChebArgs<T, V> cheb_args(Ctx &c, int degree, double ratio, T *r, V *d0, V *d1) {
    const SchurHat &h = *c.sh;
    ChebArgs<T, V> ch;
    ch.slice_ptr = h.slice_ptr;
    ch.row_len = h.row_len;
    ch.col = h.col;
    if constexpr (std::is_same<V, double>::value)
        ch.val = h.v64;
    else
        ch.val = h.v32;
    ch.dinv = Sys<T>::shat(c);
    ch.bounds = h.bounds;
    ch.ratio = ratio;
    ch.degree = degree;
    ch.r = r;
    ch.d0 = d0;
    ch.d1 = d1;
    return ch;
}

// The S-solve of Algorithm 1 step 3 as one cooperative launch of k_gmres_s
// (the inner A-solves of Algorithm 2 run inside it on the A-level buffers)
template <typename T>
void s_solve(Rec &R, Workspace &w, const hyel_solver_params &p, const T *b, T *x) {
    Ctx &c = *R.c;
    const DeviceMesh &msh = c.mesh;
    const int64_t N = msh.N;
    Level<T> &La = Sys<T>::la(w);
    Level<T> &Ls = Sys<T>::ls(w);
    T *xbar = Sys<T>::vec(w, 4, N), *xtil = Sys<T>::vec(w, 5, N);
    bool h16 = false;
    PgArgs<T> a = pg_args<T>(c, w, w.states + ST_INNER, p.inner, xbar, xtil, h16);
    SgArgs<T> sg;
    sg.slice_ptr = msh.slice_ptr;
    sg.row_len = msh.row_len;
    sg.col = msh.col;
    sg.B = Sys<T>::B(c);
    sg.C = Sys<T>::C(c);
    sg.D = Sys<T>::D(c);
    sg.shat = Sys<T>::shat(c);
    sg.xbar = xbar;
    sg.xtil = xtil;
    const bool cheb = p.s_precond == HYEL_SPREC_CHEB;
    const bool icg = p.inner_solver == HYEL_INNER_CG_SYM;
    sg.cg = CgArgs<T>{};
    if (icg) sg.cg = cg_args<T>(c, w, p, xbar, xtil);
    sg.zc = nullptr;
    sg.ch = ChebArgs<T>{};
    if (cheb) {
        // [N] buffers from workspace vector 11 (used otherwise only by multigrid A-solves)
        T *cb = Sys<T>::vec(w, 11, N);
        float *db = reinterpret_cast<float *>(cb + 2 * N);  // 2N floats fit in 2N T
        sg.zc = cb;
        sg.ch = cheb_args<T>(c, p.s_cheb_degree, p.s_cheb_ratio, cb + N, db, db + N);
    }
    GmArgs<T> &g = sg.g;
    g.N = N;
    g.b = b;
    g.x = x;
    g.V = Ls.V;
    g.U0 = Ls.z;
    g.U1 = Ls.z2;
    g.H = Ls.H;
    g.partial = Ls.pg_partial;
    g.bar = La.bar;
    g.st = w.states + ST_S;
    g.m = std::min(p.s.restart, Ls.m);
    g.maxit = p.s.maxit;
    g.rtol = p.s.rtol;
    g.atol = p.s.atol;
    g.eta2 = p.s.rtol >= kPgLoose<T> ? kPgEta2<T> : 0.5;
    g.Zb = cheb ? Ls.Z : nullptr;  // Chebyshev: flexible form, no polynomial at the end of a cycle
    // one S-iteration outside its inner A-solve: B, C, D values and column
    // indices (twice), and the vector passes over [N]-vectors
    g.it_fixed = (double)msh.nnzb * (7.0 * sizeof(T) + 8.0) + 4.0 * (N + 1);
    g.it_unit = (double)N * sizeof(T);
    if (cheb) {
        // per application: degree - 1 S^ products (FP32 values and columns, x
        // gathered) and the row-local passes (3 + 6 (degree - 1) vectors of [N])
        const SchurHat &h = *c.sh;
        const int d = p.s_cheb_degree;
        g.it_fixed += (d - 1) * ((double)h.nnz * 8.0 + (double)N * (sizeof(T) + 8.0)) +
                      (3.0 + 6.0 * (d - 1)) * (double)N * sizeof(T);
    }
    bar_reset(c, La.bar);
    const bool ach = w.a_cheb > 0;
    const void *kicg = cheb ? (const void *)k_gmres_s<T, false, true, true, false>
                            : (const void *)k_gmres_s<T, false, false, true, false>;
    const void *kach = cheb ? (const void *)k_gmres_s<T, false, true, false, true>
                            : (const void *)k_gmres_s<T, false, false, false, true>;
    cudaLaunchConfig_t cfg = coop_config(c, icg   ? resident_grid(c, kicg)
                                         : ach  ? resident_grid(c, kach)
                                         : cheb ? (h16 ? Ls.pg_grid16c : Ls.pg_gridc)
                                                : (h16 ? Ls.pg_grid16 : Ls.pg_grid));
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_GMRES_S, &ev);
    bool launched = false;
    if (icg) {
        // the inner solve reads A_sym in the level's precision (no BF16 copy)
        if (cheb)
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, true, true, false>, sg, a));
        else
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, false, true, false>, sg, a));
        launched = true;
    } else if (ach) {
        if (cheb)
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, true, false, true>, sg, a));
        else
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, false, false, true>, sg, a));
        launched = true;
    }
    if constexpr (std::is_same<T, float>::value) {
        if (h16 && !launched) {
            if (cheb)
                HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<float, true, true, false, false>, sg, a));
            else
                HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<float, true, false, false, false>, sg, a));
            launched = true;
        }
    }
    if (!launched) {
        if (cheb)
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, true, false, false>, sg, a));
        else
            HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_s<T, false, false, false, false>, sg, a));
    }
    count_launch();
    prof_end(c, HYEL_K_GMRES_S, ev, 0.0);
}

// Algorithm 2: y = D x - C A^-1 (B x), y indexed by the S-level state
template <typename T>
void schur_op(Rec &R, Workspace &w, const hyel_solver_params &p, const T *x, T *y, const int *yk, int64_t ystride) {
    Ctx &c = *R.c;
    const int64_t N = c.mesh.N;
    T *xbar = Sys<T>::vec(w, 4, N);
    T *xtil = Sys<T>::vec(w, 5, N);
    spmv_B<T>(c, Sys<T>::B(c), x, xbar, nullptr);
    if (p.inner_solver == HYEL_INNER_CG_SYM) {
        // one cooperative launch of the CG inner solve on A_sym
        CgArgs<T> cg = cg_args<T>(c, w, p, xbar, xtil);
        Level<T> &La = Sys<T>::la(w);
        bar_reset(c, La.bar);
        cudaLaunchConfig_t cfg = coop_config(c, resident_grid(c, (const void *)k_cg_a<T>));
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        HYEL_CK(cudaLaunchKernelEx(&cfg, k_cg_a<T>, cg));
        count_launch();
    } else {
        a_solve<T>(R, w, w.states + ST_INNER, p.inner, xbar, xtil);
    }
    spmv_DC_ind<T>(c, Sys<T>::D(c), Sys<T>::C(c), x, xtil, y, ystride, yk);
}

// The S^-solve of SIMPLE: one cooperative launch of k_gmres_shat on the S-level
// buffers and state
template <typename T>
void shat_solve(Rec &R, Workspace &w, const hyel_solver_params &p, const T *b, T *x) {
    Ctx &c = *R.c;
    const int64_t N = c.mesh.N;
    Level<T> &Ls = Sys<T>::ls(w);
    const SchurHat &h = *c.sh;
    ShArgs<T> sa;
    sa.slice_ptr = h.slice_ptr;
    sa.row_len = h.row_len;
    sa.col = h.col;
    if constexpr (std::is_same<T, double>::value)
        sa.val = h.v64;
    else
        sa.val = h.v32;
    sa.dinv = Sys<T>::shat(c);
    const bool cheb = p.s_precond == HYEL_SPREC_CHEB;
    sa.zc = nullptr;
    sa.ch = ChebArgs<T>{};
    if (cheb) {
        T *cb = Sys<T>::vec(w, 11, N);
        float *db = reinterpret_cast<float *>(cb + 2 * N);
        sa.zc = cb;
        sa.ch = cheb_args<T>(c, p.s_cheb_degree, p.s_cheb_ratio, cb + N, db, db + N);
    }
    GmArgs<T> &g = sa.g;
    g.N = N;
    g.b = b;
    g.x = x;
    g.V = Ls.V;
    g.U0 = Ls.z;
    g.U1 = Ls.z2;
    g.H = Ls.H;
    g.partial = Ls.pg_partial;
    g.bar = Ls.bar;
    g.st = w.states + ST_S;
    g.m = std::min(p.s.restart, Ls.m);
    g.maxit = p.s.maxit;
    g.rtol = p.s.rtol;
    g.atol = p.s.atol;
    g.eta2 = p.s.rtol >= kPgLoose<T> ? kPgEta2<T> : 0.5;
    // one iteration: S^ values and columns, the gathered vector, and (Chebyshev)
    // the polynomial's FP32 products and passes
    g.it_fixed = (double)h.nnz * (sizeof(T) + 4.0) + (double)N * (2.0 * sizeof(T) + 8.0);
    if (cheb) {
        const int d = p.s_cheb_degree;
        g.it_fixed += (d - 1) * ((double)h.nnz * 8.0 + (double)N * (sizeof(T) + 8.0)) +
                      (3.0 + 6.0 * (d - 1)) * (double)N * sizeof(T);
    }
    g.it_unit = (double)N * sizeof(T);
    bar_reset(c, Ls.bar);
    cudaLaunchConfig_t cfg = coop_config(c, cheb ? Ls.pg_grid_shc : Ls.pg_grid_sh);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_GMRES_S, &ev);
    if (cheb)
        HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_shat<T, true>, sa));
    else
        HYEL_CK(cudaLaunchKernelEx(&cfg, k_gmres_shat<T, false>, sa));
    count_launch();
    prof_end(c, HYEL_K_GMRES_S, ev, 0.0);
}

// S x_p = r_p (Algorithm 1 step 3): the persistent S-solve with block-Jacobi
// A-solves; a kernel-per-step loop with multigrid ones
template <typename T>
void s_level(Rec &R, Workspace &w, const hyel_solver_params &p, const T *rp, T *xp) {
    Ctx &c = *R.c;
    if (!w.a_amg) {
        s_solve<T>(R, w, p, rp, xp);
    } else {
        Level<T> &Ls = Sys<T>::ls(w);
        LevelState *sst = w.states + ST_S;
        gm_solve<T, 1>(R, Ls, sst, p.s, rp, xp, Sys<T>::shat(c), nullptr,
                       [&]() { schur_op<T>(R, w, p, Ls.z, Ls.V, &sst->k, Ls.n); }, true);
    }
}

// The block preconditioner: (rv, rp) -> (xv, xp). LDU is Algorithm 1 (SCR);
// DU, D and SIMPLE are the variants of §4.3–4.4.
template <typename T>
void pscr(Rec &R, Workspace &w, const hyel_solver_params &p, const T *rv, const T *rp, T *xv, T *xp) {
    Ctx &c = *R.c;
    const int64_t N = c.mesh.N;
    T *xhat = Sys<T>::vec(w, 0, N);
    T *rp2 = Sys<T>::vec(w, 1, N);
    T *rv2 = Sys<T>::vec(w, 2, N);
    switch (p.block_precond) {
        case HYEL_BLOCK_DU:
            // S x_p = r_p; A x_v = r_v - B x_p
            s_level<T>(R, w, p, rp, xp);
            spmv_B<T>(c, Sys<T>::B(c), xp, rv2, rv);
            a_solve<T>(R, w, w.states + ST_A2, p.a, rv2, xv);
            return;
        case HYEL_BLOCK_D:
            // A x_v = r_v; S x_p = r_p
            a_solve<T>(R, w, w.states + ST_A1, p.a, rv, xv);
            s_level<T>(R, w, p, rp, xp);
            return;
        case HYEL_BLOCK_SIMPLE:
            // A xhat = r_v; S^ x_p = r_p - C xhat; x_v = xhat - diag(A)^-1 B x_p
            a_solve<T>(R, w, w.states + ST_A1, p.a, rv, xhat);
            spmv_C<T>(c, Sys<T>::C(c), xhat, rp2, rp);
            shat_solve<T>(R, w, p, rp2, xp);
            spmv_B<T>(c, Sys<T>::B(c), xp, rv2, nullptr);
            LAUNCH(k_simple_update<T><<<blocks_for(N, 256), 256, 0, c.stream>>>(c.mesh.diag_slot, Sys<T>::A(c), xhat,
                                                                                rv2, xv, N));
            return;
        default:
            break;
    }
    // 1: A xhat = r_v
    a_solve<T>(R, w, w.states + ST_A1, p.a, rv, xhat);
    // 2: r_p <- r_p - C xhat
    spmv_C<T>(c, Sys<T>::C(c), xhat, rp2, rp);
    // 3: S x_p = r_p, right-preconditioned by diag(S^)^-1 or the Chebyshev
    // polynomial in S^: one persistent kernel with block-Jacobi A-solves
    s_level<T>(R, w, p, rp2, xp);
    // 4: r_v <- r_v - B x_p
    spmv_B<T>(c, Sys<T>::B(c), xp, rv2, rv);
    // 5: A x_v = r_v
    a_solve<T>(R, w, w.states + ST_A2, p.a, rv2, xv);
}

// The outer FGMRES on the scaled system: b -> xs (both FP64, fixed buffers).
void outer_solve(Rec &R, Workspace &w, const hyel_solver_params &p, const double *b, double *xs) {
    Ctx &c = *R.c;
    const int64_t N = c.mesh.N, n = 4 * N;
    Level<double> &L = w.outer;
    LevelState *st = w.states + ST_OUTER;
    auto prec = [&]() {
        if (p.precision == HYEL_PREC_FP64) {
            double *vin = Sys<double>::vec(w, 6, N), *zout = Sys<double>::vec(w, 7, N);
            LAUNCH(k_copy_ind<double, double><<<blocks_for(n, 256), 256, 0, c.stream>>>(L.V, vin, n, st, n, 0));
            pscr<double>(R, w, p, vin, vin + 3 * N, zout, zout + 3 * N);
            LAUNCH(k_copy_ind<double, double><<<blocks_for(n, 256), 256, 0, c.stream>>>(zout, L.Z, n, st, 0, n));
        } else {
            float *vf = Sys<float>::vec(w, 6, N), *zf = Sys<float>::vec(w, 7, N);
            LAUNCH(k_copy_ind<double, float><<<blocks_for(n, 256), 256, 0, c.stream>>>(L.V, vf, n, st, n, 0));
            pscr<float>(R, w, p, vf, vf + 3 * N, zf, zf + 3 * N);
            LAUNCH(k_copy_ind<float, double><<<blocks_for(n, 256), 256, 0, c.stream>>>(zf, L.Z, n, st, 0, n));
        }
    };
    auto op = [&]() { spmv_full64_ind(c, c.mat.As, c.mat.Bs, c.mat.Cs, c.mat.Ds, L.Z, L.V, n, &st->k); };
    gm_solve<double, 2>(R, L, st, p.outer, b, xs, nullptr, prec, op, false);
}

double seconds_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct CaptureScope {
    int count = 0;
    int *saved;
    CaptureScope() : saved(g_capture_count) { g_capture_count = &count; }
    ~CaptureScope() { g_capture_count = saved; }
};

// Build (or reuse) the graph of the nested solve for these parameters.
void ensure_graph(Ctx &c, Workspace &w, const hyel_solver_params &p) {
    if (w.exec && w.have_key && same_params(w.key, p)) return;
    if (w.exec) cudaGraphExecDestroy(w.exec);
    if (w.graph) cudaGraphDestroy(w.graph);
    w.exec = nullptr;
    w.graph = nullptr;
    w.sites.clear();
    if (w.streams.empty()) {
        cudaStream_t s;
        HYEL_CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        w.streams.push_back(s);
    }
    HYEL_CK(cudaStreamSynchronize(c.stream));
    const int64_t N = c.mesh.N;
    cudaStream_t user = c.stream;
    c.stream = w.streams[0];
    CaptureScope scope;
    Rec R;
    R.c = &c;
    R.graph = true;
    R.streams = &w.streams;
    R.sites = &w.sites;
    R.capture_count = &scope.count;
    cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        c.stream = user;
        check_cuda(e, "cudaStreamBeginCapture");
    }
    try {
        outer_solve(R, w, p, Sys<double>::vec(w, 8, N), Sys<double>::vec(w, 9, N));
    } catch (...) {
        cudaGraph_t g;
        cudaStreamEndCapture(c.stream, &g);
        if (g) cudaGraphDestroy(g);
        c.stream = user;
        throw;
    }
    e = cudaStreamEndCapture(c.stream, &w.graph);
    c.stream = user;
    check_cuda(e, "cudaStreamEndCapture");
    int nested = 0;
    for (auto &s : w.sites) nested += s.body_nodes + s.init_nodes;
    w.top_nodes = scope.count - nested;
    check_cuda(cudaGraphInstantiate(&w.exec, w.graph, 0), "cudaGraphInstantiate");
    w.key = p;
    w.have_key = true;
}

// Scaling, and the operators the parameters need: multigrid levels, the
// explicit S^ and its interval (FP64 copy for SIMPLE's FP64 S^-solve).
void prepare(Ctx &c, const hyel_solver_params &p) {
    solve_setup(c);
    if (p.a_precond == HYEL_APREC_AMG && !c.mat.amg_ready) {
        amg_numeric(c);
        c.mat.amg_ready = true;
    }
    if (p.s_precond == HYEL_SPREC_CHEB || p.block_precond == HYEL_BLOCK_SIMPLE) shat_setup(c);
    if (p.block_precond == HYEL_BLOCK_SIMPLE && p.precision == HYEL_PREC_FP64) shat_ensure64(c);
    if (p.inner_solver == HYEL_INNER_CG_SYM) asym_setup(c);
    if (p.a_precond == HYEL_APREC_CHEB) acheb_setup(c);
}

// The parameters a recording or launch reads from the workspace
void bind_params(Workspace &w, const hyel_solver_params &p) {
    w.a_cheb = p.a_precond == HYEL_APREC_CHEB ? p.a_cheb_degree : 0;
}

// Kernel executions of the last solve from the level statistics.
int64_t executed_kernels(Workspace &w) {
    int64_t total = w.top_nodes;
    for (auto &s : w.sites) {
        const LevelState &hs = w.h_states[s.st - w.states];
        total += (int64_t)s.body_nodes * hs.its + (int64_t)s.init_nodes * hs.solves;
    }
    return total;
}

}  // namespace

void solve_nested(Ctx &c, const hyel_solver_params &p, const double *rhs, double *x, hyel_solve_stats *out) {
    check_params(p);
    if (!c.mat.assembled) fail(HYEL_ESTATE, "solve: nothing assembled");
    auto t0 = std::chrono::steady_clock::now();
    prepare(c, p);
    Workspace &w = workspace(c, p);
    bind_params(w, p);
    if (p.graph) ensure_graph(c, w, p);
    HYEL_CK(cudaStreamSynchronize(c.stream));
    const double ms_setup = 1e3 * seconds_since(t0);
    auto t1 = std::chrono::steady_clock::now();
    const int64_t N = c.mesh.N, n = 4 * N;
    double *b = Sys<double>::vec(w, 8, N);
    double *xs = Sys<double>::vec(w, 9, N);
    double *r = Sys<double>::vec(w, 10, N);
    HYEL_CK(cudaMemsetAsync(w.states, 0, sizeof(LevelState) * 5, c.stream));
    // r* = W r
    LAUNCH(k_mul<<<blocks_for(n, 256), 256, 0, c.stream>>>(rhs, c.mat.w, b, n));
    if (p.graph) {
        HYEL_CK(cudaGraphLaunch(w.exec, c.stream));
    } else {
        Rec R;
        R.c = &c;
        R.graph = false;
        R.check_every = p.check_every;
        outer_solve(R, w, p, b, xs);
    }
    // true residual of the scaled system and unscaling x = W x*
    spmv_full64_ind(c, c.mat.As, c.mat.Bs, c.mat.Cs, c.mat.Ds, xs, r, 0, nullptr);
    LAUNCH(k_sub<double><<<blocks_for(n, 256), 256, 0, c.stream>>>(b, r, n));
    LAUNCH(k_sumsq<<<w.outer.grid, kThreads, 0, c.stream>>>(r, n, w.outer.partial, w.outer.counter, c.red + 8));
    LAUNCH(k_mul<<<blocks_for(n, 256), 256, 0, c.stream>>>(xs, c.mat.w, x, n));
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_red + 8, c.red + 8, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaMemcpyAsync(w.h_states, w.states, sizeof(LevelState) * 5, cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (p.graph) {
        const int64_t k = executed_kernels(w);
        for (int64_t q = 0; q < k; q++) count_launch();
    }
    const LevelState *hs = w.h_states;
    if (c.prof.on && !p.graph) {
        c.prof.bytes[HYEL_K_GMRES_A] += hs[ST_A1].alg_bytes + hs[ST_A2].alg_bytes;
        c.prof.bytes[HYEL_K_GMRES_S] += hs[ST_S].alg_bytes + hs[ST_INNER].alg_bytes;
    }
    const double bn = hs[ST_OUTER].bnorm;
    const double rel = bn > 0 ? std::sqrt(c.h_red[8]) / bn : std::sqrt(c.h_red[8]);
    int st = HYEL_OK;
    if (hs[ST_OUTER].status_any & 1) st = HYEL_ENAN;
    else if (hs[ST_OUTER].status_any & 2) st = HYEL_EBREAKDOWN;
    else if (!hs[ST_OUTER].converged) st = HYEL_ENOCONV;
    for (int q = 1; q < 5 && st == HYEL_OK; q++) {
        if (hs[q].status_any & 1) st = HYEL_ENAN;
    }
    if (!std::isfinite(rel)) st = HYEL_ENAN;
    const bool barrier_timeout =
        ((hs[ST_A1].status_any | hs[ST_A2].status_any | hs[ST_S].status_any | hs[ST_INNER].status_any) & 8) != 0;
    if (barrier_timeout) st = HYEL_ECUDA;
    if (out) {
        out->status = st;
        out->outer_its = (int32_t)hs[ST_OUTER].its;
        out->a_its = hs[ST_A1].its + hs[ST_A2].its;
        out->s_its = hs[ST_S].its;
        out->inner_its = hs[ST_INNER].its;
        out->a_solves = hs[ST_A1].solves + hs[ST_A2].solves;
        out->s_solves = hs[ST_S].solves;
        out->inner_solves = hs[ST_INNER].solves;
        out->rel_residual = rel;
        out->ms_setup = ms_setup;
        out->ms_solve = 1e3 * seconds_since(t1);
    }
    if (st != HYEL_OK) {
        const char *what = barrier_timeout      ? "a grid barrier of a persistent solve kernel timed out"
                           : st == HYEL_ENOCONV ? "outer FGMRES reached its iteration cap"
                           : st == HYEL_ENAN    ? "NaN or Inf in the solve"
                           : st == HYEL_EBREAKDOWN ? "GMRES breakdown without convergence"
                                                   : "solve failed";
        fail(st, std::string("solve_nested: ") + what);
    }
}

namespace {

int coop_grid(Ctx &c, const void *kernel) {
    int occ = 0;
    HYEL_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kPgThreads, 0));
    if (occ < 1) fail(HYEL_ECUDA, "schur_hat: cooperative kernel does not fit on an SM");
    const int64_t need = std::max<int64_t>(1, (c.mesh.N + 31) / 32);
    return (int)std::min<int64_t>((int64_t)occ * c.num_sms, need);
}

void coop_launch(Ctx &c, int grid, const void *kernel, void **args) {
    HYEL_CK(cudaLaunchCooperativeKernel(kernel, dim3((unsigned)grid), dim3(kPgThreads), args, 0, c.stream));
    count_launch();
}

}  // namespace

// Eigenvalues of a small symmetric matrix (n x n, row-major, overwritten) by
// cyclic Jacobi rotations (Golub and Van Loan, Matrix Computations, §8.5):
// each rotation zeroes one off-diagonal pair; sweeps until the off-diagonal
// part is negligible against the whole.
static void sym_eigenvalues(std::vector<double> &a, int n, std::vector<double> &ev) {
    for (int sweep = 0; sweep < 60; sweep++) {
        double off = 0.0, all = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = 0; q < n; q++) {
                all += a[p * n + q] * a[p * n + q];
                if (p != q) off += a[p * n + q] * a[p * n + q];
            }
        if (off <= 1e-30 * all || off == 0.0) break;
        for (int p = 0; p < n - 1; p++)
            for (int q = p + 1; q < n; q++) {
                const double apq = a[p * n + q];
                if (apq == 0.0) continue;
                const double th = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
                const double t = (th >= 0.0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int r = 0; r < n; r++) {  // columns p, q
                    const double x = a[r * n + p], y = a[r * n + q];
                    a[r * n + p] = cs * x - sn * y;
                    a[r * n + q] = sn * x + cs * y;
                }
                for (int r = 0; r < n; r++) {  // rows p, q
                    const double x = a[p * n + r], y = a[q * n + r];
                    a[p * n + r] = cs * x - sn * y;
                    a[q * n + r] = sn * x + cs * y;
                }
            }
    }
    ev.resize(n);
    for (int p = 0; p < n; p++) ev[p] = a[p * n + p];
    std::sort(ev.begin(), ev.end());
}

void shat_bounds(Ctx &c) {
    SchurHat &h = *c.sh;
    const int64_t N = c.mesh.N;
    const int K1 = kRitzSteps + 1;
    const int grid = coop_grid(c, (const void *)k_shat_arnoldi);
    const size_t gmax = (size_t)(2048 / kPgThreads) * c.num_sms;
    if (!h.partial) h.partial = dalloc_n<double>(c, 2 * gmax * K1);
    if (!h.arn_V) h.arn_V = dalloc_n<float>(c, (size_t)K1 * N);
    if (!h.arn_H) h.arn_H = dalloc_n<double>(c, (size_t)K1 * kRitzSteps);
    ArnArgs a;
    a.slice_ptr = h.slice_ptr;
    a.row_len = h.row_len;
    a.col = h.col;
    a.val = h.v32;
    a.dinv = c.mat.shat64;
    a.V = h.arn_V;
    a.U = reinterpret_cast<float *>(h.work);
    a.Sq = a.U + 2 * N;
    a.H = h.arn_H;
    a.partial = h.partial;
    a.bar = h.bar;
    a.N = N;
    bar_reset(c, h.bar);
    HYEL_CK(cudaMemsetAsync(h.arn_H, 0, sizeof(double) * K1 * kRitzSteps, c.stream));
    void *args[] = {&a};
    coop_launch(c, grid, (const void *)k_shat_arnoldi, args);
    std::vector<double> H((size_t)K1 * kRitzSteps);
    HYEL_CK(cudaMemcpyAsync(H.data(), h.arn_H, sizeof(double) * H.size(), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (!std::isfinite(H[0])) fail(HYEL_ENAN, "schur_hat: Arnoldi on S^ met NaN/Inf (or a grid barrier timed out)");
    // leading block up to the first vanishing subdiagonal entry
    int k = kRitzSteps;
    for (int j = 0; j < kRitzSteps; j++) {
        for (int l = 0; l <= j + 1; l++)
            if (!std::isfinite(H[(size_t)j * K1 + l])) fail(HYEL_ENAN, "schur_hat: Arnoldi on S^ met NaN/Inf");
        if (!(H[(size_t)j * K1 + j + 1] > 0.0)) {
            k = j + 1;
            break;
        }
    }
    std::vector<double> S((size_t)k * k), ev;
    for (int r = 0; r < k; r++)
        for (int q = 0; q < k; q++) S[r * k + q] = 0.5 * (H[(size_t)q * K1 + r] + H[(size_t)r * K1 + q]);
    sym_eigenvalues(S, k, ev);
    if (!(ev.back() > 0.0)) fail(HYEL_ENAN, "schur_hat: diag(S^)^-1 S^ has no positive Ritz value");
    double b[2] = {ev.front() / kRitzLow, kRitzSafety * ev.back()};
    h.h_bounds[0] = b[0];
    h.h_bounds[1] = b[1];
    HYEL_CK(cudaMemcpy(h.bounds, b, sizeof b, cudaMemcpyHostToDevice));
}

void shat_setup(Ctx &c) {
    solve_setup(c);
    if (c.mat.shat_ready) return;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_SCHUR_HAT, &ev);
    shat_numeric<float>(c);
    const SchurHat &h = *c.sh;
    const DeviceMesh &m = c.mesh;
    // numeric (FP32): D, C, column and diag(A) per block slot, B per
    // neighbour slot, positions, rows written; Arnoldi (FP32): S^ and the
    // basis passes per step
    // (the interval of the first Newton iteration of a time step is kept at
    // the later ones when keep_intervals is set: the matrix moves little)
    const bool estimate = !(c.keep_intervals && h.h_bounds[1] > 0.0);
    const double bytes = (double)m.nnzb * (4.0 + 12.0 + 4.0 + 12.0) + (double)m.N * (12.0 + 8.0) +
                         2.0 * (double)h.ncontrib + 4.0 * (double)h.nslots +
                         (estimate ? kRitzSteps * ((double)h.nnz * 8.0 + (double)m.N * (8.0 + 4.0 * (2 * kRitzSteps + 4)))
                                   : 0.0);
    if (estimate) shat_bounds(c);
    prof_end(c, HYEL_K_SCHUR_HAT, ev, bytes);
    c.mat.shat_ready = true;
}

void acheb_free(Ctx &c) {
    delete c.ach;  // device arrays belong to the context's allocation list
    c.ach = nullptr;
}

void acheb_setup(Ctx &c) {
    solve_setup(c);
    if (c.mat.acheb_ready) return;
    if (c.keep_intervals && c.ach && c.ach->h_bounds[1] > 0.0) {
        c.mat.acheb_ready = true;  // the first Newton iteration's interval
        return;
    }
    const DeviceMesh &m = c.mesh;
    const int64_t N = m.N, n = 3 * N;
    const int K1 = kRitzSteps + 1;
    if (!c.ach) {
        AChebState *h = new AChebState();
        c.ach = h;
        const size_t gmax = (size_t)(2048 / kPgThreads) * c.num_sms;
        h->bounds = dalloc_n<double>(c, 2);
        h->V = dalloc_n<float>(c, (size_t)K1 * n);
        h->U = dalloc_n<float>(c, 3 * (size_t)n);
        h->H = dalloc_n<double>(c, (size_t)K1 * kRitzSteps);
        h->partial = dalloc_n<double>(c, 2 * gmax * K1);
        h->bar = (unsigned *)dalloc(c, kBarAlloc * sizeof(unsigned));
        h->work = dalloc_n<double>(c, (size_t)n);
        h->dwork = dalloc_n<float>(c, 2 * (size_t)n);
    }
    AChebState &h = *c.ach;
    AArnArgs a;
    a.slice_ptr = m.slice_ptr;
    a.row_len = m.row_len;
    a.col = m.col;
    a.diag_slot = m.diag_slot;
    a.Af = c.mat.Af;
    a.jac = c.mat.jac32;
    a.V = h.V;
    a.U = h.U;
    a.H = h.H;
    a.partial = h.partial;
    a.bar = h.bar;
    a.N = N;
    bar_reset(c, h.bar);
    HYEL_CK(cudaMemsetAsync(h.H, 0, sizeof(double) * K1 * kRitzSteps, c.stream));
    void *args[] = {&a};
    coop_launch(c, coop_grid(c, (const void *)k_a_arnoldi), (const void *)k_a_arnoldi, args);
    std::vector<double> H((size_t)K1 * kRitzSteps);
    HYEL_CK(cudaMemcpyAsync(H.data(), h.H, sizeof(double) * H.size(), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (!std::isfinite(H[0])) fail(HYEL_ENAN, "a_cheb: Arnoldi on M^-1 A met NaN/Inf (or a grid barrier timed out)");
    int k = kRitzSteps;
    for (int j = 0; j < kRitzSteps; j++) {
        for (int l = 0; l <= j + 1; l++)
            if (!std::isfinite(H[(size_t)j * K1 + l])) fail(HYEL_ENAN, "a_cheb: Arnoldi on M^-1 A met NaN/Inf");
        if (!(H[(size_t)j * K1 + j + 1] > 0.0)) {
            k = j + 1;
            break;
        }
    }
    std::vector<double> S((size_t)k * k), ev;
    for (int r = 0; r < k; r++)
        for (int q = 0; q < k; q++) S[r * k + q] = 0.5 * (H[(size_t)q * K1 + r] + H[(size_t)r * K1 + q]);
    sym_eigenvalues(S, k, ev);
    if (!(ev.back() > 0.0)) fail(HYEL_ENAN, "a_cheb: M^-1 A has no positive Ritz value");
    double b[2] = {ev.front() / kRitzLow, kRitzSafety * ev.back()};
    h.h_bounds[0] = b[0];
    h.h_bounds[1] = b[1];
    HYEL_CK(cudaMemcpy(h.bounds, b, sizeof b, cudaMemcpyHostToDevice));
    c.mat.acheb_ready = true;
}

void acheb_apply(Ctx &c, int degree, const double *x, double *y) {
    if (degree < 1 || degree > kChebMaxDegree) fail(HYEL_EINVAL, "a_cheb_apply: degree must be in [1, 16]");
    if (!c.ach || !c.mat.acheb_ready) fail(HYEL_ESTATE, "a_cheb_apply: no interval for the current assembly");
    AChebState &h = *c.ach;
    const DeviceMesh &m = c.mesh;
    const int64_t n = 3 * m.N;
    PgArgs<double> a{};
    a.slice_ptr = m.slice_ptr;
    a.row_len = m.row_len;
    a.col = m.col;
    a.jac = c.mat.jac64;
    a.ac.Af = c.mat.Af;
    a.ac.A = c.mat.As;
    a.ac.bounds = h.bounds;
    a.ac.degree = degree;
    a.ac.r = h.work;
    a.ac.d0 = h.dwork;
    a.ac.d1 = h.dwork + n;
    a.g.N = m.N;
    a.g.bar = h.bar;
    unsigned *status = c.err;
    bar_reset(c, h.bar);
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    void *args[] = {&a, (void *)&x, (void *)&y, &status};
    coop_launch(c, coop_grid(c, (const void *)k_acheb_apply), (const void *)k_acheb_apply, args);
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & 8u) fail(HYEL_ECUDA, "a_cheb_apply: a grid barrier timed out");
}

void shat_cheb_apply(Ctx &c, int matrix, int degree, double ratio, const double *x, double *y) {
    check_cheb(degree, ratio);
    if (matrix != HYEL_MAT_SCALED64 && matrix != HYEL_MAT_SCALED32)
        fail(HYEL_EINVAL, "schur_hat_cheb: matrix must be HYEL_MAT_SCALED64 or HYEL_MAT_SCALED32");
    if (!c.sh || !c.mat.shat_ready) fail(HYEL_ESTATE, "schur_hat: S^ is not built for the current assembly");
    SchurHat &h = *c.sh;
    const int64_t N = c.mesh.N;
    unsigned *bar = h.bar, *status = c.err;
    int64_t n = N;
    bar_reset(c, h.bar);
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    if (matrix == HYEL_MAT_SCALED64) {
        shat_ensure64(c);
        ChebArgs<double, double> ch = cheb_args<double, double>(c, degree, ratio, h.work, h.work + N, h.work + 2 * N);
        void *args[] = {&ch, (void *)&x, (void *)&y, &n, &bar, &status};
        coop_launch(c, coop_grid(c, (const void *)k_cheb_apply<double>), (const void *)k_cheb_apply<double>, args);
    } else {
        float *db = reinterpret_cast<float *>(h.work + N);
        ChebArgs<double, float> ch = cheb_args<double, float>(c, degree, ratio, h.work, db, db + N);
        void *args[] = {&ch, (void *)&x, (void *)&y, &n, &bar, &status};
        coop_launch(c, coop_grid(c, (const void *)k_cheb_apply<float>), (const void *)k_cheb_apply<float>, args);
    }
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & 8u) fail(HYEL_ECUDA, "schur_hat: a grid barrier timed out");
}

void schur_apply(Ctx &c, const hyel_solver_params &p, const double *x, double *y, hyel_solve_stats *out) {
    check_params(p);
    if (!c.mat.assembled) fail(HYEL_ESTATE, "schur_apply: nothing assembled");
    prepare(c, p);
    Workspace &w = workspace(c, p);
    bind_params(w, p);
    const int64_t N = c.mesh.N;
    HYEL_CK(cudaMemsetAsync(w.states, 0, sizeof(LevelState) * 5, c.stream));
    Rec R;
    R.c = &c;
    R.graph = false;
    R.check_every = p.check_every;
    if (p.precision == HYEL_PREC_FP64) {
        schur_op<double>(R, w, p, x, y, nullptr, 0);
    } else {
        float *xf = Sys<float>::vec(w, 6, N), *yf = Sys<float>::vec(w, 7, N);
        LAUNCH(k_copy_ind<double, float><<<blocks_for(N, 256), 256, 0, c.stream>>>(x, xf, N, nullptr, 0, 0));
        schur_op<float>(R, w, p, xf, yf, nullptr, 0);
        LAUNCH(k_copy_ind<float, double><<<blocks_for(N, 256), 256, 0, c.stream>>>(yf, y, N, nullptr, 0, 0));
    }
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(w.h_states, w.states, sizeof(LevelState) * 5, cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (out) {
        *out = hyel_solve_stats{};
        out->status = (w.h_states[ST_INNER].status_any & 8)   ? HYEL_ECUDA
                      : (w.h_states[ST_INNER].status_any & 1) ? HYEL_ENAN
                                                               : HYEL_OK;
        out->inner_its = w.h_states[ST_INNER].its;
        out->inner_solves = w.h_states[ST_INNER].solves;
    }
    if (w.h_states[ST_INNER].status_any & 8)
        fail(HYEL_ECUDA, "schur_apply: a grid barrier of the inner A-solve timed out");
    if (w.h_states[ST_INNER].status_any & 1) fail(HYEL_ENAN, "schur_apply: NaN or Inf in the inner A-solve");
}

void block_precond_apply(Ctx &c, const hyel_solver_params &p, const double *r, double *z, hyel_solve_stats *out) {
    check_params(p);
    if (!c.mat.assembled) fail(HYEL_ESTATE, "block_precond_apply: nothing assembled");
    prepare(c, p);
    Workspace &w = workspace(c, p);
    bind_params(w, p);
    const int64_t N = c.mesh.N, n = 4 * N;
    HYEL_CK(cudaMemsetAsync(w.states, 0, sizeof(LevelState) * 5, c.stream));
    Rec R;
    R.c = &c;
    R.graph = false;
    R.check_every = p.check_every;
    if (p.precision == HYEL_PREC_FP64) {
        pscr<double>(R, w, p, r, r + 3 * N, z, z + 3 * N);
    } else {
        float *vf = Sys<float>::vec(w, 6, N), *zf = Sys<float>::vec(w, 7, N);
        LAUNCH(k_copy_ind<double, float><<<blocks_for(n, 256), 256, 0, c.stream>>>(r, vf, n, nullptr, 0, 0));
        pscr<float>(R, w, p, vf, vf + 3 * N, zf, zf + 3 * N);
        LAUNCH(k_copy_ind<float, double><<<blocks_for(n, 256), 256, 0, c.stream>>>(zf, z, n, nullptr, 0, 0));
    }
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(w.h_states, w.states, sizeof(LevelState) * 5, cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    const LevelState *hs = w.h_states;
    int st = HYEL_OK;
    for (int q = 1; q < 5; q++) {
        if (hs[q].status_any & 8) st = HYEL_ECUDA;
        else if ((hs[q].status_any & 1) && st == HYEL_OK) st = HYEL_ENAN;
    }
    if (out) {
        *out = hyel_solve_stats{};
        out->status = st;
        out->a_its = hs[ST_A1].its + hs[ST_A2].its;
        out->s_its = hs[ST_S].its;
        out->inner_its = hs[ST_INNER].its;
        out->a_solves = hs[ST_A1].solves + hs[ST_A2].solves;
        out->s_solves = hs[ST_S].solves;
        out->inner_solves = hs[ST_INNER].solves;
    }
    if (st != HYEL_OK) fail(st, "block_precond_apply: a sub-solve failed (NaN/Inf or a barrier timeout)");
}

}  // namespace hyel
