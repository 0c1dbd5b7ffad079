// Sparse kernels on the SELL-32 block storage: symmetric diagonal scaling
// (§4.1), FP32 copies, 3x3 block-Jacobi inverses of A, the diagonal of
// S^ = D - C diag(A)^-1 B (§4.2), and the block SpMVs used by the solver.
//
// SpMV mapping: one thread per block row (node); a warp covers one 32-row
// slice, so every load of a block component is one coalesced 32-wide access.
// x is gathered by column (three consecutive values per node). Accumulation
// is in the value type (FP64, or FP32 for the single-precision copies), in a
// fixed order: results are bitwise reproducible.
#include <cuda_bf16.h>

#include <cmath>

#include "internal.h"

namespace hyel {

namespace {

struct ScaleArgs {
    const int32_t *diag_slot, *col_slice, *slice_ptr, *row_len, *col, *mirror;
    const double *A, *B, *C, *D;
    double *As, *Bs, *Cs, *Ds;
    float *Af, *Bf, *Cf, *Df;
    uint4 *Ah8;
    uint16_t *Ah1;
    float *Ahs;
    double *Ams;
    float *Amf;
    uint4 *Amh8;
    uint16_t *Amh1;
    float *Amhs;
    double *w;  // [4N]
    double *jac64;
    float *jac32;
    double *rdiag64;  // [3N] 1 / A_ii[s][s]
    double *shat64;
    float *shat32;
    unsigned *err;
    int64_t N, nslots;
};

__global__ void k_scale_diag(ScaleArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int64_t q = a.diag_slot[i], b = q >> 5, t = q & 31;
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const double d = fabs(a.A[(b * 9 + 4 * r) * 32 + t]);
        a.w[3 * i + r] = d >= 1e-15 ? 1.0 / sqrt(d) : 1.0;
    }
    const double d = fabs(a.D[b * 32 + t]);
    a.w[3 * a.N + i] = d >= 1e-15 ? 1.0 / sqrt(d) : 1.0;
}

// BF16 copy of one 3x3 block with one FP32 scale: s = float(max |v|),
// e_k = bf16_rn(float(v_k) / s); all zero for a zero block
__device__ __forceinline__ void quant_block(const double v[9], int64_t q, uint4 *h8, uint16_t *h1, float *hs) {
    double amax = 0.0;
#pragma unroll
    for (int k = 0; k < 9; k++) amax = fmax(amax, fabs(v[k]));
    const float sc = (float)amax;
    unsigned short h[9];
#pragma unroll
    for (int k = 0; k < 9; k++)
        h[k] = sc > 0.0f ? __bfloat16_as_ushort(__float2bfloat16_rn(__fdiv_rn((float)v[k], sc))) : (unsigned short)0;
    h8[q] = make_uint4(h[0] | ((unsigned)h[1] << 16), h[2] | ((unsigned)h[3] << 16), h[4] | ((unsigned)h[5] << 16),
                       h[6] | ((unsigned)h[7] << 16));
    h1[q] = h[8];
    hs[q] = sc;
}

__global__ void k_scale_values(ScaleArgs a) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.nslots) return;
    const int64_t b = q >> 5;
    const int t = (int)(q & 31);
    const int s = a.col_slice[b];
    const int64_t r = (int64_t)s * 32 + t;
    double wr[3] = {0, 0, 0}, wc[3] = {0, 0, 0}, wpr = 0, wpc = 0;
    if (r < a.N && b - a.slice_ptr[s] < a.row_len[r]) {
        const int64_t c = a.col[q];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            wr[k] = a.w[3 * r + k];
            wc[k] = a.w[3 * c + k];
        }
        wpr = a.w[3 * a.N + r];
        wpc = a.w[3 * a.N + c];
    }
    double v[9];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const int64_t o = (b * 9 + 3 * i + j) * 32 + t;
            v[3 * i + j] = a.A[o] * wr[i] * wc[j];
            a.As[o] = v[3 * i + j];
            a.Af[o] = (float)v[3 * i + j];
        }
    quant_block(v, q, a.Ah8, a.Ah1, a.Ahs);
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const int64_t o = (b * 3 + i) * 32 + t;
        const double vb = a.B[o] * wr[i] * wpc;
        const double vc = a.C[o] * wpr * wc[i];
        a.Bs[o] = vb;
        a.Bf[o] = (float)vb;
        a.Cs[o] = vc;
        a.Cf[o] = (float)vc;
    }
    const int64_t o = b * 32 + t;
    const double vd = a.D[o] * wpr * wpc;
    a.Ds[o] = vd;
    a.Df[o] = (float)vd;
}

// Inverse of each scaled 3x3 diagonal block of A, stored [9][N].
__global__ void k_jacobi(ScaleArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int64_t q = a.diag_slot[i], b = q >> 5, t = q & 31;
    double m[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) m[r][s] = a.As[(b * 9 + 3 * r + s) * 32 + t];
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
        atomicOr(a.err, ERR_SINGULAR);
        return;
    }
    const double id = 1.0 / det;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) {
            const double v = inv[r][s] * id;
            a.jac64[(3 * r + s) * a.N + i] = v;
            a.jac32[(3 * r + s) * a.N + i] = (float)v;
        }
    // reciprocals of the scalar diagonal, for diag(S^) (k_schur_hat)
#pragma unroll
    for (int s = 0; s < 3; s++) a.rdiag64[3 * i + s] = 1.0 / m[s][s];
}

// A~ = A M^-1 block by block: A~_(r,c) = A_(r,c) M_c^-1, M_c^-1 the inverse of
// the scaled diagonal block of node c (right block-Jacobi preconditioning
// folded into the operator of the A-solves)
__global__ void k_fold_jacobi(ScaleArgs a) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.nslots) return;
    const int64_t b = q >> 5;
    const int t = (int)(q & 31);
    const int s = a.col_slice[b];
    const int64_t r = (int64_t)s * 32 + t;
    double v[9];
#pragma unroll
    for (int k = 0; k < 9; k++) v[k] = 0.0;
    if (r < a.N && b - a.slice_ptr[s] < a.row_len[r]) {
        const int64_t c = a.col[q];
        double m[3][3], ji[3][3];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                m[i][j] = a.As[(b * 9 + 3 * i + j) * 32 + t];
                ji[i][j] = a.jac64[(3 * i + j) * a.N + c];
            }
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) v[3 * i + j] = m[i][0] * ji[0][j] + m[i][1] * ji[1][j] + m[i][2] * ji[2][j];
    }
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int64_t o = (b * 9 + k) * 32 + t;
        a.Ams[o] = v[k];
        a.Amf[o] = (float)v[k];
    }
    quant_block(v, q, a.Amh8, a.Amh1, a.Amhs);
}

// diag(S^)_i = D_ii - sum_c sum_s C_(i,c)[s] B_(c,i)[s] / A_(c,c)[s][s]  (scaled system);
// the reciprocals 1 / A_(c,c)[s][s] come from k_jacobi (one division per
// node component instead of one per block entry)
__global__ void k_schur_hat(ScaleArgs a) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    const int t = (int)(i & 31);
    const int64_t b0 = a.slice_ptr[i >> 5];
    const int len = a.row_len[i];
    double acc = 0.0;
    for (int j = 0; j < len; j++) {
        const int64_t b = b0 + j, q = b * 32 + t;
        const int64_t c = a.col[q];
        const int64_t mq = a.mirror[q], mb = mq >> 5, mt = mq & 31;
#pragma unroll
        for (int s = 0; s < 3; s++)
            acc += a.Cs[(b * 3 + s) * 32 + t] * a.Bs[(mb * 3 + s) * 32 + mt] * a.rdiag64[3 * c + s];
    }
    const int64_t dq = a.diag_slot[i], db = dq >> 5, dt = dq & 31;
    const double sh = a.Ds[db * 32 + dt] - acc;
    const double inv = fabs(sh) > 1e-300 ? 1.0 / sh : 1.0;
    a.shat64[i] = inv;
    a.shat32[i] = (float)inv;
}

// Transposed operator in the same pattern (the pattern is symmetric): block
// (i, c) of [[A^T, C^T], [B^T, D^T]] takes A(c, i)^T, C(c, i), B(c, i) and
// D(c, i) from the mirror slot of (i, c).
__global__ void k_transpose(const int32_t *__restrict__ col_slice, const int32_t *__restrict__ slice_ptr,
                            const int32_t *__restrict__ row_len, const int32_t *__restrict__ mirror,
                            const double *__restrict__ A, const double *__restrict__ B,
                            const double *__restrict__ C, const double *__restrict__ D, double *__restrict__ At,
                            double *__restrict__ Bt, double *__restrict__ Ct, double *__restrict__ Dt, int64_t N,
                            int64_t nslots) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nslots) return;
    const int64_t b = q >> 5;
    const int t = (int)(q & 31);
    const int s = col_slice[b];
    const int64_t r = (int64_t)s * 32 + t;
    if (r >= N || b - slice_ptr[s] >= row_len[r]) return;  // padding stays zero
    const int64_t mq = mirror[q], mb = mq >> 5, mt = mq & 31;
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) At[(b * 9 + 3 * i + j) * 32 + t] = A[(mb * 9 + 3 * j + i) * 32 + mt];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        Bt[(b * 3 + i) * 32 + t] = C[(mb * 3 + i) * 32 + mt];
        Ct[(b * 3 + i) * 32 + t] = B[(mb * 3 + i) * 32 + mt];
    }
    Dt[b * 32 + t] = D[mb * 32 + mt];
}

// A-block SpMVs, L lanes per block row: a warp covers 32 / L consecutive
// rows of one 32-row slice, and lane k of a row takes the row's blocks
// j = k, k + L, k + 2L, ...; the L partial sums meet by shuffles. For a given
// j the L lanes of a component read L runs of 32 / L consecutive slots, whole
// 32-byte sectors; in FP32 twice the warps of one thread per row keep more
// loads in flight (a 117,649-node matrix has only 3,677 slices).
template <int L, typename T>
__device__ __forceinline__ void lanes_reduce3(T &a0, T &a1, T &a2) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
}

template <typename T, int L>
__global__ void __launch_bounds__(128) k_spmv_A(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                                                const int32_t *__restrict__ col, const T *__restrict__ A,
                                                const T *__restrict__ x, T *__restrict__ y, int64_t N,
                                                const int *kd, int64_t ystride) {
    // kd = (k, done) of a Krylov level: output column k+1 of a basis with
    // column stride ystride; nothing to do once the level is done
    if (kd) {
        if (kd[1]) return;
        y += (int64_t)(kd[0] + 1) * ystride;
    }
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = g / L;
    const int k = (int)(g % L);
    // rows past N (the last slice may be short) stay for the shuffles with no blocks
    const bool live = r < N;
    const int t = (int)(r & 31);
    const int64_t b0 = live ? slice_ptr[r >> 5] : 0;
    const int len = live ? row_len[r] : 0;
    T a0 = 0, a1 = 0, a2 = 0;
#pragma unroll 2
    for (int j = k; j < len; j += L) {
        const int64_t b = b0 + j;
        const int64_t c = __ldg(col + b * 32 + t);
        const T *Ab = A + b * 288 + t;
        const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
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
    lanes_reduce3<L>(a0, a1, a2);
    if (live && k == 0) {
        y[3 * r] = a0;
        y[3 * r + 1] = a1;
        y[3 * r + 2] = a2;
    }
}

// A-SpMV on the BF16-with-block-scale copy, FP32 accumulation: per block,
// t_i = sum_j e_ij x_j, y_i += s t_i. Entry 2k of a block sits in the low half
// of word k of its 16-byte record, entry 2k+1 in the high half; a BF16 value
// widens to FP32 by a 16-bit shift. L lanes per row as above.
template <int L>
__global__ void __launch_bounds__(128) k_spmv_A16(const int32_t *__restrict__ slice_ptr,
                                                  const int32_t *__restrict__ row_len, const int32_t *__restrict__ col,
                                                  const uint4 *__restrict__ Ah8, const uint16_t *__restrict__ Ah1,
                                                  const float *__restrict__ Ahs, const float *__restrict__ x,
                                                  float *__restrict__ y, int64_t N, const int *kd, int64_t ystride) {
    if (kd) {
        if (kd[1]) return;
        y += (int64_t)(kd[0] + 1) * ystride;
    }
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = g / L;
    const int k = (int)(g % L);
    const bool live = r < N;
    const int t = (int)(r & 31);
    const int64_t b0 = live ? slice_ptr[r >> 5] : 0;
    const int len = live ? row_len[r] : 0;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll 2
    for (int j = k; j < len; j += L) {
        const int64_t q = (b0 + j) * 32 + t;
        const int64_t c = __ldg(col + q);
        const uint4 w = __ldg(Ah8 + q);
        const unsigned e8 = __ldg(Ah1 + q);
        const float s = __ldg(Ahs + q);
        const float x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
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
    }
    lanes_reduce3<L>(a0, a1, a2);
    if (live && k == 0) {
        y[3 * r] = a0;
        y[3 * r + 1] = a1;
        y[3 * r + 2] = a2;
    }
}

__global__ void __launch_bounds__(128) k_spmv_full64(const int32_t *__restrict__ slice_ptr,
                                                     const int32_t *__restrict__ row_len,
                                                     const int32_t *__restrict__ col, const double *__restrict__ A,
                                                     const double *__restrict__ B, const double *__restrict__ C,
                                                     const double *__restrict__ D, const double *__restrict__ x,
                                                     double *__restrict__ y, int64_t N, const int *kd,
                                                     int64_t stride) {
    // kd = (k, done): input column k, output column k+1 (FGMRES Z_k -> V_{k+1})
    if (kd) {
        if (kd[1]) return;
        x += (int64_t)kd[0] * stride;
        y += (int64_t)(kd[0] + 1) * stride;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int t = (int)(r & 31);
    const int64_t b0 = slice_ptr[r >> 5];
    const int len = row_len[r];
    const double *xp = x + 3 * N;
    double a0 = 0, a1 = 0, a2 = 0, ap = 0;
#pragma unroll 2
    for (int j = 0; j < len; j++) {
        const int64_t b = b0 + j;
        const int64_t c = __ldg(col + b * 32 + t);
        const double *Ab = A + b * 288 + t;
        const double *Bb = B + b * 96 + t;
        const double *Cb = C + b * 96 + t;
        const double x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2), xq = __ldg(xp + c);
        a0 = fma(__ldg(Ab + 0), x0, a0);
        a0 = fma(__ldg(Ab + 32), x1, a0);
        a0 = fma(__ldg(Ab + 64), x2, a0);
        a0 = fma(__ldg(Bb + 0), xq, a0);
        a1 = fma(__ldg(Ab + 96), x0, a1);
        a1 = fma(__ldg(Ab + 128), x1, a1);
        a1 = fma(__ldg(Ab + 160), x2, a1);
        a1 = fma(__ldg(Bb + 32), xq, a1);
        a2 = fma(__ldg(Ab + 192), x0, a2);
        a2 = fma(__ldg(Ab + 224), x1, a2);
        a2 = fma(__ldg(Ab + 256), x2, a2);
        a2 = fma(__ldg(Bb + 64), xq, a2);
        ap = fma(__ldg(Cb + 0), x0, ap);
        ap = fma(__ldg(Cb + 32), x1, ap);
        ap = fma(__ldg(Cb + 64), x2, ap);
        ap = fma(__ldg(D + b * 32 + t), xq, ap);
    }
    y[3 * r] = a0;
    y[3 * r + 1] = a1;
    y[3 * r + 2] = a2;
    y[3 * N + r] = ap;
}

// yv = r - B xp   (r == nullptr: yv = B xp)
template <typename T>
__global__ void k_spmv_B(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                         const int32_t *__restrict__ col, const T *__restrict__ B, const T *__restrict__ xp,
                         T *__restrict__ yv, const T *__restrict__ rin, int64_t N, const int *done) {
    if (done && *done) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int t = (int)(r & 31);
    const int64_t b0 = slice_ptr[r >> 5];
    const int len = row_len[r];
    T a0 = 0, a1 = 0, a2 = 0;
    for (int j = 0; j < len; j++) {
        const int64_t b = b0 + j;
        const int64_t c = __ldg(col + b * 32 + t);
        const T xq = __ldg(xp + c);
        const T *Bb = B + b * 96 + t;
        a0 = fma(__ldg(Bb), xq, a0);
        a1 = fma(__ldg(Bb + 32), xq, a1);
        a2 = fma(__ldg(Bb + 64), xq, a2);
    }
    if (rin) {
        yv[3 * r] = rin[3 * r] - a0;
        yv[3 * r + 1] = rin[3 * r + 1] - a1;
        yv[3 * r + 2] = rin[3 * r + 2] - a2;
    } else {
        yv[3 * r] = a0;
        yv[3 * r + 1] = a1;
        yv[3 * r + 2] = a2;
    }
}

// yp = r - C xv   (r == nullptr: yp = C xv)
template <typename T>
__global__ void k_spmv_C(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                         const int32_t *__restrict__ col, const T *__restrict__ C, const T *__restrict__ xv,
                         T *__restrict__ yp, const T *__restrict__ rin, int64_t N, const int *done) {
    if (done && *done) return;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int t = (int)(r & 31);
    const int64_t b0 = slice_ptr[r >> 5];
    const int len = row_len[r];
    T a = 0;
    for (int j = 0; j < len; j++) {
        const int64_t b = b0 + j;
        const int64_t c = __ldg(col + b * 32 + t);
        const T *Cb = C + b * 96 + t;
        a = fma(__ldg(Cb), __ldg(xv + 3 * c), a);
        a = fma(__ldg(Cb + 32), __ldg(xv + 3 * c + 1), a);
        a = fma(__ldg(Cb + 64), __ldg(xv + 3 * c + 2), a);
    }
    yp[r] = rin ? rin[r] - a : a;
}

// yp = D xp - C xv  (xv == nullptr: yp = D xp)
template <typename T>
__global__ void k_spmv_DC(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                          const int32_t *__restrict__ col, const T *__restrict__ D, const T *__restrict__ C,
                          const T *__restrict__ xp, const T *__restrict__ xv, T *__restrict__ yp, int64_t N,
                          const int *kd, int64_t ystride) {
    if (kd) {  // output column k+1 of a Krylov basis (see k_spmv_A)
        if (kd[1]) return;
        yp += (int64_t)(kd[0] + 1) * ystride;
    }
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int t = (int)(r & 31);
    const int64_t b0 = slice_ptr[r >> 5];
    const int len = row_len[r];
    T a = 0, m = 0;
    for (int j = 0; j < len; j++) {
        const int64_t b = b0 + j;
        const int64_t c = __ldg(col + b * 32 + t);
        a = fma(__ldg(D + b * 32 + t), __ldg(xp + c), a);
        if (xv) {
            const T *Cb = C + b * 96 + t;
            m = fma(__ldg(Cb), __ldg(xv + 3 * c), m);
            m = fma(__ldg(Cb + 32), __ldg(xv + 3 * c + 1), m);
            m = fma(__ldg(Cb + 64), __ldg(xv + 3 * c + 2), m);
        }
    }
    yp[r] = a - m;
}

ScaleArgs scale_args(Ctx &c) {
    ScaleArgs a;
    DeviceMesh &m = c.mesh;
    DeviceMatrix &M = c.mat;
    a.diag_slot = m.diag_slot;
    a.col_slice = m.col_slice;
    a.slice_ptr = m.slice_ptr;
    a.row_len = m.row_len;
    a.col = m.col;
    a.mirror = m.mirror;
    a.A = M.A;
    a.B = M.B;
    a.C = M.C;
    a.D = M.D;
    a.As = M.As;
    a.Bs = M.Bs;
    a.Cs = M.Cs;
    a.Ds = M.Ds;
    a.Af = M.Af;
    a.Bf = M.Bf;
    a.Cf = M.Cf;
    a.Df = M.Df;
    a.Ah8 = M.Ah8;
    a.Ah1 = M.Ah1;
    a.Ahs = M.Ahs;
    a.Ams = M.Ams;
    a.Amf = M.Amf;
    a.Amh8 = M.Amh8;
    a.Amh1 = M.Amh1;
    a.Amhs = M.Amhs;
    a.w = M.w;
    a.jac64 = M.jac64;
    a.rdiag64 = M.rdiag64;
    a.jac32 = M.jac32;
    a.shat64 = M.shat64;
    a.shat32 = M.shat32;
    a.err = c.err;
    a.N = m.N;
    a.nslots = m.nslots;
    return a;
}

}  // namespace

void solve_setup(Ctx &c) {
    if (!c.mat.assembled) fail(HYEL_ESTATE, "solve_setup: nothing assembled");
    if (c.mat.scaled) return;
    ScaleArgs a = scale_args(c);
    const int64_t N = c.mesh.N;
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    (k_scale_diag<<<blocks_for(N, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
    (k_scale_values<<<blocks_for(c.mesh.nslots, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
    (k_jacobi<<<blocks_for(N, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
    (k_fold_jacobi<<<blocks_for(c.mesh.nslots, 256), 256, 0, c.stream>>>(a), ::hyel::count_launch());
    (k_schur_hat<<<blocks_for(N, 128), 128, 0, c.stream>>>(a), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & ERR_SINGULAR) fail(HYEL_ESINGULAR, "solve_setup: a 3x3 diagonal block of A is singular");
    c.mat.scaled = true;
    c.mat.amg_ready = false;
    c.mat.shat_ready = false;
    c.mat.shat64_ready = false;
    c.mat.asym_ready = false;
    c.mat.acheb_ready = false;
}

namespace {

// A_sym = (A + A^T)/2 block by block: block (i, c) is (A_(i,c) + A_(c,i)^T)/2,
// A_(c,i) at the mirror slot; padding slots get 0
__global__ void k_symmetrize(const int32_t *__restrict__ mirror, const double *__restrict__ As,
                             double *__restrict__ S64, float *__restrict__ S32, int64_t nslots) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nslots) return;
    const int64_t b = q >> 5, t = q & 31, mq = mirror[q];
    const int64_t mb = mq >> 5, mt = mq & 31;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) {
            const double v = mq < 0 ? 0.0 : 0.5 * (As[(b * 9 + 3 * r + s) * 32 + t] + As[(mb * 9 + 3 * s + r) * 32 + mt]);
            S64[(b * 9 + 3 * r + s) * 32 + t] = v;
            S32[(b * 9 + 3 * r + s) * 32 + t] = (float)v;
        }
}

// inverses of the 3x3 diagonal blocks of Av (adjugate over determinant)
__global__ void k_block_inv3(const int32_t *__restrict__ diag_slot, const double *__restrict__ Av, double *j64,
                             float *j32, int64_t N, unsigned *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t q = diag_slot[i], b = q >> 5, t = q & 31;
    double m[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int s = 0; s < 3; s++) m[r][s] = Av[(b * 9 + 3 * r + s) * 32 + t];
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
            const double v = inv[r][s] * id;
            j64[(3 * r + s) * N + i] = v;
            j32[(3 * r + s) * N + i] = (float)v;
        }
}

}  // namespace

void asym_setup(Ctx &c) {
    solve_setup(c);
    if (c.mat.asym_ready) return;
    const DeviceMesh &m = c.mesh;
    DeviceMatrix &M = c.mat;
    if (!M.Asym64) {
        M.Asym64 = dalloc_n<double>(c, 9 * (size_t)m.nslots);
        M.Asym32 = dalloc_n<float>(c, 9 * (size_t)m.nslots);
        M.jsym64 = dalloc_n<double>(c, 9 * (size_t)m.N);
        M.jsym32 = dalloc_n<float>(c, 9 * (size_t)m.N);
    }
    HYEL_CK(cudaMemsetAsync(c.err, 0, sizeof(unsigned), c.stream));
    (k_symmetrize<<<blocks_for(m.nslots, 256), 256, 0, c.stream>>>(m.mirror, M.As, M.Asym64, M.Asym32, m.nslots),
     ::hyel::count_launch());
    (k_block_inv3<<<blocks_for(m.N, 256), 256, 0, c.stream>>>(m.diag_slot, M.Asym64, M.jsym64, M.jsym32, m.N, c.err),
     ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    HYEL_CK(cudaMemcpyAsync(c.h_err, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    HYEL_CK(cudaStreamSynchronize(c.stream));
    if (*c.h_err & ERR_SINGULAR) fail(HYEL_ESINGULAR, "asym_setup: a 3x3 diagonal block of (A + A^T)/2 is singular");
    M.asym_ready = true;
}

void transpose_assembled(Ctx &c) {
    if (!c.mat.assembled) fail(HYEL_ESTATE, "transpose: nothing assembled");
    if (c.mat.transposed) return;
    const DeviceMesh &m = c.mesh;
    DeviceMatrix &M = c.mat;
    (k_transpose<<<blocks_for(m.nslots, 256), 256, 0, c.stream>>>(m.col_slice, m.slice_ptr, m.row_len, m.mirror, M.A,
                                                                  M.B, M.C, M.D, M.At, M.Bt, M.Ct, M.Dt, m.N,
                                                                  m.nslots),
     ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    M.transposed = true;
}

template <typename T>
void spmv_A_ind(Ctx &c, const T *Av, const T *x, T *y, int64_t ystride, const int *kd) {
    const DeviceMesh &m = c.mesh;
    const int cls = sizeof(T) == 8 ? HYEL_K_SPMV_A64 : HYEL_K_SPMV_A32;
    cudaEvent_t ev;
    prof_begin(c, cls, &ev);
    // FP64: one thread per row in one-warp blocks (the FP64 pipe, not the
    // load rate, limits it; single-slice blocks spread the rows evenly over
    // the SMs); FP32: two lanes per row in 128-thread blocks. Both were the
    // fastest of a sweep over 1-8 lanes per row and 32-256 threads per block
    // on the 48^3 cube's pattern.
    if constexpr (sizeof(T) == 8)
        (k_spmv_A<T, 1><<<blocks_for(m.N, 32), 32, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, Av, x, y, m.N, kd,
                                                                   ystride), ::hyel::count_launch());
    else
        (k_spmv_A<T, 2><<<blocks_for(2 * m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, Av, x, y, m.N,
                                                                         kd, ystride), ::hyel::count_launch());
    // algorithmic bytes: 9 values + 1 column index per block, x and y once
    prof_end(c, cls, ev, (double)m.nnzb * (9.0 * sizeof(T) + 4.0) + 4.0 * (m.N + 1) + 2.0 * 3 * m.N * sizeof(T));
}
template <typename T>
void spmv_A(Ctx &c, const T *Av, const T *x, T *y) {
    spmv_A_ind<T>(c, Av, x, y, 0, nullptr);
}
template void spmv_A<double>(Ctx &, const double *, const double *, double *);
template void spmv_A<float>(Ctx &, const float *, const float *, float *);
template void spmv_A_ind<double>(Ctx &, const double *, const double *, double *, int64_t, const int *);
template void spmv_A_ind<float>(Ctx &, const float *, const float *, float *, int64_t, const int *);

void spmv_A16_ind(Ctx &c, const uint4 *h8, const uint16_t *h1, const float *hs, const float *x, float *y,
                  int64_t ystride, const int *kd) {
    const DeviceMesh &m = c.mesh;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_SPMV_A16, &ev);
    (k_spmv_A16<2><<<blocks_for(2 * m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, h8, h1, hs, x, y,
                                                                     m.N, kd, ystride), ::hyel::count_launch());
    // algorithmic bytes: 9 BF16 values + 1 FP32 scale + 1 column index per block, x and y once
    prof_end(c, HYEL_K_SPMV_A16, ev, (double)m.nnzb * (18.0 + 4.0 + 4.0) + 4.0 * (m.N + 1) + 2.0 * 3 * m.N * 4);
}

void spmv_full64_ind(Ctx &c, const double *A, const double *B, const double *C, const double *D, const double *x,
                     double *y, int64_t stride, const int *kd) {
    const DeviceMesh &m = c.mesh;
    cudaEvent_t ev;
    prof_begin(c, HYEL_K_SPMV_FULL64, &ev);
    (k_spmv_full64<<<blocks_for(m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, A, B, C, D, x, y, m.N,
                                                              kd, stride), ::hyel::count_launch());
    prof_end(c, HYEL_K_SPMV_FULL64, ev, (double)m.nnzb * (16.0 * 8 + 4.0) + 4.0 * (m.N + 1) + 2.0 * 4 * m.N * 8);
}
void spmv_full64(Ctx &c, const double *A, const double *B, const double *C, const double *D, const double *x,
                 double *y) {
    spmv_full64_ind(c, A, B, C, D, x, y, 0, nullptr);
}

template <typename T>
void spmv_B(Ctx &c, const T *B, const T *xp, T *yv, const T *r) {
    const DeviceMesh &m = c.mesh;
    (k_spmv_B<T><<<blocks_for(m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, B, xp, yv, r, m.N,
                                                            nullptr), ::hyel::count_launch());
}
template <typename T>
void spmv_C(Ctx &c, const T *C, const T *xv, T *yp, const T *r) {
    const DeviceMesh &m = c.mesh;
    (k_spmv_C<T><<<blocks_for(m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, C, xv, yp, r, m.N,
                                                            nullptr), ::hyel::count_launch());
}
template <typename T>
void spmv_D(Ctx &c, const T *D, const T *xp, T *yp) {
    const DeviceMesh &m = c.mesh;
    (k_spmv_DC<T><<<blocks_for(m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, D, (const T *)nullptr, xp,
                                                             (const T *)nullptr, yp, m.N, nullptr, 0),
     ::hyel::count_launch());
}
template <typename T>
void spmv_DC_ind(Ctx &c, const T *D, const T *C, const T *xp, const T *xv, T *yp, int64_t ystride, const int *kd) {
    const DeviceMesh &m = c.mesh;
    (k_spmv_DC<T><<<blocks_for(m.N, 128), 128, 0, c.stream>>>(m.slice_ptr, m.row_len, m.col, D, C, xp, xv, yp, m.N, kd,
                                                             ystride), ::hyel::count_launch());
}
#define HYEL_INST(T)                                                                              \
    template void spmv_B<T>(Ctx &, const T *, const T *, T *, const T *);                         \
    template void spmv_C<T>(Ctx &, const T *, const T *, T *, const T *);                         \
    template void spmv_D<T>(Ctx &, const T *, const T *, T *);                                    \
    template void spmv_DC_ind<T>(Ctx &, const T *, const T *, const T *, const T *, T *, int64_t, const int *);
HYEL_INST(double)
HYEL_INST(float)
#undef HYEL_INST

}  // namespace hyel
