// Explicit sparse S^ = D - C diag(A)^-1 B of the scaled system (§4.2: the
// approximation of the Schur complement from which the paper builds the
// preconditioner of the S-solve), diag(A) the scalar diagonal of A.
//
// * Pattern, once per mesh, on the host: row i of S^ couples node i with every
//   node j two block-graph steps away (i - k - j through a shared neighbour k,
//   which includes k = i and k = j, so D's pattern is inside). Stored SELL-32
//   like the block pattern, columns ascending. For every contribution to row
//   i, in the order the numeric kernel visits them, the index of its entry in
//   the row is recorded (a uint16 position list), so no search runs on the GPU.
// * Values, after every scaling of a new assembly, on the GPU: one thread per
//   row sums D_ik and -sum_s C_ik[s] B_kj[s] / A_kk[s][s] into a per-thread
//   row buffer in shared memory (column-major over the block's threads, so
//   every lane stays in its own bank), in a fixed order (bitwise
//   reproducible), then writes the row out coalesced. The solver's copy is
//   summed in FP32 from the FP32 scaled blocks (the preconditioner's
//   precision; FP64 arithmetic is scarce on this GPU); the FP64 copy is
//   summed from the FP64 blocks when an FP64 entry point first asks for it.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace hyel {

namespace {

constexpr int kShatSmemMax = 200 * 1024;  // dynamic shared memory of the numeric kernel

template <typename T>
T *upload_sync(Ctx &c, const std::vector<T> &h) {
    if (h.empty()) return nullptr;
    T *d = dalloc_n<T>(c, h.size());
    HYEL_CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return d;
}

template <typename V>
struct NumArgs {
    // block pattern and scaled blocks of precision V
    const int32_t *slice_ptr, *row_len, *col, *diag_slot;
    const V *As, *Bs, *Cs, *Ds;
    // S^
    const int32_t *h_slice_ptr, *h_row_len;
    const int64_t *cptr;
    const uint16_t *pos;
    V *val;
    int64_t N;
    int tb;  // threads per block (row stride of the shared buffer)
};

template <typename V>
__global__ void k_shat_numeric(NumArgs<V> a) {
    extern __shared__ unsigned char s_raw[];
    V *s_row = reinterpret_cast<V *>(s_raw);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    V *acc = s_row + threadIdx.x;
    const int tb = a.tb;
    const int lh = a.h_row_len[i];
    for (int p = 0; p < lh; p++) acc[p * tb] = 0;
    const int t = (int)(i & 31);
    const int64_t b0 = a.slice_ptr[i >> 5];
    const int len = a.row_len[i];
    const uint16_t *pos = a.pos + a.cptr[i];
    int cp = 0;
    for (int kk = 0; kk < len; kk++) {
        const int64_t b = b0 + kk, q = b * 32 + t;
        const int64_t k = a.col[q];
        acc[pos[cp++] * tb] += a.Ds[q];
        const int64_t dq = a.diag_slot[k], db = dq >> 5, dt = dq & 31;
        const V c0 = a.Cs[(b * 3) * 32 + t] / a.As[(db * 9) * 32 + dt];
        const V c1 = a.Cs[(b * 3 + 1) * 32 + t] / a.As[(db * 9 + 4) * 32 + dt];
        const V c2 = a.Cs[(b * 3 + 2) * 32 + t] / a.As[(db * 9 + 8) * 32 + dt];
        const int64_t kb0 = a.slice_ptr[k >> 5];
        const int tk = (int)(k & 31);
        const int lk = a.row_len[k];
        for (int jj = 0; jj < lk; jj++) {
            const V *Bb = a.Bs + ((kb0 + jj) * 3) * 32 + tk;
            const V v = c0 * Bb[0] + c1 * Bb[32] + c2 * Bb[64];
            acc[pos[cp++] * tb] -= v;
        }
    }
    const int64_t hb0 = a.h_slice_ptr[i >> 5];
    const int w = a.h_slice_ptr[(i >> 5) + 1] - (int)hb0;
    for (int p = 0; p < w; p++) a.val[(hb0 + p) * 32 + t] = p < lh ? acc[p * tb] : (V)0;
}

template <typename T>
__global__ void k_shat_spmv(const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len,
                            const int32_t *__restrict__ col, const T *__restrict__ val, const T *__restrict__ x,
                            T *__restrict__ y, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int t = (int)(i & 31);
    const int64_t b0 = slice_ptr[i >> 5];
    const int len = row_len[i];
    T s = 0;
    for (int p = 0; p < len; p++) {
        const int64_t q = (b0 + p) * 32 + t;
        s = fma(val[q], x[col[q]], s);
    }
    y[i] = s;
}

void shat_build(Ctx &c) {
    const DeviceMesh &m = c.mesh;
    const int64_t N = m.N;
    const std::vector<int32_t> &rp = m.h_row_ptr, &cols = m.h_col;
    // distance-2 rows, ascending
    std::vector<int64_t> hrp(N + 1, 0);
    std::vector<int32_t> hcol;
    hcol.reserve((size_t)N * 64);
    std::vector<int64_t> mark(N, -1);
    std::vector<int32_t> cand;
    int64_t ncontrib = 0;
    for (int64_t i = 0; i < N; i++) {
        cand.clear();
        for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
            const int32_t k = cols[p];
            ncontrib += 1 + (rp[k + 1] - rp[k]);
            for (int32_t p2 = rp[k]; p2 < rp[k + 1]; p2++) {
                const int32_t j = cols[p2];
                if (mark[j] != i) {
                    mark[j] = i;
                    cand.push_back(j);
                }
            }
        }
        std::sort(cand.begin(), cand.end());
        hcol.insert(hcol.end(), cand.begin(), cand.end());
        hrp[i + 1] = (int64_t)hcol.size();
    }
    int32_t max_row = 0;
    for (int64_t i = 0; i < N; i++) max_row = std::max<int32_t>(max_row, (int32_t)(hrp[i + 1] - hrp[i]));
    if (max_row > 65535 || (int64_t)32 * max_row * 8 > kShatSmemMax)
        fail(HYEL_EINVAL, "schur_hat: a distance-2 row is too long");
    // SELL-32
    const int64_t ns = (N + 31) / 32;
    std::vector<int32_t> sp(ns + 1, 0), rl(N);
    for (int64_t s = 0; s < ns; s++) {
        int64_t w = 0;
        for (int t = 0; t < 32; t++) {
            const int64_t r = s * 32 + t;
            if (r < N) w = std::max<int64_t>(w, hrp[r + 1] - hrp[r]);
        }
        if ((int64_t)sp[s] + w >= ((int64_t)1 << 31) / 32) fail(HYEL_EINVAL, "schur_hat: pattern too large");
        sp[s + 1] = sp[s] + (int32_t)w;
    }
    const int64_t ncols = sp[ns], nslots = ncols * 32;
    std::vector<int32_t> scol(nslots);
    for (int64_t r = 0; r < N; r++) {
        rl[r] = (int32_t)(hrp[r + 1] - hrp[r]);
        const int32_t w = sp[(r >> 5) + 1] - sp[r >> 5];
        for (int32_t p = 0; p < w; p++)
            scol[((int64_t)sp[r >> 5] + p) * 32 + (r & 31)] = p < rl[r] ? hcol[hrp[r] + p] : (int32_t)r;
    }
    // contribution positions, in the numeric kernel's order
    std::vector<int64_t> cptr(N + 1, 0);
    std::vector<uint16_t> pos((size_t)ncontrib);
    std::vector<int32_t> where(N, -1);
    int64_t o = 0;
    for (int64_t i = 0; i < N; i++) {
        for (int64_t p = hrp[i]; p < hrp[i + 1]; p++) where[hcol[p]] = (int32_t)(p - hrp[i]);
        for (int32_t p = rp[i]; p < rp[i + 1]; p++) {
            const int32_t k = cols[p];
            pos[o++] = (uint16_t)where[k];
            for (int32_t p2 = rp[k]; p2 < rp[k + 1]; p2++) pos[o++] = (uint16_t)where[cols[p2]];
        }
        cptr[i + 1] = o;
    }
    SchurHat *h = new SchurHat();
    c.sh = h;
    h->nnz = (int64_t)hcol.size();
    h->ncols = ncols;
    h->nslots = nslots;
    h->ncontrib = ncontrib;
    h->max_row = max_row;
    h->slice_ptr = upload_sync(c, sp);
    h->row_len = upload_sync(c, rl);
    h->col = upload_sync(c, scol);
    h->cptr = upload_sync(c, cptr);
    h->pos = upload_sync(c, pos);
    h->v64 = dalloc_n<double>(c, (size_t)nslots);
    h->v32 = dalloc_n<float>(c, (size_t)nslots);
    h->bounds = dalloc_n<double>(c, 2);
    h->work = dalloc_n<double>(c, 3 * (size_t)N);
    h->bar = (unsigned *)dalloc(c, kBarAlloc * sizeof(unsigned));  // the grid barrier's four 128-byte lines
}

}  // namespace

void shat_free(Ctx &c) {
    delete c.sh;  // device arrays belong to the context's allocation list
    c.sh = nullptr;
}

template <typename V>
void shat_numeric(Ctx &c) {
    if (!c.mat.scaled) fail(HYEL_ESTATE, "schur_hat: the scaled system is not set up");
    if (!c.sh) shat_build(c);
    const SchurHat &h = *c.sh;
    const DeviceMesh &m = c.mesh;
    NumArgs<V> a;
    a.slice_ptr = m.slice_ptr;
    a.row_len = m.row_len;
    a.col = m.col;
    a.diag_slot = m.diag_slot;
    if constexpr (std::is_same<V, double>::value) {
        a.As = c.mat.As;
        a.Bs = c.mat.Bs;
        a.Cs = c.mat.Cs;
        a.Ds = c.mat.Ds;
        a.val = h.v64;
    } else {
        a.As = c.mat.Af;
        a.Bs = c.mat.Bf;
        a.Cs = c.mat.Cf;
        a.Ds = c.mat.Df;
        a.val = h.v32;
    }
    a.h_slice_ptr = h.slice_ptr;
    a.h_row_len = h.row_len;
    a.cptr = h.cptr;
    a.pos = h.pos;
    a.N = m.N;
    int tb = 128;
    while (tb > 32 && (int64_t)tb * h.max_row * (int64_t)sizeof(V) > kShatSmemMax) tb /= 2;
    a.tb = tb;
    const int smem = tb * h.max_row * (int)sizeof(V);
    HYEL_CK(cudaFuncSetAttribute(k_shat_numeric<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    (k_shat_numeric<V><<<blocks_for(m.N, tb), tb, smem, c.stream>>>(a), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
}
template void shat_numeric<double>(Ctx &);
template void shat_numeric<float>(Ctx &);

void shat_ensure64(Ctx &c) {
    if (!c.sh || !c.mat.shat_ready) fail(HYEL_ESTATE, "schur_hat: S^ is not built for the current assembly");
    if (!c.mat.shat64_ready) {
        shat_numeric<double>(c);
        c.mat.shat64_ready = true;
    }
}

template <typename T>
void shat_spmv(Ctx &c, const T *x, T *y) {
    if (!c.sh || !c.mat.shat_ready) fail(HYEL_ESTATE, "schur_hat: S^ is not built for the current assembly");
    if constexpr (std::is_same<T, double>::value) shat_ensure64(c);
    const SchurHat &h = *c.sh;
    const T *val;
    if constexpr (std::is_same<T, double>::value)
        val = h.v64;
    else
        val = h.v32;
    (k_shat_spmv<T><<<blocks_for(c.mesh.N, 128), 128, 0, c.stream>>>(h.slice_ptr, h.row_len, h.col, val, x, y,
                                                                      c.mesh.N),
     ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
}
template void shat_spmv<double>(Ctx &, const double *, double *);
template void shat_spmv<float>(Ctx &, const float *, float *);

}  // namespace hyel
