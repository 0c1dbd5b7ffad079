// hyel_residual_norm_static: the residual norms ||b - M x|| and ||b|| of the
// coupled operator M = [[A, B], [C, D]] without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// residual check: frameworks that hand all device memory to their own pool
// allocator and forbid direct cudaMalloc calls beside it, callers that run
// with a hard device-memory budget already spent, and latency-critical loops
// in which an allocation (and the device synchronization cudaFree implies)
// costs more than the check itself. For them this entry point keeps its
// reduction scratch (per-block partial sums and the completion counter) in a
// fixed, file-scope device array instead of the context's workspace; it calls
// no cudaMalloc, cudaFree or allocating routine.
//
// The array's device address is looked up once per device (at the first call
// with that device current) and cached for the life of the process. A
// cudaDeviceReset of that device, or any other teardown of its primary
// context, unloads the module and invalidates the cached address: do not call
// this entry point again in a process that has reset the device.
//
// The arithmetic is that of the solver's true-residual check: each block row
// is formed in the same order as the full-operator SpMV, squared and summed
// per block, and the last block to finish adds the block partials in a fixed
// order.
#include <mutex>

#include "internal.h"

namespace hyel {

namespace {

constexpr int kNsThreads = 128;
constexpr int kNsMaxBlocks = 8192;  // one block per 128 block rows: N <= 1,048,576 nodes

// [0, 2*kNsMaxBlocks): per-block partial sums (||r||^2, ||b||^2);
// [2*kNsMaxBlocks]: completion counter; the rest pads to 256-byte alignment.
static __device__ __align__(256) double g_ns_scratch[2 * kNsMaxBlocks + 32];

std::mutex g_ns_mutex;
double *g_ns_ptr[64] = {nullptr};  // device address of the array, per device

double *scratch_for_device(int dev) {
    if (dev < 0 || dev >= 64) fail(HYEL_EINVAL, "residual_norm_static: device index out of range");
    std::lock_guard<std::mutex> lock(g_ns_mutex);
    if (!g_ns_ptr[dev]) {
        void *p = nullptr;
        // host code must ask for the address: the symbol itself is a host-side stand-in
        check_cuda(cudaGetSymbolAddress(&p, g_ns_scratch), "cudaGetSymbolAddress(g_ns_scratch)");
        g_ns_ptr[dev] = static_cast<double *>(p);
    }
    return g_ns_ptr[dev];
}

__global__ void __launch_bounds__(kNsThreads) k_residual_norm_static(
    const int32_t *__restrict__ slice_ptr, const int32_t *__restrict__ row_len, const int32_t *__restrict__ col,
    const double *__restrict__ A, const double *__restrict__ B, const double *__restrict__ C,
    const double *__restrict__ D, const double *__restrict__ x, const double *__restrict__ b, int64_t N,
    double *scratch, double *out) {
    __shared__ double red[2][kNsThreads / 32];
    __shared__ bool last;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + 2 * kNsMaxBlocks);
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0, bb = 0.0;
    if (r < N) {
        const int t = (int)(r & 31);
        const int64_t b0 = slice_ptr[r >> 5];
        const int len = row_len[r];
        const double *xp = x + 3 * N;
        double a0 = 0, a1 = 0, a2 = 0, ap = 0;
        for (int j = 0; j < len; j++) {
            const int64_t bk = b0 + j;
            const int64_t c = col[bk * 32 + t];
            const double *Ab = A + bk * 288 + t;
            const double *Bb = B + bk * 96 + t;
            const double *Cb = C + bk * 96 + t;
            const double x0 = x[3 * c], x1 = x[3 * c + 1], x2 = x[3 * c + 2], xq = xp[c];
            a0 = fma(Ab[0], x0, a0);
            a0 = fma(Ab[32], x1, a0);
            a0 = fma(Ab[64], x2, a0);
            a0 = fma(Bb[0], xq, a0);
            a1 = fma(Ab[96], x0, a1);
            a1 = fma(Ab[128], x1, a1);
            a1 = fma(Ab[160], x2, a1);
            a1 = fma(Bb[32], xq, a1);
            a2 = fma(Ab[192], x0, a2);
            a2 = fma(Ab[224], x1, a2);
            a2 = fma(Ab[256], x2, a2);
            a2 = fma(Bb[64], xq, a2);
            ap = fma(Cb[0], x0, ap);
            ap = fma(Cb[32], x1, ap);
            ap = fma(Cb[64], x2, ap);
            ap = fma(D[bk * 32 + t], xq, ap);
        }
        const double bv[4] = {b[3 * r], b[3 * r + 1], b[3 * r + 2], b[3 * N + r]};
        const double e[4] = {bv[0] - a0, bv[1] - a1, bv[2] - a2, bv[3] - ap};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            rr = fma(e[k], e[k], rr);
            bb = fma(bv[k], bv[k], bb);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rr += __shfl_down_sync(0xffffffffu, rr, o);
        bb += __shfl_down_sync(0xffffffffu, bb, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = rr;
        red[1][threadIdx.x >> 5] = bb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int q = 0; q < kNsThreads / 32; q++) s += red[threadIdx.x][q];
        scratch[2 * blockIdx.x + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (w < 2) {  // warp w sums quantity w over the blocks, lanes striding, fixed order
        double s = 0.0;
        for (unsigned k = l; k < gridDim.x; k += 32) s += ((volatile double *)scratch)[2 * k + w];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (l == 0) out[w] = sqrt(s);
    }
    if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace

void residual_norm_static(Ctx &c, int matrix, const double *x, const double *b, double *out) {
    if (!x || !b || !out) fail(HYEL_EINVAL, "residual_norm_static: null pointer");
    if (matrix != HYEL_MAT_ASSEMBLED && matrix != HYEL_MAT_SCALED64)
        fail(HYEL_EINVAL, "residual_norm_static: matrix must be HYEL_MAT_ASSEMBLED or HYEL_MAT_SCALED64");
    if (!c.mat.assembled) fail(HYEL_ESTATE, "residual_norm_static: nothing assembled");
    if (matrix == HYEL_MAT_SCALED64 && !c.mat.scaled) fail(HYEL_ESTATE, "residual_norm_static: call hyel_solve_setup first");
    const DeviceMesh &m = c.mesh;
    if (m.N <= 0) fail(HYEL_ESTATE, "residual_norm_static: no mesh uploaded");
    const int64_t blocks = (m.N + kNsThreads - 1) / kNsThreads;
    if (blocks > kNsMaxBlocks)
        fail(HYEL_EINVAL, "residual_norm_static: mesh has " + std::to_string(m.N) +
                              " nodes; the fixed scratch supports at most " +
                              std::to_string((int64_t)kNsMaxBlocks * kNsThreads));
    double *scratch = scratch_for_device(c.device);
    // the completion counter must start at zero on every call
    check_cuda(cudaMemsetAsync(scratch + 2 * kNsMaxBlocks, 0, sizeof(unsigned), c.stream), "cudaMemsetAsync");
    const bool s = matrix == HYEL_MAT_SCALED64;
    const DeviceMatrix &M = c.mat;
    (k_residual_norm_static<<<(int)blocks, kNsThreads, 0, c.stream>>>(
         m.slice_ptr, m.row_len, m.col, s ? M.As : M.A, s ? M.Bs : M.B, s ? M.Cs : M.C, s ? M.Ds : M.D, x, b, m.N,
         scratch, out),
     ::hyel::count_launch());
    check_cuda(cudaGetLastError(), "k_residual_norm_static");
}

}  // namespace hyel
