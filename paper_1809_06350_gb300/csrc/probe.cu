// hyel_fp64_fma_probe: a compute-only kernel that measures the FP64 FMA rate
// of the device it runs on, the denominator of the element kernel's roofline
// (that kernel is bound by FP64 arithmetic, not by memory).
//
// Every thread runs kChains independent dependent-FMA chains x <- x * a + b
// for `iters` rounds (kChains FMAs in flight per thread hide the FMA latency),
// on a grid of 8 blocks of 256 threads per SM. Nothing is read from memory
// inside the loop; one value per thread is folded and written at the end so
// that the chains are not optimized away. The caller times the launch (CUDA
// events on the context's stream) and divides the flop count this entry
// point returns by that time. It changes no device setting.
#include "internal.h"

namespace hyel {

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;
constexpr int kChains = 8;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_fma_probe(int64_t iters, double a, double b, double *sink) {
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int64_t it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    // a and b keep |x| bounded (|a| < 1); the store is taken only by a value
    // the chains cannot reach, so the kernel writes nothing in practice
    if (s == 12345.678) sink[0] = s;
}

}  // namespace

double fp64_fma_probe(Ctx &c, int64_t iters, double *sink) {
    if (iters < 1 || iters > (int64_t)1 << 24) fail(HYEL_EINVAL, "fp64_fma_probe: iters must be in [1, 2^24]");
    if (!sink) fail(HYEL_EINVAL, "fp64_fma_probe: null sink");
    const int grid = kProbeBlocksPerSm * c.num_sms;
    (k_fp64_fma_probe<<<grid, kProbeThreads, 0, c.stream>>>(iters, 0.999999, 1e-7, sink), ::hyel::count_launch());
    HYEL_CK(cudaGetLastError());
    return 2.0 * (double)iters * kChains * (double)kProbeThreads * grid;
}

}  // namespace hyel
