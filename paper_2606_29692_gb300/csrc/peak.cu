// The float64 FMA rate of the device: the roofline of the kernels that the
// float64 pipe bounds.
//
// On this part the float64 pipe issues at a small fraction of the float32
// rate, and the complex128 Taylor-5 updates (closed form c5 psi + s5 A psi
// and the norm's |psi|^2, 12 float64 operations per support pair) are
// limited by it rather than by HBM.  Neither measured peak beside the
// kernels (a copy's HBM rate, a bf16 GEMM's tensor rate) bounds them, so
// this kernel measures the float64 rate itself.  Every thread runs eight
// independent chains of dependent fused multiply-adds a <- a m + c, with m
// and c passed at launch so that nothing folds at compile time.  With
// 0 < m < 1 and c > 0 each chain moves towards c / (1 - m) and stays in
// the normal range, so no denormal slows it.  Eight chains per thread and
// a full SM of threads keep enough independent operations in flight to
// cover the pipe's latency.  The rate is counted in float64 lane
// operations per second: one FMA (two flops) on one lane each.
#include "api_internal.h"

namespace tq {
namespace {

constexpr int FR_BS = 256;
constexpr int FR_BLOCKS_PER_SM = 8;
constexpr int FR_CHAINS = 8;

__global__ void __launch_bounds__(FR_BS) k_fp64_fma_rate(double m, double c, int iters, double* sink) {
    double a[FR_CHAINS];
#pragma unroll
    for (int j = 0; j < FR_CHAINS; ++j) a[j] = (double)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < FR_CHAINS; ++j) a[j] = fma(a[j], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < FR_CHAINS; ++j) s += a[j];
    if (s < 0.0) *sink = s;   // never taken (every chain stays positive); keeps the chains live
}

}  // namespace
}  // namespace tq

using namespace tq;
using namespace tq::api;

extern "C" int tq_fp64_fma_rate(tq_ctx* c, int iters, double* lane_ops_per_s) {
    API_BEGIN
    TQ_REQUIRE(c && lane_ops_per_s, "null argument");
    TQ_REQUIRE(iters >= 1 && iters <= (1 << 20), "iters outside [1, 2^20]");
    set_device(c);
    double* sink = static_cast<double*>(scratch(c, S_STAGE, sizeof(double)));
    const int grid = c->sm_count * FR_BLOCKS_PER_SM;
    const double m = 1.0 - 1.0 / 1048576.0, add = 1.0 / 1024.0;
    auto once = [&](int n) {
        launch(c, "fp64_fma_rate", 0, [&] {
            k_fp64_fma_rate<<<grid, FR_BS>>>(m, add, n, sink);
            return 1;
        });
    };
    once(std::min(iters, 64));   // warm-up
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        TQ_CUDA(cudaEventRecord(e0, 0));
        once(iters);
        TQ_CUDA(cudaEventRecord(e1, 0));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double ops = (double)grid * FR_BS * FR_CHAINS * (double)iters;
    *lane_ops_per_s = ops / (best * 1e-3);
    API_END
}
