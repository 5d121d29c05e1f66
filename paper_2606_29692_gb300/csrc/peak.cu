// Measured rates of the device that the copy and GEMM peaks beside the
// kernels do not give: the float64 FMA rate (the roofline of the kernels
// that the float64 pipe bounds) and the L2 read rate (the roofline of the
// kernels whose working set stays in L2).
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
//
// The L2 read rate: a buffer well inside L2 read over and over by a full
// grid with 16-byte loads that skip L1, counted in bytes per second.
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

// Reads `n16` 16-byte words, `reps` times over, bypassing L1 (ld.global.cg)
// so that every load is served by L2 once the buffer is resident there.
constexpr int L2_BS = 512;
__global__ void __launch_bounds__(L2_BS) k_l2_read(const uint4* __restrict__ buf, long long n16, int reps,
                                                    unsigned* sink) {
    unsigned acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long q = i + j * stride;
                v[j] = q < n16 ? __ldcg(buf + q) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) acc ^= v[j].x ^ v[j].y ^ v[j].z ^ v[j].w;
        }
    }
    if (acc == 0x9e3779b9u) *sink = acc;   // the buffer is zero: never taken, keeps the loads live
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

extern "C" int tq_l2_read_rate(tq_ctx* c, long long bytes, int reps, double* bytes_per_s) {
    API_BEGIN
    TQ_REQUIRE(c && bytes_per_s, "null argument");
    TQ_REQUIRE(bytes >= (1 << 20) && bytes <= (256ll << 20) && bytes % 16 == 0,
               "bytes outside [1 MiB, 256 MiB] or not a multiple of 16");
    TQ_REQUIRE(reps >= 1 && reps <= 4096, "reps outside [1, 4096]");
    set_device(c);
    unsigned char* buf = static_cast<unsigned char*>(scratch(c, S_STAGE, (size_t)bytes + 256));
    unsigned* sink = reinterpret_cast<unsigned*>(buf + bytes);
    TQ_CUDA(cudaMemset(buf, 0, (size_t)bytes));
    const long long n16 = bytes / 16;
    const int grid = c->sm_count * 4;
    auto once = [&](int n) {
        launch(c, "l2_read_rate", 0, [&] {
            k_l2_read<<<grid, L2_BS>>>(reinterpret_cast<const uint4*>(buf), n16, n, sink);
            return 1;
        });
    };
    once(2);   // warm-up: brings the buffer into L2
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
        TQ_CUDA(cudaEventRecord(e0, 0));
        once(reps);
        TQ_CUDA(cudaEventRecord(e1, 0));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        best = std::min(best, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *bytes_per_s = (double)bytes * reps / (best * 1e-3);
    API_END
}
