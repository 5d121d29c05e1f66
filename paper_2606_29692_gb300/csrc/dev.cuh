// Device helpers shared by the kernels.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "common.h"

namespace tq {

// complex type per precision: float2 (TQ_C64) or double2 (TQ_C128)
template <typename T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

__device__ __forceinline__ int parity32(uint32_t v) { return __popc(v) & 1; }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Error-free float32 sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Warp sum of float32 partials carried as (hi, lo) pairs with TwoSum at
// every level; lane 0 returns hi + lo in float64.  Keeps the reduction
// accurate to float64 level without float64 arithmetic on every lane.
__device__ __forceinline__ double warp_sum_compensated(float v) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        hi = s;
        lo = lo + ol + e;
    }
    return (double)hi + (double)lo;
}
__device__ __forceinline__ double warp_sum_compensated(double v) { return warp_sum(v); }

// The same for per-lane (hi, lo) pairs.
__device__ __forceinline__ double warp_sum_compensated_pair(float hi, float lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, oh, s, e);
        hi = s;
        lo = lo + ol + e;
    }
    return (double)hi + (double)lo;
}

// Block-wide float64 sum of `n` values per thread (n <= 4); result valid in
// thread 0.  `sh` needs blockDim/32 * n doubles.  Deterministic: fixed tree.
template <int n>
__device__ __forceinline__ void block_sum(double (&v)[n], double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < n; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < n; ++i) sh[wid * n + i] = v[i];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = lane < nw ? sh[lane * n + i] : 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = warp_sum(v[i]);
    }
    __syncthreads();
}

// Sums of n (num, den) partial pairs part[2i], part[2i+1], i in [first,
// first + n), by the whole block in a fixed order (strided, then a fixed
// tree); result in thread 0.  Reads bypass L1 (other CTAs wrote them).
__device__ __forceinline__ void block_sum_pairs(const double* part, int first, int n, double* sh,
                                                double& a, double& b) {
    double v[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        v[0] += __ldcg(part + 2 * (first + i));
        v[1] += __ldcg(part + 2 * (first + i) + 1);
    }
    block_sum<2>(v, sh);
    a = v[0];
    b = v[1];
}

// Value A_k[r][r ^ x] of pool generator k at column col = r ^ x.
template <typename T>
__device__ __forceinline__ T op_value(const PoolView& p, int k, uint32_t col);

template <>
__device__ __forceinline__ float op_value<float>(const PoolView& p, int k, uint32_t col) {
    if (p.fok[k]) {
        const int m = p.fm[k];
        int par = 0;
        for (int i = 0; i < m; ++i) par |= parity32(col & p.fd[3 * k + i]) << i;
        if (par != p.ft[k]) return 0.0f;
        return parity32(col & p.fz0[k]) ? -p.fc0f[k] : p.fc0f[k];
    }
    float s = 0.0f;
    const int nt = p.nterm[k];
    for (int t = 0; t < nt; ++t) {
        const float c = p.cf[8 * k + t];
        s += parity32(col & p.z[8 * k + t]) ? -c : c;
    }
    return s;
}

template <>
__device__ __forceinline__ double op_value<double>(const PoolView& p, int k, uint32_t col) {
    if (p.fok[k]) {
        const int m = p.fm[k];
        int par = 0;
        for (int i = 0; i < m; ++i) par |= parity32(col & p.fd[3 * k + i]) << i;
        if (par != p.ft[k]) return 0.0;
        return parity32(col & p.fz0[k]) ? -p.fc0d[k] : p.fc0d[k];
    }
    double s = 0.0;
    const int nt = p.nterm[k];
    for (int t = 0; t < nt; ++t) {
        const double c = p.cd[8 * k + t];
        s += parity32(col & p.z[8 * k + t]) ? -c : c;
    }
    return s;
}

// Per-op sign data cached in registers for a tile of work.
template <typename T>
struct OpSign {
    int fok, m, t, nt;
    uint32_t x, z0, d0, d1, d2;
    T c0;
    uint32_t z[8];
    T c[8];

    __device__ __forceinline__ void load(const PoolView& p, int k);
    __device__ __forceinline__ T value(uint32_t col) const {
        if (fok) {
            int par = parity32(col & d0);
            if (m > 1) par |= parity32(col & d1) << 1;
            if (m > 2) par |= parity32(col & d2) << 2;
            if (par != t) return T(0);
            return parity32(col & z0) ? -c0 : c0;
        }
        T s = T(0);
        for (int i = 0; i < nt; ++i) s += parity32(col & z[i]) ? -c[i] : c[i];
        return s;
    }
};

template <>
__device__ __forceinline__ void OpSign<float>::load(const PoolView& p, int k) {
    fok = p.fok[k]; m = p.fm[k]; t = p.ft[k]; nt = p.nterm[k];
    x = p.x[k]; z0 = p.fz0[k];
    d0 = p.fd[3 * k]; d1 = p.fd[3 * k + 1]; d2 = p.fd[3 * k + 2];
    c0 = p.fc0f[k];
    for (int i = 0; i < 8; ++i) { z[i] = p.z[8 * k + i]; c[i] = p.cf[8 * k + i]; }
}
template <>
__device__ __forceinline__ void OpSign<double>::load(const PoolView& p, int k) {
    fok = p.fok[k]; m = p.fm[k]; t = p.ft[k]; nt = p.nterm[k];
    x = p.x[k]; z0 = p.fz0[k];
    d0 = p.fd[3 * k]; d1 = p.fd[3 * k + 1]; d2 = p.fd[3 * k + 2];
    c0 = p.fc0d[k];
    for (int i = 0; i < 8; ++i) { z[i] = p.z[8 * k + i]; c[i] = p.cd[8 * k + i]; }
}

// Insert a zero bit at position b of v.
__device__ __forceinline__ uint32_t insert_zero(uint32_t v, int b) {
    const uint32_t lo = v & ((1u << b) - 1u);
    return ((v >> b) << (b + 1)) | lo;
}

}  // namespace tq
