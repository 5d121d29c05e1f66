// Device code of the pool-gradient reduction (Eq. (5)):
//   g_k = 2 Re<w|A_k psi> / <psi|psi>,  w = H psi,
// shared by the single-state and trajectory-batch kernels.
//
// Only the support of A_k contributes, {r : A_k[r][r^x] != 0}, an affine
// subspace of codimension m (1 for singles, 3 for doubles): support row u is
// u with zeros inserted at m pivot bits, each pivot then set by one parity.
// A work item is (op, chunk of support rows).  Products run in the state's
// precision; complex64 items accumulate TwoSum-compensated float32 sums and
// widen to float64 per warp, so the reduction keeps float64 accuracy without
// float64 arithmetic per row.
#pragma once

#include "dev.cuh"

namespace tq {

constexpr int GRAD_CHUNK = 8192;   // support rows per work item
constexpr int GRAD_TPB = 256;

struct SuppRec {
    uint32_t x, z0, e0, e1, e2;
    int m, p0, p1, p2, target;
};

__device__ __forceinline__ SuppRec load_supp(const PoolView& p, int k) {
    SuppRec s;
    const int4 f = p.supp[k];
    s.x = p.x[k];
    s.z0 = p.fz0[k];
    s.m = f.x & 0xff;
    s.target = f.x >> 8;
    s.p0 = f.y & 0xff;
    s.p1 = (f.y >> 8) & 0xff;
    s.p2 = (f.y >> 16) & 0xff;
    s.e0 = p.supe[3 * k];
    s.e1 = p.supe[3 * k + 1];
    s.e2 = p.supe[3 * k + 2];
    return s;
}

__device__ __forceinline__ uint32_t supp_row(const SuppRec& s, uint32_t u) {
    uint32_t r = u;
    if (s.m > 0) r = insert_zero(r, s.p0);
    if (s.m > 1) r = insert_zero(r, s.p1);
    if (s.m > 2) r = insert_zero(r, s.p2);
    if (s.m > 0) r |= (uint32_t)((s.target ^ parity32(r & s.e0)) & 1) << s.p0;
    if (s.m > 1) r |= (uint32_t)(((s.target >> 1) ^ parity32(r & s.e1)) & 1) << s.p1;
    if (s.m > 2) r |= (uint32_t)(((s.target >> 2) ^ parity32(r & s.e2)) & 1) << s.p2;
    return r;
}

// Sum of one item over the block; valid in thread 0.  `sh` holds 2 * warps
// doubles.  W is float2 (complex64: w in float32) or double2.
template <typename T, typename W, typename V>
__device__ __forceinline__ double grad_item(const SuppRec& s, T c0, const W* __restrict__ w,
                                            const V* __restrict__ psi, uint32_t u0, uint32_t cnt,
                                            double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T hi = T(0), lo = T(0);
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t r = supp_row(s, u0 + i);
        const uint32_t q = r ^ s.x;
        const T sg = parity32(q & s.z0) ? -c0 : c0;
        const W wr = w[r];
        const V v = psi[q];
        const T prod = sg * fma((T)wr.x, (T)v.x, (T)wr.y * (T)v.y);
        if constexpr (sizeof(T) == 4) {
            T sum, err;
            two_sum(hi, prod, sum, err);
            hi = sum;
            lo += err;
        } else {
            hi += prod;
        }
    }
    double part;
    if constexpr (sizeof(T) == 4) part = warp_sum_compensated_pair(hi, lo);
    else part = warp_sum(hi);
    if (lane == 0) sh[wid] = part;
    __syncthreads();
    double tot = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) tot += sh[i];
    __syncthreads();
    return tot;
}

}  // namespace tq
