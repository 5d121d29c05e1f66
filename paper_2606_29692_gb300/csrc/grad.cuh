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
constexpr int GRAD_U = 4;          // rounds of support rows with loads in flight

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

// Whether row r lies in the support: every condition's parity equals its
// target.
__device__ __forceinline__ bool in_support(const SuppRec& s, uint32_t r) {
    int ok = 1;
    if (s.m > 0) ok &= (parity32(r & s.e0) == (s.target & 1));
    if (s.m > 1) ok &= (parity32(r & s.e1) == ((s.target >> 1) & 1));
    if (s.m > 2) ok &= (parity32(r & s.e2) == ((s.target >> 2) & 1));
    return ok != 0;
}

// Pair u -> support row r, with the generator's masks worked out once per
// tile: a zero inserted at the representative's bit (position hp among the
// free bits) and at each pivot (ascending), as (v & lo) | ((v & ~lo) << 1)
// with lo the bits below the insertion (one less than the inserted bit);
// then each pivot set to its target xor the parity of r over its condition
// mask (every mask holds its own pivot and no other, so the parities read
// only free bits).  An absent condition has pivot bit 0.
struct RowExp {
    uint32_t hb;                   // 1 << hp
    uint32_t pb0, pb1, pb2;        // pivot bits (0: no such condition)
    uint32_t e0, e1, e2;           // condition masks
    uint32_t tb;                   // target bits at the pivots
};

__device__ __forceinline__ RowExp make_rowexp(const SuppRec& s, int hp) {
    RowExp x;
    x.hb = 1u << hp;
    x.pb0 = s.m > 0 ? 1u << s.p0 : 0u;
    x.pb1 = s.m > 1 ? 1u << s.p1 : 0u;
    x.pb2 = s.m > 2 ? 1u << s.p2 : 0u;
    x.e0 = s.e0;
    x.e1 = s.e1;
    x.e2 = s.e2;
    x.tb = ((s.target & 1) ? x.pb0 : 0u) | ((s.target & 2) ? x.pb1 : 0u) | ((s.target & 4) ? x.pb2 : 0u);
    return x;
}

__device__ __forceinline__ uint32_t ins0(uint32_t v, uint32_t bit) {
    const uint32_t lo = bit - 1u;
    return (v & lo) | ((v & ~lo) << 1);
}

// supp_row(s, insert_zero(u, hp)), the same row.
__device__ __forceinline__ uint32_t expand_row(const RowExp& x, uint32_t u) {
    uint32_t r = ins0(u, x.hb);
    if (x.pb0) r = ins0(r, x.pb0);
    if (x.pb1) r = ins0(r, x.pb1);
    if (x.pb2) r = ins0(r, x.pb2);
    uint32_t piv = 0u;
    if (x.pb0) piv |= x.pb0 & (0u - (__popc(r & x.e0) & 1u));
    if (x.pb1) piv |= x.pb1 & (0u - (__popc(r & x.e1) & 1u));
    if (x.pb2) piv |= x.pb2 & (0u - (__popc(r & x.e2) & 1u));
    return r | (piv ^ x.tb);
}

// Support row u itself (no representative bit): u with zeros at the
// pivots, each then set by its condition; the same row as supp_row(s, u).
__device__ __forceinline__ uint32_t expand_support_row(const RowExp& x, uint32_t u) {
    uint32_t r = u;
    if (x.pb0) r = ins0(r, x.pb0);
    if (x.pb1) r = ins0(r, x.pb1);
    if (x.pb2) r = ins0(r, x.pb2);
    uint32_t piv = 0u;
    if (x.pb0) piv |= x.pb0 & (0u - (__popc(r & x.e0) & 1u));
    if (x.pb1) piv |= x.pb1 & (0u - (__popc(r & x.e1) & 1u));
    if (x.pb2) piv |= x.pb2 & (0u - (__popc(r & x.e2) & 1u));
    return r | (piv ^ x.tb);
}

// Sum of one item over the block of GRAD_TPB threads; valid in thread 0.
// `sh` holds 2 * warps doubles.  W is float2 (complex64: w in float32) or
// double2.
//
// The map u -> support row is affine over GF(2) (zeros inserted, then each
// pivot set to a parity of the row plus its target), so
// row(a ^ b) = row(a) ^ row(b) ^ row(0), with row(0) the target bits.  The
// thread's rows are u = (u0 + GRAD_TPB k) ^ tid, u0 and GRAD_TPB k clear of
// the thread bits, hence row = R_k ^ L with L = row(tid) ^ row(0) worked out
// once and R_k = row(u0 + GRAD_TPB k) by lane k of the warp (k < 32), read
// with a shuffle: the same rows, visited in the same order, as expanding
// every u.
static_assert(GRAD_CHUNK % GRAD_TPB == 0 && GRAD_CHUNK <= 32 * GRAD_TPB, "one row base per lane");
template <typename T, typename W, typename V>
__device__ __forceinline__ double grad_item(const SuppRec& s, T c0, const W* __restrict__ w,
                                            const V* __restrict__ psi, uint32_t u0, uint32_t cnt,
                                            double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = GRAD_TPB >> 5;
    const RowExp rx = make_rowexp(s, 0);   // the representative bit is not used here
    const uint32_t L = expand_support_row(rx, threadIdx.x) ^ rx.tb;
    const uint32_t Rl = expand_support_row(rx, u0 + (uint32_t)lane * GRAD_TPB);
    const uint32_t nk = (cnt + GRAD_TPB - 1) / GRAD_TPB;
    T hi = T(0), lo = T(0);
    // GRAD_U rounds' loads are issued before their products are summed (in
    // round order); k + u < 32 since nk <= 32 and GRAD_U divides 32
    for (uint32_t k = 0; k < nk; k += GRAD_U) {
        uint32_t r[GRAD_U];
        bool in[GRAD_U];
        W wr[GRAD_U];
        V v[GRAD_U];
#pragma unroll
        for (int u = 0; u < GRAD_U; ++u) {
            r[u] = __shfl_sync(0xffffffffu, Rl, k + u) ^ L;
            in[u] = threadIdx.x + (k + u) * GRAD_TPB < cnt;
        }
#pragma unroll
        for (int u = 0; u < GRAD_U; ++u)
            if (in[u]) {
                wr[u] = w[r[u]];
                v[u] = psi[r[u] ^ s.x];
            }
#pragma unroll
        for (int u = 0; u < GRAD_U; ++u)
            if (in[u]) {
                const T sg = parity32((r[u] ^ s.x) & s.z0) ? -c0 : c0;
                const T prod = sg * fma((T)wr[u].x, (T)v[u].x, (T)wr[u].y * (T)v[u].y);
                if constexpr (sizeof(T) == 4) {
                    T sum, err;
                    two_sum(hi, prod, sum, err);
                    hi = sum;
                    lo += err;
                } else {
                    hi += prod;
                }
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
