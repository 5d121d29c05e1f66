// Fused CSR SpMV + float64 energy dots over a range of rows (Eq. (1)),
// shared by the single-state and trajectory-batch energy kernels.
#pragma once

#include "dev.cuh"

namespace tq {

constexpr int ENERGY_ROWS = 64;     // rows per work item (8 warps x 8 rows)
constexpr int ENERGY_WARP_ROWS = 8;

// Rows [r0, r1) (at most 64) of w = H psi with a block of 256 threads: warp
// w takes rows r0 + 8w .. r0 + 8w + 7; inside the warp, groups of L lanes
// share a row and each group walks 8L/32 consecutive rows.  Per row the
// group strides over the non-zeros with four gathers in flight per lane and
// reduces with an xor butterfly in the state's precision; lane j of the
// group keeps its j-th row's sum and finishes that row in float64
// (diagonal, w, <psi|w>, <psi|psi>).  Loops are uniform per warp, so every
// shuffle has all 32 lanes.
template <typename T, typename VT, int L>
__device__ __forceinline__ void energy_rows(const int* __restrict__ rowptr, const int* __restrict__ col,
                                            const VT* __restrict__ val, const double* __restrict__ diag,
                                            const typename C2<T>::type* __restrict__ psi,
                                            double2* __restrict__ w64, float2* __restrict__ w32,
                                            long long r0, long long r1, double& num, double& den) {
    using V = typename C2<T>::type;
    constexpr int RPG = ENERGY_WARP_ROWS * L / 32 > 0 ? ENERGY_WARP_ROWS * L / 32 : 1;  // rows per group
    const int gl = threadIdx.x % L;
    const long long base = r0 + (threadIdx.x >> 5) * ENERGY_WARP_ROWS + ((threadIdx.x & 31) / L) * RPG;
    T mx = T(0), my = T(0);
    for (int j = 0; j < RPG; ++j) {
        const long long r = base + j;
        T px = T(0), py = T(0);
        if (r < r1) row_dot<T, VT, V, L>(col, val, psi, rowptr[r], rowptr[r + 1], gl, px, py);
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            px += __shfl_xor_sync(0xffffffffu, px, o, L);
            py += __shfl_xor_sync(0xffffffffu, py, o, L);
        }
        if (gl == j) {
            mx = px;
            my = py;
        }
    }
    const long long r = base + gl;
    if (gl < RPG && r < r1) {
        const V pv = psi[r];
        const double prx = (double)pv.x, pry = (double)pv.y;
        const double dg = diag[r];
        const double wx = fma(dg, prx, (double)mx), wy = fma(dg, pry, (double)my);
        if (w64) w64[r] = make_double2(wx, wy);
        if (w32) w32[r] = make_float2((float)wx, (float)wy);
        num += prx * wx + pry * wy;
        den += prx * prx + pry * pry;
    }
}

}  // namespace tq
