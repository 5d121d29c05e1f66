// Fused CSR SpMV + float64 energy dots over a range of rows (Eq. (1)),
// shared by the single-state and trajectory-batch energy kernels.
#pragma once

#include "dev.cuh"

namespace tq {

constexpr int ENERGY_ROWS = 64;     // rows per work item (8 warps x 8 rows)
constexpr int ENERGY_WARP_ROWS = 8;

// Sum over one CSR row of val[e] * x[col[e]] for the entries e = e0 + lane,
// e0 + lane + L, ... (L lanes per row), four independent gathers in flight
// per lane and the next four columns and values loading behind them.
// Products and sums in T (the state's precision), in entry order.
template <typename T, typename VT, typename V, int L>
__device__ __forceinline__ void row_dot(const int* __restrict__ col, const VT* __restrict__ val,
                                        const V* __restrict__ x, int e0, int e1, int lane, T& px,
                                        T& py) {
    int e = e0 + lane;
    if (e + 3 * L < e1) {
        // software pipelined: the next four columns and values are loaded
        // while this group's four gathers are in flight (same products, same
        // order)
        int c0 = col[e], c1 = col[e + L], c2 = col[e + 2 * L], c3 = col[e + 3 * L];
        VT a0 = val[e], a1 = val[e + L], a2 = val[e + 2 * L], a3 = val[e + 3 * L];
        for (;;) {
            const V v0 = x[c0], v1 = x[c1], v2 = x[c2], v3 = x[c3];
            const int en = e + 4 * L;
            const bool more = en + 3 * L < e1;
            int n0 = 0, n1 = 0, n2 = 0, n3 = 0;
            VT b0 = VT(0), b1 = VT(0), b2 = VT(0), b3 = VT(0);
            if (more) {
                n0 = col[en];
                n1 = col[en + L];
                n2 = col[en + 2 * L];
                n3 = col[en + 3 * L];
                b0 = val[en];
                b1 = val[en + L];
                b2 = val[en + 2 * L];
                b3 = val[en + 3 * L];
            }
            px = fma((T)a0, v0.x, px);
            py = fma((T)a0, v0.y, py);
            px = fma((T)a1, v1.x, px);
            py = fma((T)a1, v1.y, py);
            px = fma((T)a2, v2.x, px);
            py = fma((T)a2, v2.y, py);
            px = fma((T)a3, v3.x, px);
            py = fma((T)a3, v3.y, py);
            e = en;
            if (!more) break;
            c0 = n0; c1 = n1; c2 = n2; c3 = n3;
            a0 = b0; a1 = b1; a2 = b2; a3 = b3;
        }
    }
    for (; e < e1; e += L) {
        const T a = (T)val[e];
        const V v = x[col[e]];
        px = fma(a, v.x, px);
        py = fma(a, v.y, py);
    }
}

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
