// Support-only batched Taylor-5 update (Sec. III-C, Eqs. (6)-(8)).
//
// Each product v_k = A v_{k-1} of Eq. (7) costs O(nnz(A)), and a pool
// generator's non-zeros sit on its support S = {r : A[r][r ^ x] != 0}: a
// single excitation has |S| = D/2, a double D/8.  A row outside S is
// annihilated by A, so every term k >= 1 of Eq. (6) leaves it at zero and
// psi'[r] = psi[r] there.  An in-place update therefore reads and writes
// the amplitudes of S only, where the full-state pair kernel streams all D.
//
// S is an affine subspace of codimension m (the generator's conditions on
// the column, rewritten on the row: pivots p_i and masks e_i, as the
// gradient kernel uses them) and is closed under r -> r ^ x.  One member
// of each pair {r, r ^ x} is taken: the one whose bit h is 0, h a free
// (non-pivot) bit of x (one always exists: if every set bit of x were a
// pivot, the conditions A x = 0 on S would force x = 0).  Pair u of a
// generator is then u with a zero inserted at h's position among the free
// bits, expanded by the pivots.  Consecutive u give consecutive rows
// wherever the low bits are free, so a warp's loads stay coalesced.
//
// The squared norm is carried, not recomputed: on exit
// ||psi'||^2 = ||psi||^2 + sum_S (|psi'_r|^2 - |psi_r|^2).  In complex64
// each difference is formed as (a' - a)(a' + a) per component, so the small
// change keeps its relative accuracy; complex128 pairs in closed form add
// (c5^2 + s5^2 - 1) (|psi_r|^2 + |psi_q|^2), exact for A^2 = -I.  The five
// products run exactly as in the full-state kernel (complex64: packed
// float32 chain; complex128 with entries +-1: the closed form
// c5 psi + s5 A psi), so the two kernels give equal amplitudes.
#include "dev.cuh"
#include "grad.cuh"
#include "pair.cuh"
#include "tma.cuh"

#include <algorithm>

namespace tq {

namespace {

constexpr int SUPP_BS = 128;   // threads per CTA of both support-only forms

// Conditions of the support (codimension m): the pivot bits present.
__device__ __forceinline__ int rowexp_m(const RowExp& x) { return (x.pb0 != 0u) + (x.pb1 != 0u) + (x.pb2 != 0u); }

// What the update loops read of a generator: its X-mask, sign mask, row
// expansion and leading coefficient.
template <typename T>
struct SupOp {
    uint32_t x, z0;
    RowExp rx;
    int unit;    // every entry of A is 0 or +-1
    int c0neg;
    int px;      // parity(x & z0): the sign bit of A[r][q] is that of A[q][r] xor px
    T c0;
};

template <typename T>
__device__ __forceinline__ SupOp<T> load_supop(const PoolView& p, int k) {
    SupOp<T> o;
    const SuppRec s = load_supp(p, k);
    o.x = s.x;
    o.z0 = s.z0;
    o.rx = make_rowexp(s, p.supp[k].z);
    o.c0 = sizeof(T) == 4 ? (T)p.fc0f[k] : (T)p.fc0d[k];
    o.unit = fabsf(p.fc0f[k]) == 1.0f;
    o.c0neg = p.fc0f[k] < 0.0f;
    o.px = parity32(s.x & s.z0);
    return o;
}

// A complex64 warp partial of norm changes as a (sum, 0) float pair in the
// 8-byte slot, by a plain float32 shuffle tree: the summands are the
// squared-norm changes of the warp's pairs (about theta^6 / 360 and
// rounding), far below the float64 norm they are added to, so the
// compensated tree of store_partial buys nothing here.
__device__ __forceinline__ void store_partial_small(double* slot, float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2*>(slot) = make_float2(v, 0.f);
}
__device__ __forceinline__ void store_partial_small(double* slot, double v) { store_partial(slot, v); }

// Start of tile tl's pair range when a generator's 2^lp support pairs are
// split over 2^lt tiles: tl 2^lp / 2^lt by shifts (both are powers of two).
__device__ __forceinline__ uint32_t pair_bound(int lp, unsigned tl, int lt) {
    return (uint32_t)(((unsigned long long)tl << lp) >> lt);
}

// The update of one support pair (r, q = r ^ x) with nr, nq the sign bits of
// A[r][q] and A[q][r].  Returns true when the pair took the complex128
// closed form (entries +-1, A[q][r] = -A[r][q], so A^2 = -I on the pair):
// there |psi'_r|^2 + |psi'_q|^2 = (c5^2 + s5^2)(|psi_r|^2 + |psi_q|^2)
// exactly, and the caller adds the norm change in closed form.
template <typename T>
__device__ __forceinline__ bool sup_pair(const SupOp<T>& op, int nr, int nq, const T (&cf)[6], double c5,
                                         double s5, typename C2<T>::type& ar, typename C2<T>::type& aq) {
    if constexpr (sizeof(T) == 8) {
        if (op.unit && nr != nq) {
            const int sr = (nr != op.c0neg) ? -1 : 1;
            closed_pair_sign(sr, -sr, cf, c5, s5, ar, aq);
            return true;
        }
    }
    chain_pair(nr ? -op.c0 : op.c0, nq ? -op.c0 : op.c0, cf, ar, aq);
    return false;
}

__device__ __forceinline__ double pair_norm2(double2 a, double2 b, double acc) {
    return fma(a.x, a.x, fma(a.y, a.y, fma(b.x, b.x, fma(b.y, b.y, acc))));
}
__device__ __forceinline__ double pair_norm2(float2, float2, double acc) { return acc; }

// c5^2 + s5^2 - 1 for the fifth-order series of a generator with A^2 = -I:
// theta^6/360 - theta^8/960 + theta^10/14400, without the cancellation of
// forming c5^2 + s5^2 first.
__device__ __forceinline__ double norm_growth(double theta) {
    const double t2 = theta * theta, t6 = t2 * t2 * t2;
    return t6 * fma(t2, fma(t2, 1.0 / 14400.0, -1.0 / 960.0), 1.0 / 360.0);
}

// The float64 coefficients of one tile: theta^k / k! (k = 0..5), the
// closed-form c5 and s5, and the norm growth, in that order.
constexpr int N_COEF = 9;
__device__ __forceinline__ void tile_coefs(double theta, double* sc) {
    double cf[6], c5, s5;
    taylor_coefs_fast<double>(theta, cf);
    closed_coefs(cf, c5, s5);
#pragma unroll
    for (int k = 0; k < 6; ++k) sc[k] = cf[k];
    sc[6] = c5;
    sc[7] = s5;
    sc[8] = norm_growth(theta);
}

// Updates the support pairs [i0, i1) of one state with the tile's
// coefficients (c5, s5 and growth are used by complex128 only); returns the
// thread's sum of |psi'|^2 - |psi|^2.
template <typename T, int PPT>
__device__ __forceinline__ T support_tile(const SupOp<T>& op, const T (&cf)[6], double c5, double s5, double growth,
                                          typename C2<T>::type* __restrict__ base, uint32_t i0, uint32_t i1) {
    using V = typename C2<T>::type;
    T delta = T(0);
    double nsq = 0.0;   // complex128 closed-form pairs: sum of |psi|^2 before the update
    for (uint32_t i = i0 + threadIdx.x; i < i1; i += SUPP_BS * PPT) {
        uint32_t rr[PPT];
        V a[PPT], b[PPT];
        bool ok[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const uint32_t u = i + j * SUPP_BS;
            ok[j] = u < i1;
            if (!ok[j]) continue;
            const uint32_t r = expand_row(op.rx, u);
            rr[j] = r;
            a[j] = base[r];
            b[j] = base[r ^ op.x];
        }
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            if (!ok[j]) continue;
            const uint32_t r = rr[j], q = r ^ op.x;
            const int nq = parity32(r & op.z0), nr = nq ^ op.px;   // signs of A[q][r], A[r][q]
            V ar = a[j], aq = b[j];
            if (sup_pair<T>(op, nr, nq, cf, c5, s5, ar, aq)) {
                nsq = pair_norm2(a[j], b[j], nsq);
            } else {
                delta += (ar.x - a[j].x) * (ar.x + a[j].x) + (ar.y - a[j].y) * (ar.y + a[j].y);
                delta += (aq.x - b[j].x) * (aq.x + b[j].x) + (aq.y - b[j].y) * (aq.y + b[j].y);
            }
            base[r] = ar;
            base[q] = aq;
        }
    }
    if constexpr (sizeof(T) == 8) delta += growth * nsq;
    return delta;
}

// Persistent grid over (state, tile) items; tile tl of a state whose
// generator has P support pairs covers pairs [tl P / tps, (tl + 1) P / tps)
// (tps, the tiles per state, a power of two).
// With one tile per state and `norm2` set, the CTA finishes the state's
// norm itself (norm2[b] += the fixed-order sum of its warps' partials);
// otherwise every warp leaves its partial for the reduction kernel.  In
// complex128 with one tile per state, thread 0 also works out the next
// tile's coefficients between the norm's two barriers, once per CTA: the
// float64 pipe is this kernel's limit, and every warp would otherwise
// repeat them.  With `sched` (and one tile per state, norm2 set) states
// are handed out dynamically, as in the pipelined form below: thread 0
// requests the state after next at the top of each state, and the value is
// read after the state's first barrier (the second barrier separates that
// read from the next request).
template <typename T, int PPT>
__global__ void __launch_bounds__(SUPP_BS)
k_taylor5_support(PoolView p, int n_states, typename C2<T>::type* psi, const int* kk, const double* th,
                  double* partials, int tiles_per_state, double* norm2, unsigned* sched) {
    const int warp = threadIdx.x >> 5;
    constexpr int NW = SUPP_BS / 32;
    __shared__ double red[NW];
    __shared__ double sc[N_COEF];
    __shared__ unsigned next_sh;
    const bool fold = tiles_per_state == 1 && norm2 != nullptr;
    const bool dyn = fold && sched != nullptr;        // uniform
    constexpr bool wide = sizeof(T) == 8;
    const long long D = 1ll << p.nq;
    const unsigned tps = (unsigned)tiles_per_state;
    const int lt = __ffs(tiles_per_state) - 1;        // tps is a power of two
    const unsigned total = (unsigned)n_states * tps;
    unsigned tile = blockIdx.x;
    unsigned queued = tile + gridDim.x;               // the tile after the current one
    if (dyn) {
        if (threadIdx.x == 0) next_sh = tile < total ? gridDim.x + atomicAdd(sched, 1u) : total;
        __syncthreads();
        queued = next_sh;
    }
    int b = (int)(tile >> lt);
    int k = tile < total ? kk[b] : 0;
    double theta = tile < total ? th[b] : 0.0;
    if (wide && fold) {
        if (threadIdx.x == 0 && tile < total) tile_coefs(theta, sc);
        __syncthreads();
    }
    while (tile < total) {
        const unsigned tl = tile & (tps - 1);
        const unsigned ntile = queued;
        if (dyn && threadIdx.x == 0 && ntile < total) next_sh = gridDim.x + atomicAdd(sched, 1u);
        const int nb = (int)(ntile >> lt);
        int nk = 0;
        double nth = 0.0;
        if (ntile < total) {
            nk = kk[nb];
            nth = th[nb];
        }
        double* slot = fold ? &red[warp] : partials + (size_t)tile * NW + warp;
        if (k < 0 || k >= p.M) {
            store_nan_partial(slot, T(0));   // the state is left untouched, its norm poisoned
        } else {
            const SupOp<T> op = load_supop<T>(p, k);
            const int lp = p.nq - rowexp_m(op.rx) - 1;
            const uint32_t i0 = pair_bound(lp, tl, lt), i1 = pair_bound(lp, tl + 1, lt);
            T cf[6];
            double c5 = 0.0, s5 = 0.0, growth = 0.0;
            if (wide && fold) {
#pragma unroll
                for (int j = 0; j < 6; ++j) cf[j] = (T)sc[j];
                c5 = sc[6];
                s5 = sc[7];
                growth = sc[8];
            } else if constexpr (wide) {
                double w[N_COEF];
                tile_coefs(theta, w);
#pragma unroll
                for (int j = 0; j < 6; ++j) cf[j] = (T)w[j];
                c5 = w[6];
                s5 = w[7];
                growth = w[8];
            } else {
                taylor_coefs_fast<T>(theta, cf);
            }
            const T d = support_tile<T, PPT>(op, cf, c5, s5, growth, psi + (long long)b * D, i0, i1);
            store_partial_small(slot, d);
        }
        if (fold) {
            __syncthreads();   // the partials are in red, and every thread has read sc
            if (dyn && ntile < total) queued = next_sh;
            if (threadIdx.x == 0) {
                norm2[b] = norm2[b] + sum_partials<T, NW>(red);
                if (wide && ntile < total) tile_coefs(nth, sc);
            }
            __syncthreads();
        }
        if (!dyn) queued = ntile + gridDim.x;
        tile = ntile;
        b = nb;
        k = nk;
        theta = nth;
    }
    if (dyn && threadIdx.x == 0 && atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
        atomicExch(sched, 0u);       // every request has returned: reset for the next launch
        atomicExch(sched + 1, 0u);
    }
}



// ------------------------------------------------ pipelined (cp.async) form
//
// The same update with the amplitudes staged in shared memory by cp.async:
// each thread copies the PPT pairs of its next pass (of the same tile, or
// the first pass of its CTA's next tile) while it computes the current
// one, so the bytes in flight per SM are bounded by shared memory rather
// than by registers.  Every thread reads back only its own slots, so no
// barrier orders the copies; the CTA synchronises only to finish a norm.

__device__ __forceinline__ void cp_async(void* dst, const float2* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(void* dst, const double2* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <typename T>
struct SupTile {
    SupOp<T> op;
    T theta;           // in the kernel's precision: converted once per tile
    int b;
    int bad;           // op index outside [0, M): state untouched, norm NaN
    uint32_t i0, i1;   // the tile's pair range
};

template <typename T>
__device__ __forceinline__ SupTile<T> sup_tile(const PoolView& p, const int* kk, const double* th, unsigned tile,
                                               int lt) {
    SupTile<T> t;
    t.b = (int)(tile >> lt);
    const unsigned tl = tile & ((1u << lt) - 1u);
    const int k = kk[t.b];
    t.theta = (T)th[t.b];
    t.bad = k < 0 || k >= p.M;
    t.i0 = t.i1 = 0;
    if (!t.bad) {
        t.op = load_supop<T>(p, k);
        const int lp = p.nq - rowexp_m(t.op.rx) - 1;
        t.i0 = pair_bound(lp, tl, lt);
        t.i1 = pair_bound(lp, tl + 1, lt);
    }
    return t;
}

template <typename T, int PPT>
__device__ __forceinline__ void sup_issue(const SupTile<T>& t, uint32_t pos, const typename C2<T>::type* base,
                                          typename C2<T>::type* stage, uint32_t* rows) {
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const uint32_t u = pos + j * SUPP_BS + threadIdx.x;
        if (u < t.i1) {
            const uint32_t r = expand_row(t.op.rx, u);
            rows[j * SUPP_BS + threadIdx.x] = r;
            cp_async(&stage[(2 * j) * SUPP_BS + threadIdx.x], base + r);
            cp_async(&stage[(2 * j + 1) * SUPP_BS + threadIdx.x], base + (r ^ t.op.x));
        }
    }
}

// TOUCH: the memory-only floor of the same pass, every support row
// written back as it was read (no update, no norm change).
template <typename T, int PPT, bool TOUCH = false>
__device__ __forceinline__ T sup_compute(const SupTile<T>& t, uint32_t pos, typename C2<T>::type* base,
                                         const typename C2<T>::type* stage, const uint32_t* rows) {
    using V = typename C2<T>::type;
    if constexpr (TOUCH) {
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const uint32_t u = pos + j * SUPP_BS + threadIdx.x;
            if (u >= t.i1) continue;
            const uint32_t r = rows[j * SUPP_BS + threadIdx.x];
            base[r] = stage[(2 * j) * SUPP_BS + threadIdx.x];
            base[r ^ t.op.x] = stage[(2 * j + 1) * SUPP_BS + threadIdx.x];
        }
        return T(0);
    }
    T cf[6];
    taylor_coefs_typed<T>(t.theta, cf);
    double c5 = 0.0, s5 = 0.0;
    if constexpr (sizeof(T) == 8) closed_coefs(cf, c5, s5);
    T delta = T(0);
    double nsq = 0.0;
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const uint32_t u = pos + j * SUPP_BS + threadIdx.x;
        if (u >= t.i1) continue;
        const uint32_t r = rows[j * SUPP_BS + threadIdx.x], q = r ^ t.op.x;
        const V a = stage[(2 * j) * SUPP_BS + threadIdx.x], b = stage[(2 * j + 1) * SUPP_BS + threadIdx.x];
        const int nq = parity32(r & t.op.z0), nr = nq ^ t.op.px;   // q & z0 = (r ^ x) & z0
        V ar = a, aq = b;
        if (sup_pair<T>(t.op, nr, nq, cf, c5, s5, ar, aq)) {
            nsq = pair_norm2(a, b, nsq);
        } else {
            delta += (ar.x - a.x) * (ar.x + a.x) + (ar.y - a.y) * (ar.y + a.y);
            delta += (aq.x - b.x) * (aq.x + b.x) + (aq.y - b.y) * (aq.y + b.y);
        }
        base[r] = ar;
        base[q] = aq;
    }
    if constexpr (sizeof(T) == 8) delta += norm_growth((double)t.theta) * nsq;
    return delta;
}

// norm2 += the CTA's warp partials, by warp 0: a fixed-order shuffle tree
// (complex64: TwoSum-compensated float32 over the (hi, lo) slots; complex128:
// float64), then one float64 addition.  Keeps the float64 pipe, which
// issues a warp instruction every 64 cycles on this part, out of the
// per-state finish.
template <typename T, int NW>
__device__ __forceinline__ void warp0_finish(const double* red, double* norm2) {
    const int lane = threadIdx.x & 31;
    if constexpr (sizeof(T) == 4) {
        float hi = 0.f, lo = 0.f;
        if (lane < NW) {
            const float2 hl = *reinterpret_cast<const float2*>(&red[lane]);
            hi = hl.x;
            lo = hl.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, hi, o);
            const float ol = __shfl_down_sync(0xffffffffu, lo, o);
            float sum, err;
            two_sum(hi, oh, sum, err);
            hi = sum;
            lo = lo + ol + err;
        }
        if (lane == 0) *norm2 = *norm2 + ((double)hi + (double)lo);
    } else {
        double v = lane < NW ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) *norm2 = *norm2 + v;
    }
}

// With one tile per state and norm2 set, the CTA finishes each state's
// norm itself: its warps' partials go to one of two shared buffers, one
// barrier, then warp 0 adds them to norm2[b] (warp0_finish) while the
// other warps start the next tile, whose partials go to the other buffer;
// warp 0 reaches that tile's barrier only after reading this one.
// In that form, with `sched` set, states are handed out dynamically: a
// single costs four times a double, so a fixed stride leaves the CTAs that
// drew more singles running long after the rest (a spread of about 17 % per
// CTA over 18 states).  Thread 0 requests the state after next from
// sched[0] while the current one is processed, and the per-state barrier
// publishes it; the last CTA to finish (sched[1]) sets both counters back
// to zero for the next launch.  The request goes to one of two shared
// slots alternately (the norm buffers' parity), so each write is separated
// by a barrier from every read of the value it replaces.
// CTAs are SUPP_BS = 128 threads: a state's pairs then come to about 11 per
// thread, over which the per-state work (tile set-up, coefficients, the
// norm partial's shuffle tree, barrier, queue) is spread (256 threads:
// 2-3 % slower in both precisions).  The bounds leave the compiler free up
// to 102 registers (complex64, four pairs: 86, five CTAs per SM); holding
// the forms to 48-62 registers for more resident CTAs measured 3 % slower.
template <typename T, int PPT, bool TOUCH = false>
__global__ void __launch_bounds__(SUPP_BS, sizeof(T) == 4 ? (PPT <= 2 ? 5 : (PPT == 4 ? 3 : 1)) : 1)
k_taylor5_support_pipe(PoolView p, int n_states, typename C2<T>::type* psi, const int* kk, const double* th,
                       double* partials, int tiles_per_state, double* norm2, unsigned* sched) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char supp_smem[];
    V* stages = reinterpret_cast<V*>(supp_smem);    // [2][PPT][2][SUPP_BS]
    constexpr int NW = SUPP_BS / 32;
    constexpr int STAGE = 2 * PPT * SUPP_BS;
    uint32_t* rowbuf = reinterpret_cast<uint32_t*>(stages + 2 * STAGE);   // [2][PPT][SUPP_BS]
    __shared__ double red[2][NW];
    __shared__ unsigned next_sh[2];
    // launched with programmatic stream serialisation: the next launch in
    // the stream may be scheduled at once, and every launch waits here,
    // before its first global access, for the previous grid to complete
    // (any state may be written late by it, and the state counters are
    // reset by its last CTA); what overlaps is the launch and the CTAs'
    // start, 1.5 % of a back-to-back step
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int rp = 0;
    const int warp = threadIdx.x >> 5;
    const bool fold = tiles_per_state == 1 && norm2 != nullptr;
    const bool dyn = fold && sched != nullptr;        // uniform
    const long long D = 1ll << p.nq;
    const unsigned tps = (unsigned)tiles_per_state;
    const int lt = __ffs(tiles_per_state) - 1;        // tps is a power of two
    const unsigned total = (unsigned)n_states * tps;
    unsigned tile = blockIdx.x;
    if (tile >= total) {                              // not with the launcher's grid (at most one CTA per tile)
        if (dyn && threadIdx.x == 0 && atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
            atomicExch(sched, 0u);
            atomicExch(sched + 1, 0u);
        }
        return;
    }
    unsigned queued = tile + gridDim.x;               // the tile after the current one
    if (dyn) {
        if (threadIdx.x == 0) next_sh[1] = gridDim.x + atomicAdd(sched, 1u);
        __syncthreads();
        queued = next_sh[1];
    }
    SupTile<T> cur = sup_tile<T>(p, kk, th, tile, lt);
    uint32_t pos = cur.i0;
    int st = 0;
    if (!cur.bad) sup_issue<T, PPT>(cur, pos, psi + (long long)cur.b * D, stages, rowbuf);
    cp_commit();
    T delta = T(0);
    for (;;) {
        // the next pass: later in this tile, or the first of the next tile
        uint32_t npos = pos + SUPP_BS * PPT;
        const bool tile_end = cur.bad || npos >= cur.i1;
        const unsigned ntile = tile_end ? queued : tile;
        const bool more = ntile < total;
        // the request for the tile after ntile overlaps this pass
        if (dyn && tile_end && more && threadIdx.x == 0) next_sh[rp] = gridDim.x + atomicAdd(sched, 1u);
        SupTile<T> nxt = cur;
        if (tile_end && more) {
            nxt = sup_tile<T>(p, kk, th, ntile, lt);
            npos = nxt.i0;
        }
        if (more && !nxt.bad)
            sup_issue<T, PPT>(nxt, npos, psi + (long long)nxt.b * D, stages + (st ^ 1) * STAGE,
                              rowbuf + (st ^ 1) * PPT * SUPP_BS);
        cp_commit();
        cp_wait_one();
        if (!cur.bad)
            delta += sup_compute<T, PPT, TOUCH>(cur, pos, psi + (long long)cur.b * D, stages + st * STAGE,
                                         rowbuf + st * PPT * SUPP_BS);
        if (tile_end) {
            double* slot = fold ? &red[rp][warp] : partials + (size_t)tile * NW + warp;
            if (cur.bad) store_nan_partial(slot, T(0));
            else store_partial_small(slot, delta);
            delta = T(0);
            if (fold) {
                __syncthreads();
                if (dyn && more) queued = next_sh[rp];   // written before the barrier
                if (warp == 0) warp0_finish<T, NW>(red[rp], norm2 + cur.b);
                rp ^= 1;
            } else {
                queued = ntile + gridDim.x;
            }
        }
        if (!more) break;
        tile = ntile;
        cur = nxt;
        pos = npos;
        st ^= 1;
    }
    if (dyn && threadIdx.x == 0) {
        // every request of this CTA has returned; the last CTA to get here
        // resets the counters for the next launch
        if (atomicAdd(sched + 1, 1u) == gridDim.x - 1) {
            atomicExch(sched, 0u);
            atomicExch(sched + 1, 0u);
        }
    }
}

template <typename T, int PPT, bool TOUCH = false>
int launch_support_pipe(const PoolView& p, int n_states, void* psi, const int* k, const double* theta,
                        double* partials, int tps, double* norm2, int sms, int ctas, cudaStream_t s,
                        unsigned* sched) {
    using V = typename C2<T>::type;
    const long long total = (long long)n_states * tps;
    if (total >= (1ll << 31)) return -1;
    const size_t smem = (size_t)2 * PPT * SUPP_BS * (2 * sizeof(V) + sizeof(uint32_t));
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncSetAttribute(k_taylor5_support_pipe<T, PPT, TOUCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_taylor5_support_pipe<T, PPT, TOUCH>, SUPP_BS, smem);
        per_sm = n < 1 ? 1 : n;
    }
    long long grid = (long long)(ctas > 0 && ctas < per_sm ? ctas : per_sm) * sms;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(SUPP_BS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // a launch error stays pending for the caller's cudaGetLastError check
    (void)cudaLaunchKernelEx(&cfg, k_taylor5_support_pipe<T, PPT, TOUCH>, p, n_states, static_cast<V*>(psi), k,
                             theta, partials, tps, norm2, sched);
    return 1;
}

template <typename T, int PPT>
int launch_support(const PoolView& p, int n_states, void* psi, const int* k, const double* theta,
                   double* partials, int tps, double* norm2, int sms, int ctas, cudaStream_t s, unsigned* sched) {
    using V = typename C2<T>::type;
    const long long total = (long long)n_states * tps;
    if (total >= (1ll << 31)) return -1;
    static int per_sm = 0;
    if (per_sm == 0) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_taylor5_support<T, PPT>, SUPP_BS, 0);
        per_sm = n < 1 ? 1 : n;
    }
    long long grid = (long long)(ctas > 0 && ctas < per_sm ? ctas : per_sm) * sms;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    k_taylor5_support<T, PPT><<<(int)grid, SUPP_BS, 0, s>>>(p, n_states, static_cast<V*>(psi), k, theta,
                                                             partials, tps, norm2, sched);
    return 1;
}

template <typename T>
int dispatch_support(int ppt, const PoolView& p, int n_states, void* psi, const int* k, const double* theta,
                     double* partials, int tps, double* norm2, int sms, int ctas, cudaStream_t s,
                     unsigned* sched) {
    switch (ppt) {
        case 1: return launch_support<T, 1>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case 2: return launch_support<T, 2>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case 4: return launch_support<T, 4>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case 8: return launch_support<T, 8>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case -1: return launch_support_pipe<T, 1>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case -2: return launch_support_pipe<T, 2>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case -4: return launch_support_pipe<T, 4>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        case -8: return launch_support_pipe<T, 8>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas, s, sched);
        default: return -1;
    }
}

}  // namespace

// Tiles per state: a double excitation (the smallest support, 2^(nq-4)
// pairs) fills one tile of SUPP_BS * ppt pairs; small batches split states
// further (down to 32 pairs of a double per tile) to fill the GPU.
int support_tiles(int nq, int n_states, int ppt, int sms) {
    // the pipelined form streams several passes per tile: a tile of a
    // double then spans four of its passes
    const int passes = ppt < 0 ? 4 : 1;
    ppt = ppt < 0 ? -ppt : ppt;
    const long long dpairs = nq >= 4 ? 1ll << (nq - 4) : 1;
    long long t = dpairs / ((long long)SUPP_BS * ppt * passes);
    if (t < 1) t = 1;
    const long long want = (4ll * sms + n_states - 1) / std::max(n_states, 1);
    const long long cap = std::max(1ll, dpairs / 32);
    while (t < want && t * 2 <= cap) t *= 2;
    return (int)t;
}

int support_parts(int tiles) { return tiles * (SUPP_BS / 32); }

int launch_taylor5_support_touch(const PoolView& p, int n_states, int prec, int ppt, void* psi, const int* k,
                                 const double* theta, double* partials, int tps, double* norm2, int sms,
                                 cudaStream_t s, int ctas_per_sm, unsigned* sched) {
    if (tps < 1 || (tps & (tps - 1)) != 0) return -1;
    const int u = ppt < 0 ? -ppt : ppt;   // the pipelined form with the same pairs per pass
    if (prec == TQ_C128) {
        switch (u) {
            case 1: return launch_support_pipe<double, 1, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
            case 2: return launch_support_pipe<double, 2, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
            case 4: return launch_support_pipe<double, 4, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
            case 8: return launch_support_pipe<double, 8, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
            default: return -1;
        }
    }
    switch (u) {
        case 1: return launch_support_pipe<float, 1, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
        case 2: return launch_support_pipe<float, 2, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
        case 4: return launch_support_pipe<float, 4, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
        case 8: return launch_support_pipe<float, 8, true>(p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s, sched);
        default: return -1;
    }
}

int launch_taylor5_support(const PoolView& p, int n_states, int prec, int ppt, void* psi, const int* k,
                           const double* theta, double* partials, int tps, double* norm2, int sms,
                           cudaStream_t s, int ctas_per_sm, unsigned* sched) {
    if (tps < 1 || (tps & (tps - 1)) != 0) return -1;   // the kernels split by shifts
    if (prec == TQ_C128)
        return dispatch_support<double>(ppt, p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s,
                                        sched);
    return dispatch_support<float>(ppt, p, n_states, psi, k, theta, partials, tps, norm2, sms, ctas_per_sm, s,
                                   sched);
}

}  // namespace tq
