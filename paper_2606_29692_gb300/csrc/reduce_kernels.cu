// Energy (Eq. (1)), pool gradients (Eq. (5)) and the device-side ADAPT
// glue (Sec. III-D step 3): operator choice, convergence test and the
// line search for the new angle.
//
// Every float64 reduction is deterministic: warps reduce with a fixed
// shuffle tree, CTAs write one partial each, and the last CTA to finish
// (atomic ticket, reset by that CTA) sums the partials in index order.
#include "dev.cuh"
#include "grad.cuh"
#include "spmv.cuh"
#include "tma.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <vector>

namespace tq {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Last-CTA finalisation: returns true in every thread of the last CTA.
__device__ __forceinline__ bool last_block(unsigned* ticket, unsigned nblocks) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        is_last = (t == nblocks - 1);
    }
    __syncthreads();
    return is_last;
}

template <typename T> __device__ __forceinline__ double2 to_d2(typename C2<T>::type v) {
    return make_double2((double)v.x, (double)v.y);
}

// w = H psi (diagonal float64 + CSR off-diagonal) and the float64 sums
// <psi|w>, <psi|psi>: a persistent grid over 256-row items (energy_rows),
// one partial pair per CTA, the last CTA sums them in order.
template <typename T, typename VT, int L>
__global__ void __launch_bounds__(256)
k_energy_csr(HamView h, const typename C2<T>::type* __restrict__ psi, double2* __restrict__ w,
             float2* __restrict__ w32, double* partials, unsigned* ticket, DevStep* step) {
    __shared__ double sh[2 * 8];
    const VT* __restrict__ val = static_cast<const VT*>(h.val);
    double num = 0.0, den = 0.0;
    const long long items = (h.D + ENERGY_ROWS - 1) / ENERGY_ROWS;
    for (long long it = blockIdx.x; it < items; it += gridDim.x) {
        const long long r0 = it * ENERGY_ROWS;
        const long long r1 = r0 + ENERGY_ROWS < h.D ? r0 + ENERGY_ROWS : h.D;
        energy_rows<T, VT, L>(h.rowptr, h.col, val, h.diag, psi, w, w32, r0, r1, num, den);
    }
    double v[2] = {num, den};
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = v[0];
        partials[2 * blockIdx.x + 1] = v[1];
    }
    if (last_block(ticket, gridDim.x)) {
        double a, b;
        block_sum_pairs(partials, 0, (int)gridDim.x, sh, a, b);
        if (threadIdx.x == 0) {
            step->e_num = a;
            step->e_den = b;
            step->energy = a / b;
            *ticket = 0u;
        }
    }
}

// The XOR-ELL energy with the pair stream staged through shared memory by
// bulk copies (TMA).  Each CTA owns a contiguous range of row blocks,
// balanced by pair count (h.xsplit), so its pairs form one contiguous run
// of the (mask, values) arrays.  Warp 8 is the producer: one lane copies
// the run in chunks of XT_CHUNK pairs into a ring of xt_stages<VT>() stages,
// each guarded by a `full` barrier (copy landed) and an `empty` barrier
// (all eight consumer warps are past it).  Warps 0-7 consume: lane l of
// warp w serves rows 2u, 2u+1 (u = l & 3) of pair slot 8w + (l >> 2), so
// the two amplitudes a lane needs, (8R + 2u) ^ x and its bit-0 partner,
// are one aligned 16-byte load for complex64; masks and values come from
// shared memory and psi from L2, so no thread waits on DRAM for the
// stream.  Rounds are straight-line (no per-pair branches).  Each block's
// slot sums are reduced in the warp and parked in shared memory; every
// XT_GROUP blocks (256 rows) the consumers finish one row each in float64,
// with psi and the diagonal loaded at the start of the group, between two
// named barriers.  On a wait time-out the block sets its abort flag,
// finishes its control flow without using the stream, drains its copies
// and reports energy NaN with status TQ_ETIMEOUT.
constexpr int XT_CHUNK_LOG = 8;
constexpr int XT_CHUNK = 1 << XT_CHUNK_LOG;       // pairs per copy chunk
constexpr int XT_CONSUMERS = 256;
constexpr int XT_THREADS = XT_CONSUMERS + 32;
constexpr int XT_SLOTS = XT_CONSUMERS / 4;        // pairs per round of the block
constexpr int XT_GROUP = XT_CONSUMERS / XELL_ROWS;   // row blocks finished together (one row per thread)
// ring depth (a power of two, at least 2: a round spans at most two chunks)
template <typename VT> constexpr int xt_stages() { return sizeof(VT) == 4 ? 4 : 2; }

// The ring is S * XT_CHUNK consecutive pairs (a power of two): pair p of
// the CTA's run sits at ring index (p - k0 * XT_CHUNK) & (S * XT_CHUNK - 1).
template <typename T, typename VT>
struct XtSmem {
    static constexpr int S = xt_stages<VT>();
    uint32_t mask[S * XT_CHUNK];
    VT val[S * XT_CHUNK * XELL_ROWS];
    uint64_t full[S];
    uint64_t empty[S];
    T red[XT_GROUP][XT_CONSUMERS / 32][XELL_ROWS][2];   // per block, warp, row: slot sums
    double sh[2 * (XT_THREADS / 32)];
    int abort;
};

// The amplitudes of rows 2u and 2u + 1 (2u even) at columns a = 2u ^ x and
// a ^ 1.
template <typename V>
__device__ __forceinline__ void gather_two(const V* __restrict__ psi, uint32_t a, V& v0, V& v1) {
    v0 = __ldg(psi + a);
    v1 = __ldg(psi + (a ^ 1u));
}

// K k-steps of one round for one lane: pairs lp0 + 64k (local indices) of
// the ring, rows 2u and 2u + 1.  Straight-line: a pair at or past the
// block's end `le` reads a stale ring entry, whose gather stays in bounds
// (masked index) and whose coefficients are replaced by zero; rows at or
// beyond D (D < 8 only) carry zero values from the build.
template <typename T, typename VT, int K>
__device__ __forceinline__ void xt_round(const uint32_t* mask, const typename C2<VT>::type* sval,
                                         const typename C2<T>::type* __restrict__ psi, uint32_t ru, uint32_t dmask,
                                         int lp0, int kRing, int le, int u, T& ax, T& ay, T& bx, T& by) {
    using V = typename C2<T>::type;
    using VT2 = typename C2<VT>::type;
    uint32_t x[K];
    VT2 av[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int lp = lp0 + XT_SLOTS * k;
        const int ri = lp & kRing;
        x[k] = mask[ri];
        const VT2 a = sval[ri * (XELL_ROWS / 2) + u];
        av[k] = lp < le ? a : VT2{};
    }
    V v0[K], v1[K];
#pragma unroll
    for (int k = 0; k < K; ++k) gather_two(psi, (ru ^ x[k]) & dmask, v0[k], v1[k]);
    if constexpr (sizeof(T) == 4) {
        // packed float32x2: (re, im) of a row in one instruction
        float2 A = make_float2(ax, ay), B = make_float2(bx, by);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            A = __ffma2_rn(make_float2(av[k].x, av[k].x), v0[k], A);
            B = __ffma2_rn(make_float2(av[k].y, av[k].y), v1[k], B);
        }
        ax = A.x;
        ay = A.y;
        bx = B.x;
        by = B.y;
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            ax = fma((T)av[k].x, v0[k].x, ax);
            ay = fma((T)av[k].x, v0[k].y, ay);
            bx = fma((T)av[k].y, v1[k].x, bx);
            by = fma((T)av[k].y, v1[k].y, by);
        }
    }
}

template <typename T, typename VT>
__global__ void __launch_bounds__(XT_THREADS, sizeof(VT) == 4 ? 3 : 2)
k_energy_xell_tma(HamView h, const typename C2<T>::type* __restrict__ psi, double2* __restrict__ w,
                  float2* __restrict__ w32, double* partials, unsigned* ticket, DevStep* step, int withhold) {
    using V = typename C2<T>::type;
    constexpr int S = xt_stages<VT>();
    extern __shared__ __align__(128) unsigned char xt_raw[];
    XtSmem<T, VT>& sm = *reinterpret_cast<XtSmem<T, VT>*>(xt_raw);
    volatile int* abort = &sm.abort;
    const int t = threadIdx.x;
    const VT* __restrict__ xval = static_cast<const VT*>(h.xval);
    const long long b0 = h.xsplit[blockIdx.x], b1 = h.xsplit[blockIdx.x + 1];
    const int P0 = h.xptr[b0], P1 = h.xptr[b1];
    const int k0 = P0 / XT_CHUNK;
    const int nk = P1 > P0 ? (P1 - 1) / XT_CHUNK - k0 + 1 : 0;
    if (t == 0) {
        for (int st = 0; st < S; ++st) {
            mbar_init(&sm.full[st], 1);
            mbar_init(&sm.empty[st], XT_CONSUMERS / 32);
        }
        sm.abort = 0;
        mbar_init_fence();
    }
    __syncthreads();
    double num = 0.0, den = 0.0;
    if (t >= XT_CONSUMERS) {
        if (t == XT_CONSUMERS) {
            constexpr unsigned kBytes = XT_CHUNK * (4 + XELL_ROWS * sizeof(VT));
            int fills[S];
            for (int st = 0; st < S; ++st) fills[st] = 0;
            for (int j = 0; j < nk; ++j) {
                const int st = j % S;
                if (j >= S && !mbar_wait(&sm.empty[st], ((j / S) - 1) & 1, abort)) break;
                if (j == withhold) continue;       // failure-path test: this chunk never arrives
                ++fills[st];
                mbar_arrive_expect_tx(&sm.full[st], kBytes);
                const size_t c = (size_t)(k0 + j) * XT_CHUNK;
                bulk_load(sm.mask + st * XT_CHUNK, h.xmask + c, XT_CHUNK * 4, &sm.full[st]);
                bulk_load(sm.val + st * XT_CHUNK * XELL_ROWS, xval + c * XELL_ROWS,
                          XT_CHUNK * XELL_ROWS * sizeof(VT), &sm.full[st]);
            }
            // every issued copy lands before the block may exit: wait for the
            // last phase of each stage that was filled (phases complete in order)
            for (int st = 0; st < S; ++st)
                if (fills[st] > 0) mbar_wait(&sm.full[st], (fills[st] - 1) & 1, abort, false);
        }
    } else {
        using VT2 = typename C2<VT>::type;
        const int wid = t >> 5, lane = t & 31, u = lane & 3, sub = lane >> 2;
        const uint32_t dmask = (uint32_t)(h.D - 1);
        const int base = k0 * XT_CHUNK;                   // pair index of ring position 0
        constexpr int kRing = S * XT_CHUNK - 1;
        const VT2* __restrict__ sval = reinterpret_cast<const VT2*>(sm.val);
        int next_wait = 0, next_rel = 0;
        auto wait_next = [&]() {
            uint64_t* bar = &sm.full[next_wait % S];
            const unsigned ph = (unsigned)(next_wait / S) & 1u;
            if (!mbar_try_wait(bar, ph)) mbar_wait(bar, ph, abort);
            ++next_wait;
        };
        // releases every chunk wholly below pair `lo` (waiting first for any
        // chunk this warp has not seen, so arrivals stay in chunk order)
        auto release_below = [&](int lo) {
            const int below = min((lo - base) >> XT_CHUNK_LOG, nk);
            while (next_rel < below) {
                while (next_wait <= next_rel) wait_next();
                __syncwarp();
                if (lane == 0) mbar_arrive(&sm.empty[next_rel % S]);
                ++next_rel;
            }
        };
        int pb = P0, pe = b0 < b1 ? h.xptr[b0 + 1] : P0;
        for (long long G0 = b0; G0 < b1; G0 += XT_GROUP) {
            const long long G1 = G0 + XT_GROUP < b1 ? G0 + XT_GROUP : b1;
            // this thread's row of the group, finished after the group's blocks
            const long long rf = G0 * XELL_ROWS + t;
            const bool fin = rf < G1 * XELL_ROWS && rf < h.D;
            V pr = V{};
            double dg = 0.0;
            if (fin) {
                pr = psi[rf];
                dg = h.diag[rf];
            }
            for (long long R = G0; R < G1; ++R) {
                const int pn = R + 2 <= b1 ? h.xptr[R + 2] : pe;     // next block's end, one block ahead
                const uint32_t ru = (uint32_t)(R * XELL_ROWS + 2 * u);
                T ax = T(0), ay = T(0), bx = T(0), by = T(0);
                const int le = pe - base;                          // block end, local
                // warp-uniform rounds: pairs q + 64k + sub, k < 4
                for (int q = pb + 8 * wid; q < pe; q += 4 * XT_SLOTS) {
                    const int lq = q - base;
                    const int need = (min(lq + 3 * XT_SLOTS + 7, le - 1)) >> XT_CHUNK_LOG;
                    while (next_wait <= need) wait_next();
                    xt_round<T, VT, 4>(sm.mask, sval, psi, ru, dmask, lq + sub, kRing, le, u, ax, ay, bx, by);
                    release_below(q + 4 * XT_SLOTS < pe ? q + 4 * XT_SLOTS : pe);
                }
                release_below(pe);
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    ax += __shfl_xor_sync(0xffffffffu, ax, o);
                    ay += __shfl_xor_sync(0xffffffffu, ay, o);
                    bx += __shfl_xor_sync(0xffffffffu, bx, o);
                    by += __shfl_xor_sync(0xffffffffu, by, o);
                }
                if (lane < 4) {
                    T (*rb)[XELL_ROWS][2] = sm.red[R - G0];
                    rb[wid][2 * u][0] = ax;
                    rb[wid][2 * u][1] = ay;
                    rb[wid][2 * u + 1][0] = bx;
                    rb[wid][2 * u + 1][1] = by;
                }
                pb = pe;
                pe = pn;
            }
            named_sync(XT_CONSUMERS);
            if (fin) {
                T mx = T(0), my = T(0);
#pragma unroll
                for (int k = 0; k < XT_CONSUMERS / 32; ++k) {
                    mx += sm.red[t / XELL_ROWS][k][t % XELL_ROWS][0];
                    my += sm.red[t / XELL_ROWS][k][t % XELL_ROWS][1];
                }
                const double prx = (double)pr.x, pry = (double)pr.y;
                const double wx = fma(dg, prx, (double)mx), wy = fma(dg, pry, (double)my);
                if (w) w[rf] = make_double2(wx, wy);
                if (w32) w32[rf] = make_float2((float)wx, (float)wy);
                num += prx * wx + pry * wy;
                den += prx * prx + pry * pry;
            }
            named_sync(XT_CONSUMERS);
        }
    }
    __syncthreads();
    if (*abort) {
        num = nan("");
        if (t == 0) atomicExch(&step->status, (int)TQ_ETIMEOUT);
    }
    double v[2] = {num, den};
    block_sum<2>(v, sm.sh);
    if (t == 0) {
        partials[2 * blockIdx.x] = v[0];
        partials[2 * blockIdx.x + 1] = v[1];
    }
    if (last_block(ticket, gridDim.x)) {
        double a, b;
        block_sum_pairs(partials, 0, (int)gridDim.x, sm.sh, a, b);
        if (t == 0) {
            step->e_num = a;
            step->e_den = b;
            step->energy = a / b;
            *ticket = 0u;
        }
    }
}

// Same energy from the X-mask-grouped terms (no CSR), one row per lane:
// the warp walks the groups together, so every lane reads the same term
// (a broadcast) and the 32 gathers psi[r ^ x] of its consecutive rows fall
// in aligned runs.  Each lane sums its row's signed terms in float64, group
// by group in term order, then the diagonal terms.  A lane past D (D < 32)
// repeats the warp's first row and adds nothing, so every index stays
// below D.
template <typename T>
__global__ void __launch_bounds__(256)
k_energy_mf(HamView h, const typename C2<T>::type* __restrict__ psi, double* partials,
            unsigned* ticket, DevStep* step) {
    __shared__ double sh[2 * 8];
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    double num = 0.0, den = 0.0;
    for (long long rb = (long long)blockIdx.x * blockDim.x + (threadIdx.x - lane); rb < h.D; rb += stride) {
        const long long r = rb + lane;
        const bool active = r < h.D;
        const uint32_t ru = (uint32_t)(active ? r : rb);
        double sx = 0.0, sy = 0.0, dg = 0.0;
        for (int g = 0; g < h.G; ++g) {
            const uint32_t c = ru ^ h.gx[g];
            double a = 0.0;
            for (int t = h.goff[g]; t < h.goff[g + 1]; ++t)
                a += parity32(c & h.tz[t]) ? -h.tc[t] : h.tc[t];
            const double2 v = to_d2<T>(psi[c]);
            sx = fma(a, v.x, sx);
            sy = fma(a, v.y, sy);
        }
        for (int t = 0; t < h.Kd; ++t) dg += parity32(ru & h.dz[t]) ? -h.dc[t] : h.dc[t];
        if (active) {
            const double2 pr = to_d2<T>(psi[ru]);
            const double wx = fma(dg, pr.x, sx), wy = fma(dg, pr.y, sy);
            num += pr.x * wx + pr.y * wy;
            den += pr.x * pr.x + pr.y * pr.y;
        }
    }
    double v[2] = {num, den};
    block_sum<2>(v, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = v[0];
        partials[2 * blockIdx.x + 1] = v[1];
    }
    if (last_block(ticket, gridDim.x)) {
        double a, b;
        block_sum_pairs(partials, 0, (int)gridDim.x, sh, a, b);
        if (threadIdx.x == 0) {
            step->e_num = a;
            step->e_den = b;
            step->energy = a / b;
            *ticket = 0u;
        }
    }
}

// g_k = 2 Re<w|A_k psi> / <psi|psi> for all k in one persistent launch:
// work items (op, chunk of support rows); per-op tickets pick the CTA that
// finalises g_k from the op's chunk partials in order.
template <typename T, typename W>
__global__ void __launch_bounds__(GRAD_TPB)
k_pool_grad(PoolView p, const W* __restrict__ w, const typename C2<T>::type* __restrict__ psi,
            const DevStep* step, double* partials, unsigned* tickets, double* g,
            const int2* items, int n_items, const int* first_item) {
    __shared__ double sh[GRAD_TPB / 32];
    __shared__ bool last;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 kc = items[it];
        const int k = kc.x;
        const SuppRec s = load_supp(p, k);
        const uint32_t size = (uint32_t)((1ll << p.nq) >> s.m);
        const uint32_t u0 = (uint32_t)kc.y * GRAD_CHUNK;
        const uint32_t cnt = min((uint32_t)GRAD_CHUNK, size - u0);
        const T c0 = sizeof(T) == 4 ? (T)p.fc0f[k] : (T)p.fc0d[k];
        const double v = grad_item<T>(s, c0, w, psi, u0, cnt, sh);
        const int nch = first_item[k + 1] - first_item[k];
        if (threadIdx.x == 0) {
            partials[it] = v;
            __threadfence();
            last = atomicAdd(&tickets[k], 1u) == (unsigned)nch - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            double acc = 0.0;
            for (int i = first_item[k]; i < first_item[k + 1]; ++i) acc += __ldcg(partials + i);
            g[k] = 2.0 * acc / step->e_den;
            tickets[k] = 0u;
        }
        __syncthreads();
    }
}

// Operator choice and convergence (one CTA of SELECT_BS threads).  A
// non-negative double orders like its bit pattern, so max |g| and the
// threshold test run on the integer pipe (float64 compares and maxima each
// hold the float64 pipe for a warp instruction's 64 cycles on this part);
// NaN gradients are skipped.
constexpr int SELECT_BS = 256;
__global__ void __launch_bounds__(SELECT_BS) k_select(const double* g, int M, double eps, int prec, DevStep* step) {
    constexpr int NW = SELECT_BS / 32;
    constexpr unsigned long long kAbs = 0x7fffffffffffffffull, kInf = 0x7ff0000000000000ull;
    __shared__ unsigned long long smax[NW];
    __shared__ int smin[NW];
    __shared__ unsigned long long thr_sh;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long m = 0;
    for (int k = threadIdx.x; k < M; k += SELECT_BS) {
        const unsigned long long a = (unsigned long long)__double_as_longlong(g[k]) & kAbs;
        if (a <= kInf && a > m) m = a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if (lane == 0) smax[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long mm = smax[0];
        for (int i = 1; i < NW; ++i) mm = smax[i] > mm ? smax[i] : mm;
        const double gmax = __longlong_as_double((long long)mm);
        const double tau = prec == TQ_C128 ? 1e-9 * fmax(1.0, gmax) : 1e-5;
        const double t = gmax - tau;
        thr_sh = t > 0.0 ? (unsigned long long)__double_as_longlong(t) : 0ull;   // |g| >= gmax - tau
        smax[0] = mm;
    }
    __syncthreads();
    const unsigned long long thr = thr_sh;
    int best = M;
    for (int k = threadIdx.x; k < M; k += SELECT_BS) {
        const unsigned long long a = (unsigned long long)__double_as_longlong(g[k]) & kAbs;
        if (a <= kInf && a >= thr && k < best) best = k;
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
    if (lane == 0) smin[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = smin[0];
        for (int i = 1; i < NW; ++i) b = min(b, smin[i]);
        const double gmax = __longlong_as_double((long long)smax[0]);
        step->selected = b < M ? b : 0;
        step->max_grad = gmax;
        step->converged = gmax < eps ? 1 : 0;
    }
}

// The line search's vectors psi, u1 = A psi and u2 = A u1 for the selected
// op, interleaved per row as one record {psi, u1, u2, 0} of four complex
// values (32 bytes in complex64, 64 in complex128), so that the pass over H
// gathers all three at a column with one sector (complex64).  In the
// state's precision: the entries of A are +-c0, exact for c0 = +-1.
template <typename T>
__global__ void k_apply_twice(PoolView p, const DevStep* step, const typename C2<T>::type* psi,
                              typename C2<T>::type* z, long long D) {
    using V = typename C2<T>::type;
    if (step->converged) return;
    OpSign<T> op;
    op.load(p, step->selected);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride) {
        const uint32_t r = (uint32_t)i, q = r ^ op.x;
        const T s_r = op.value(q);   // A[r][q]
        const T s_q = op.value(r);   // A[q][r]
        const V pq = psi[q], pr = psi[r];
        const T s2 = s_r * s_q;
        V* rec = z + 4 * i;
        rec[0] = pr;
        rec[1] = V{s_r * pq.x, s_r * pq.y};
        rec[2] = V{s2 * pr.x, s2 * pr.y};
        rec[3] = V{T(0), T(0)};
    }
}

// Error-free float32 accumulation of products: (hi, lo) carries the sum of
// a*v with the rounding of each product (an FMA gives it exactly) and of
// each addition (TwoSum), about 48 significant bits in float32 arithmetic.
struct F32x2 {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_product(float a, float v) {
        const float p = __fmul_rn(a, v);   // not contracted into the sum below
        const float e = fmaf(a, v, -p);
        float s, r;
        two_sum(hi, p, s, r);
        hi = s;
        lo += r + e;
    }
    __device__ __forceinline__ void add(float h2, float l2) {
        float s, r;
        two_sum(hi, h2, s, r);
        hi = s;
        lo += r + l2;
    }
    __device__ __forceinline__ void shfl_xor(int o) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        add(h2, l2);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// y_i = H x_i for the line search's three vectors (psi, A psi, A^2 psi) in
// one pass over H: L lanes per row, 32/L rows per warp, each entry's value
// and column read once and applied to all three.  The diagonal term and
// the results are float64.  Complex64 products run on the float32 pipe
// with compensated sums (F32x2), about 48 bits: the line search decides a
// tie between the two minima of a pi-periodic energy curve at 1e-10, and
// that curve is pi-periodic only through exact relations between its
// coefficients (<H psi|A^2 psi> = -<psi|H psi> when A^2 psi = -psi), which
// hold when all three products share one arithmetic and are accurate well
// below 1e-10; float64 instructions would cost several times more here.
// The record {x0, x1, x2, pad} of row c, as three complex values.
__device__ __forceinline__ void line_rec(const float2* __restrict__ z, long long c, float2 (&v)[3]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(z + 4 * c));
    const float4 b = __ldg(reinterpret_cast<const float4*>(z + 4 * c + 2));
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
}
__device__ __forceinline__ void line_rec(const double2* __restrict__ z, long long c, double2 (&v)[3]) {
    v[0] = __ldg(z + 4 * c);
    v[1] = __ldg(z + 4 * c + 1);
    v[2] = __ldg(z + 4 * c + 2);
}

template <typename T, int L>
__global__ void __launch_bounds__(256)
k_line_spmv(HamView h, const typename C2<T>::type* __restrict__ z, double2* __restrict__ y0,
            double2* __restrict__ y1, double2* __restrict__ y2, const DevStep* gate) {
    using V = typename C2<T>::type;
    if (gate && gate->converged) return;
    const T* __restrict__ val = static_cast<const T*>(h.val);
    const int lane = threadIdx.x & 31, sub = lane & (L - 1);
    constexpr int RPW = 32 / L;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    double2* ys[3] = {y0, y1, y2};
    for (long long r0 = warp * RPW; r0 < h.D; r0 += nwarps * RPW) {
        const long long r = r0 + (lane / L);
        double sx[3], sy[3];
        if constexpr (sizeof(T) == 4) {
            F32x2 ax[3], ay[3];
            if (r < h.D) {
                // four entries in flight per lane: values and columns first,
                // then the four records, then the products in entry order
                constexpr int U = 4;
                const int e1 = h.rowptr[r + 1];
                for (int e0 = h.rowptr[r] + sub; e0 < e1; e0 += U * L) {
                    float a[U];
                    int c[U];
#pragma unroll
                    for (int j = 0; j < U; ++j) {
                        const int e = e0 + j * L;
                        a[j] = e < e1 ? val[e] : 0.f;
                        c[j] = e < e1 ? h.col[e] : -1;
                    }
                    V v[U][3];
#pragma unroll
                    for (int j = 0; j < U; ++j)
                        if (c[j] >= 0) line_rec(z, c[j], v[j]);
#pragma unroll
                    for (int j = 0; j < U; ++j) {
                        if (c[j] < 0) continue;
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            ax[i].add_product(a[j], v[j][i].x);
                            ay[i].add_product(a[j], v[j][i].y);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) {
                    ax[i].shfl_xor(o);
                    ay[i].shfl_xor(o);
                }
                sx[i] = ax[i].value();
                sy[i] = ay[i].value();
            }
        } else {
            double ax[3] = {0.0, 0.0, 0.0}, ay[3] = {0.0, 0.0, 0.0};
            if (r < h.D) {
                for (int e = h.rowptr[r] + sub; e < h.rowptr[r + 1]; e += L) {
                    const double a = val[e];
                    V v[3];
                    line_rec(z, h.col[e], v);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        ax[i] = fma(a, v[i].x, ax[i]);
                        ay[i] = fma(a, v[i].y, ay[i]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) {
                    ax[i] += __shfl_xor_sync(0xffffffffu, ax[i], o);
                    ay[i] += __shfl_xor_sync(0xffffffffu, ay[i], o);
                }
                sx[i] = ax[i];
                sy[i] = ay[i];
            }
        }
        if (sub == 0 && r < h.D) {
            const double d = h.diag[r];
            V p[3];
            line_rec(z, r, p);
#pragma unroll
            for (int i = 0; i < 3; ++i)
                ys[i][r] = make_double2(fma(d, (double)p[i].x, sx[i]), fma(d, (double)p[i].y, sy[i]));
        }
    }
}

// The six Re-dots of the line search, divided by <psi|psi>, with
// w0 = H psi, w1 = H u1, w2 = H u2 from one pass:
// dots = {<psi|w0>, <w0|u1>, <w0|u2>, <u1|w1>, <w1|u2>, <u2|w2>}.  <psi|w0>
// and <w0|u2> are written in the same shape so that u2 = -psi gives
// exactly opposite values (and <u2|w2> exactly <psi|w0>).
template <typename T>
__global__ void __launch_bounds__(256)
k_line_dots(const typename C2<T>::type* z, const double2* w0, const double2* w1, const double2* w2, long long D,
            double* partials, unsigned* ticket, DevStep* step) {
    __shared__ double sh[6 * 8];
    if (step->converged) return;
    double a[6] = {0, 0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride) {
        const double2 x0 = w0[i], x1 = w1[i], x2 = w2[i];
        const double2 p = to_d2<T>(z[4 * i]), v1 = to_d2<T>(z[4 * i + 1]), v2 = to_d2<T>(z[4 * i + 2]);
        a[0] += x0.x * p.x + x0.y * p.y;
        a[1] += x0.x * v1.x + x0.y * v1.y;
        a[2] += x0.x * v2.x + x0.y * v2.y;
        a[3] += v1.x * x1.x + v1.y * x1.y;
        a[4] += x1.x * v2.x + x1.y * v2.y;
        a[5] += x2.x * v2.x + x2.y * v2.y;
    }
    // two-stage block sum (block_sum handles up to 4 values)
    double lo[4] = {a[0], a[1], a[2], a[3]};
    double hi[2] = {a[4], a[5]};
    block_sum<4>(lo, sh);
    block_sum<2>(hi, sh + 32);
    if (threadIdx.x == 0) {
        for (int j = 0; j < 4; ++j) partials[6 * blockIdx.x + j] = lo[j];
        partials[6 * blockIdx.x + 4] = hi[0];
        partials[6 * blockIdx.x + 5] = hi[1];
    }
    if (last_block(ticket, gridDim.x)) {
        // every thread sums a fixed stride of the blocks, then a fixed tree
        double f[6] = {0, 0, 0, 0, 0, 0};
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            for (int j = 0; j < 6; ++j) f[j] += __ldcg(partials + 6 * b + j);
        double lo2[4] = {f[0], f[1], f[2], f[3]};
        double hi2[2] = {f[4], f[5]};
        block_sum<4>(lo2, sh);
        block_sum<2>(hi2, sh + 32);
        if (threadIdx.x == 0) {
            const double tot[6] = {lo2[0], lo2[1], lo2[2], lo2[3], hi2[0], hi2[1]};
            for (int j = 0; j < 6; ++j) step->dots[j] = tot[j] / step->e_den;
            *ticket = 0u;
        }
    }
}

// The line search's matrix elements from the chosen generator's support S
// only.  u1 = A psi and u2 = A^2 psi vanish off S, so every element but
// <psi|H psi> is a sum over rows of S, and on S, u1_r = A[r][r^x] psi_{r^x}
// and u2_r = -psi_r (A^2 = -I there).  Per row r of S the pass keeps three
// sums over the row's entries: y_S over columns in S (H psi_S, psi_S the
// part of psi on S), y_O over the rest, and y_1 (H u1, columns in S).  With
// x0 = (H psi)_r = y_S + y_O + d psi_r and xS = (H psi_S)_r = y_S + d psi_r:
//   H01 = Re<H psi|u1> = sum re(x0, u1)     H02 = Re<H psi|u2> = -sum re(x0, psi)
//   H11 = Re<u1|H u1>  = sum re(u1, y_1 + d u1)
//   H12 = Re<H u1|u2>  = -Re<u1|H psi_S> = -sum re(xS, u1)   (H = H^+)
//   H22 = Re<u2|H u2>  = sum re(xS, psi)
// H00 is the Rayleigh quotient the energy pass of the same step computed:
// it only shifts the curve.
//
// When psi lies in S the curve along exp(theta A) psi is pi-periodic and
// its two minima tie, through H12 = -H01 and H22 = -H02.  Written this way
// both hold bit for bit in any precision: y_O is then exactly zero, so x0
// and xS are the same bits, and each pair of elements sums the same
// products with opposite signs in the same order, with no contraction.  No
// element needs more than the state's own precision, so the sums are plain
// float32 (complex64) or float64 (complex128).
//
template <typename T>
__device__ __forceinline__ T sup_sign(const SuppRec& s, T c0, uint32_t col) {
    return parity32(col & s.z0) ? -c0 : c0;   // A[r][col], r = col ^ x in S
}

// Re(conj(a) b) with no contraction: the same bits for (a, b) and (-a, b)
// up to sign.
__device__ __forceinline__ double re_dot(double2 a, double2 b) {
    return __dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}

// Row sums of one support row before its float64 finish: y_S (columns in
// S) and y_1 (H u1 over columns in S) as compensated (hi, lo) pairs per
// component, y_O (columns outside S) plain.  complex128: float64 sums.
template <typename T> struct LineSums {
    typename C2<T>::type s, o, u;   // y_S, y_O, y_1
};

template <typename T, int L>
__global__ void __launch_bounds__(256)
k_line_support(HamView h, PoolView p, const typename C2<T>::type* __restrict__ psi, DevStep* step,
               double* partials, unsigned* ticket) {
    using V = typename C2<T>::type;
    __shared__ double sh[4 * 8];
    // the sums of a warp's 32 rows, finished in float64 by one lane each
    __shared__ LineSums<T> stash[8][32];
    if (step->converged) return;
    const T* __restrict__ val = static_cast<const T*>(h.val);
    const int k = step->selected;
    const SuppRec s = load_supp(p, k);
    const RowExp rx = make_rowexp(s, 0);
    const T c0 = sizeof(T) == 4 ? (T)p.fc0f[k] : (T)p.fc0d[k];
    const long long nrows = 1ll << (p.nq - s.m);
    const int lane = threadIdx.x & 31, sub = lane & (L - 1), wid = threadIdx.x >> 5;
    constexpr int RPW = 32 / L;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // H01, H02, H11, H12, H22 (before / <psi|psi>)
    // rows per warp group: 32 (one float64 finish per lane) when the support
    // has rows enough for every warp, fewer for small supports so that all
    // warps get work (a power of two, at least the RPW rows of one round)
    int G = 32;
    while (G > RPW && (long long)G * nwarps > nrows) G >>= 1;
    const int rounds = G / RPW;
    for (long long g0 = warp * G; g0 < nrows; g0 += nwarps * G) {
        // `rounds` rounds of RPW rows fill the warp's G slots
        for (int rd = 0; rd < rounds; ++rd) {
            const int slot = rd * RPW + lane / L;
            const long long i = g0 + slot;
            const bool live = i < nrows;
            const uint32_t r = live ? expand_support_row(rx, (uint32_t)i) : 0u;
            LineSums<T> out;
            if constexpr (sizeof(T) == 4) {
                float2 yS = make_float2(0.f, 0.f), yO = yS, y1 = yS;
                if (live) {
                    // U entries per lane in flight; the next U columns and
                    // values load while this group's gathers are out
                    constexpr int U = 4;
                    const int e1 = h.rowptr[r + 1];
                    int e0 = h.rowptr[r] + sub;
                    float av[U];
                    int c[U];
#pragma unroll
                    for (int j = 0; j < U; ++j) {
                        const int e = e0 + j * L;
                        av[j] = e < e1 ? val[e] : 0.f;
                        c[j] = e < e1 ? h.col[e] : -1;
                    }
                    while (e0 < e1) {
                        V v[U], w[U];
                        bool ins[U];
#pragma unroll
                        for (int j = 0; j < U; ++j) {
                            ins[j] = c[j] >= 0 && in_support(s, (uint32_t)c[j]);
                            v[j] = c[j] >= 0 ? __ldg(psi + c[j]) : V{};
                            w[j] = ins[j] ? __ldg(psi + ((uint32_t)c[j] ^ s.x)) : V{};
                        }
                        const int en = e0 + U * L;
                        float nav[U];
                        int nc[U];
#pragma unroll
                        for (int j = 0; j < U; ++j) {
                            const int e = en + j * L;
                            nav[j] = e < e1 ? val[e] : 0.f;
                            nc[j] = e < e1 ? h.col[e] : -1;
                        }
#pragma unroll
                        for (int j = 0; j < U; ++j) {
                            // an entry adds to y_S or to y_O (the other gets an
                            // exact zero); u1_c = A[c][c ^ x] psi_{c ^ x}
                            const float aS = ins[j] ? av[j] : 0.f, aO = ins[j] ? 0.f : av[j];
                            const float a1 = ins[j] ? sup_sign<float>(s, c0, (uint32_t)c[j] ^ s.x) * av[j] : 0.f;
                            yS = __ffma2_rn(make_float2(aS, aS), v[j], yS);
                            yO = __ffma2_rn(make_float2(aO, aO), v[j], yO);
                            y1 = __ffma2_rn(make_float2(a1, a1), w[j], y1);
                        }
                        e0 = en;
#pragma unroll
                        for (int j = 0; j < U; ++j) {
                            av[j] = nav[j];
                            c[j] = nc[j];
                        }
                    }
                }
#pragma unroll
                for (int o = L / 2; o > 0; o >>= 1) {
                    yS.x += __shfl_xor_sync(0xffffffffu, yS.x, o);
                    yS.y += __shfl_xor_sync(0xffffffffu, yS.y, o);
                    yO.x += __shfl_xor_sync(0xffffffffu, yO.x, o);
                    yO.y += __shfl_xor_sync(0xffffffffu, yO.y, o);
                    y1.x += __shfl_xor_sync(0xffffffffu, y1.x, o);
                    y1.y += __shfl_xor_sync(0xffffffffu, y1.y, o);
                }
                out.s = yS;
                out.o = yO;
                out.u = y1;
            } else {
                double ax[3] = {0.0, 0.0, 0.0}, ay[3] = {0.0, 0.0, 0.0};   // y_S, y_O, y_1
                if (live) {
                    for (int e = h.rowptr[r] + sub; e < h.rowptr[r + 1]; e += L) {
                        const double av = val[e];
                        const uint32_t c = (uint32_t)h.col[e];
                        const V v = __ldg(psi + c);
                        if (in_support(s, c)) {
                            ax[0] = fma(av, v.x, ax[0]);
                            ay[0] = fma(av, v.y, ay[0]);
                            const V w = __ldg(psi + (c ^ s.x));
                            const double sg = sup_sign<double>(s, c0, c ^ s.x) * av;
                            ax[2] = fma(sg, w.x, ax[2]);
                            ay[2] = fma(sg, w.y, ay[2]);
                        } else {
                            ax[1] = fma(av, v.x, ax[1]);
                            ay[1] = fma(av, v.y, ay[1]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
#pragma unroll
                    for (int o = L / 2; o > 0; o >>= 1) {
                        ax[q] += __shfl_xor_sync(0xffffffffu, ax[q], o);
                        ay[q] += __shfl_xor_sync(0xffffffffu, ay[q], o);
                    }
                }
                out.s = make_double2(ax[0], ay[0]);
                out.o = make_double2(ax[1], ay[1]);
                out.u = make_double2(ax[2], ay[2]);
            }
            if (sub == 0) stash[wid][slot] = out;
        }
        __syncwarp();
        // lane g < G finishes row g0 + g in float64
        const long long i = g0 + lane;
        if (lane < G && i < nrows) {
            const uint32_t r = expand_support_row(rx, (uint32_t)i);
            const LineSums<T> in = stash[wid][lane];
            const double sSx = (double)in.s.x, sSy = (double)in.s.y;
            const double d = h.diag[r];
            const V pr = psi[r], pq = psi[r ^ s.x];
            const double sg = (double)sup_sign<T>(s, c0, r ^ s.x);
            const double2 p0 = make_double2((double)pr.x, (double)pr.y);
            const double2 u1 = make_double2(sg * (double)pq.x, sg * (double)pq.y);
            // (H psi)_r, (H psi_S)_r and (H u1)_r
            const double2 x0 = make_double2(fma(d, p0.x, sSx + (double)in.o.x), fma(d, p0.y, sSy + (double)in.o.y));
            const double2 xS = make_double2(fma(d, p0.x, sSx), fma(d, p0.y, sSy));
            const double2 x1 = make_double2(fma(d, u1.x, (double)in.u.x), fma(d, u1.y, (double)in.u.y));
            a[0] = __dadd_rn(a[0], re_dot(x0, u1));     // H01
            a[1] = __dsub_rn(a[1], re_dot(x0, p0));     // H02
            a[2] = __dadd_rn(a[2], re_dot(u1, x1));     // H11
            a[3] = __dsub_rn(a[3], re_dot(xS, u1));     // H12
            a[4] = __dadd_rn(a[4], re_dot(xS, p0));     // H22
        }
        __syncwarp();   // the stash is refilled by the next group
    }
    double lo[4] = {a[0], a[1], a[2], a[3]};
    double hi[1] = {a[4]};
    block_sum<4>(lo, sh);
    block_sum<1>(hi, sh + 24);
    if (threadIdx.x == 0) {
        for (int j = 0; j < 4; ++j) partials[5 * blockIdx.x + j] = lo[j];
        partials[5 * blockIdx.x + 4] = hi[0];
    }
    if (last_block(ticket, gridDim.x)) {
        double f[5] = {0, 0, 0, 0, 0};
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
            for (int j = 0; j < 5; ++j) f[j] = __dadd_rn(f[j], __ldcg(partials + 5 * b + j));
        double lo2[4] = {f[0], f[1], f[2], f[3]};
        double hi2[1] = {f[4]};
        block_sum<4>(lo2, sh);
        block_sum<1>(hi2, sh + 24);
        if (threadIdx.x == 0) {
            const double tot[5] = {lo2[0], lo2[1], lo2[2], lo2[3], hi2[0]};
            step->dots[0] = step->energy;
            for (int j = 0; j < 5; ++j) step->dots[j + 1] = tot[j] / step->e_den;
            *ticket = 0u;
        }
    }
}

// E(theta) from sin(theta) and cos(theta).
__device__ __forceinline__ double line_e_sc(const double* c, double s, double co) {
    const double u = 1.0 - co;
    return c[0] + 2 * s * c[1] + 2 * u * c[2] + s * s * c[3] + 2 * s * u * c[4] + u * u * c[5];
}
__device__ __forceinline__ double line_e(const double* c, double th) { return line_e_sc(c, sin(th), cos(th)); }
// dE/dtheta and d2E/dtheta2 from sin(theta) = s and cos(theta) = cc.
__device__ __forceinline__ double line_d1(const double* c, double s, double cc) {
    const double u = 1.0 - cc;
    return 2 * cc * c[1] + 2 * s * c[2] + 2 * s * cc * c[3] + 2 * (cc * u + s * s) * c[4] + 2 * u * s * c[5];
}
__device__ __forceinline__ double line_d2(const double* c, double s, double cc) {
    const double u = 1.0 - cc;
    return -2 * s * c[1] + 2 * cc * c[2] + 2 * (cc * cc - s * s) * c[3] +
           2 * (3 * s * cc - s * u) * c[4] + 2 * (s * s + u * cc) * c[5];
}
__host__ __device__ __forceinline__ double sample_theta(int m) {
    return -kPi + 2.0 * kPi * (double)(m + 1) / 4096.0;
}

// sin and cos of theta0 + d from those of theta0 and the Taylor series of
// sin d and cos d (angle addition).  The polish keeps |d| within one sample
// spacing, 2 pi / 4096 < 1.6e-3, where the first omitted terms (d^9 / 9!,
// d^10 / 10!) are below 1e-30: no float64 sincos per Newton step.
__device__ __forceinline__ void sincos_near(double2 sc0, double d, double& s, double& c) {
    const double q = d * d;
    const double sd = d * fma(q, fma(q, fma(q, -1.0 / 5040.0, 1.0 / 120.0), -1.0 / 6.0), 1.0);
    const double cd = fma(q, fma(q, fma(q, fma(q, 1.0 / 40320.0, -1.0 / 720.0), 1.0 / 24.0), -0.5), 1.0);
    s = fma(sc0.x, cd, sc0.y * sd);
    c = fma(sc0.y, cd, -(sc0.x * sd));
}

// Order-preserving int64 key of a double: the integer order of the keys is
// the numeric order of the values (NaN last); key_value inverts it.
__device__ __forceinline__ long long order_key(double v) {
    if (v != v) return LLONG_MAX;
    const long long b = __double_as_longlong(v);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double key_value(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

// sin and cos of the 4096 sample angles, computed once per context (float64
// transcendentals are slow on this part; the search would otherwise spend
// most of its time on them).
__global__ void k_line_table(double2* sc) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < 4096) {
        const double th = sample_theta(m);
        sc[m] = make_double2(sin(th), cos(th));
    }
}

// Angle for the update: the given one, or the line-search minimiser
// (4096 samples over (-pi, pi], ties within 1e-10 max(1,|E_min|) to the
// smallest |theta| then lowest index, Newton polish within one spacing).
// The samples are spread over LS_BLOCKS blocks, one per thread, from the
// context's sin/cos table; the last block to finish (a ticket) takes the
// minimum, applies the tie rule and polishes.  Energies are kept as
// order-preserving int64 keys, and the tie rule reads the context's rank
// table (rank[m]: the position of sample m in the order (|theta_m|, m),
// from the same float64 |theta_m|), so the minimum, the tolerance test and
// the tie pick are integer work; the float64 pipe issues a warp
// instruction only every 64 cycles on this part.
constexpr int LS_BS = 256;
constexpr int LS_BLOCKS = 4096 / LS_BS;

__global__ void __launch_bounds__(LS_BS)
k_line_search(DevStep* step, double theta_given, const double* theta_list, const double2* __restrict__ sc,
              const int* __restrict__ rank, long long* se, unsigned* ticket) {
    __shared__ long long red[LS_BS / 32];
    __shared__ int redi[LS_BS / 32];
    __shared__ long long thr_sh;
    if (step->converged) return;                 // uniform over the grid
    if (theta_list) theta_given = theta_list[step->iter];
    if (!isnan(theta_given)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) step->theta = theta_given;
        return;
    }
    double c[6];
    c[0] = step->dots[0];   // H00, from the same products as the others
    c[1] = step->dots[1];   // H01
    c[2] = step->dots[2];   // H02
    c[3] = step->dots[3];   // H11
    c[4] = step->dots[4];   // H12
    c[5] = step->dots[5];   // H22
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = LS_BS / 32;
    const int m0 = blockIdx.x * LS_BS + threadIdx.x;
    const double2 t0 = sc[m0];
    const long long key = order_key(line_e_sc(c, t0.x, t0.y));
    se[m0] = key;
    long long mn = key;
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if (lane == 0) red[wid] = mn;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = red[0];
        for (int i = 1; i < NW; ++i) b = min(b, red[i]);
        se[4096 + blockIdx.x] = b;
    }
    __threadfence();                              // every sample visible before the ticket
    if (!last_block(ticket, gridDim.x)) return;
    // the last block: global minimum, tolerance, tie rule, polish
    if (threadIdx.x < 32) {
        long long b = threadIdx.x < LS_BLOCKS ? __ldcg(se + 4096 + threadIdx.x) : LLONG_MAX;
        for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_down_sync(0xffffffffu, b, o));
        if (threadIdx.x == 0) {
            const double emin = key_value(b);
            thr_sh = order_key(emin + 1e-10 * fmax(1.0, fabs(emin)));
        }
    }
    __syncthreads();
    const long long thr = thr_sh;
    int best = INT_MAX;   // rank * 4096 + m of the preferred sample within the tolerance
    {
        // every key load issued before the first comparison waits on one
        constexpr int PER = 4096 / LS_BS;
        long long key_m[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) key_m[j] = __ldcg(se + threadIdx.x + j * LS_BS);
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int m = threadIdx.x + j * LS_BS;
            if (key_m[j] <= thr) best = min(best, rank[m] * 4096 + m);
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
    if (lane == 0) redi[wid] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        int b = redi[0];
        for (int i = 1; i < NW; ++i) b = min(b, redi[i]);
        const int mb = b & 4095;                  // the global minimum is always within the tolerance
        const double th0 = sample_theta(mb);
        const double2 s0 = sc[mb];
        const double e0 = key_value(__ldcg(se + mb));
        const double h = 2.0 * kPi / 4096.0;
        double th = th0;
        for (int it = 0; it < 8; ++it) {
            double sn, cs;
            sincos_near(s0, th - th0, sn, cs);
            const double d2 = line_d2(c, sn, cs);
            if (!(d2 > 0.0)) break;
            const double stp = line_d1(c, sn, cs) / d2;
            const double nt = th - stp;
            if (fabs(nt - th0) > h) break;
            th = nt;
            if (fabs(stp) < 1e-15) break;
        }
        double sn, cs;
        sincos_near(s0, th - th0, sn, cs);
        if (line_e_sc(c, sn, cs) > e0) th = th0;
        step->theta = th;
        *ticket = 0u;
    }
}

}  // namespace

void line_rank_table(int* rank) {
    std::vector<int> idx(4096);
    for (int m = 0; m < 4096; ++m) idx[m] = m;
    std::stable_sort(idx.begin(), idx.end(),
                     [](int a, int b) { return std::fabs(sample_theta(a)) < std::fabs(sample_theta(b)); });
    for (int i = 0; i < 4096; ++i) rank[idx[i]] = i;
}

namespace {

int grid_rows(long long D, int rows_per_block, int sms, int per_sm) {
    long long g = (D + rows_per_block - 1) / rows_per_block;
    const long long cap = (long long)sms * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int energy_grid(long long D, int sms) { return grid_rows(D, ENERGY_ROWS, sms, 8); }

int launch_energy_csr(const HamView& h, const void* psi, int psi_prec, double2* w,
                      double* partials, unsigned* ticket, DevStep* step, int sms, cudaStream_t s) {
    return launch_energy_csr2(h, psi, psi_prec, w, nullptr, partials, ticket, step, sms, s, 32);
}

namespace {

template <typename T, typename VT, int L>
int resident(int sms) {
    static int per = 0;
    if (per == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_energy_csr<T, VT, L>, 256, 0);
        if (per < 1) per = 1;
    }
    return per * sms;
}

template <typename T, typename VT, int L>
void energy_launch(const HamView& h, const void* psi, double2* w, float2* w32, double* partials,
                   unsigned* ticket, DevStep* step, int sms, cudaStream_t s) {
    using V = typename C2<T>::type;
    const long long items = (h.D + ENERGY_ROWS - 1) / ENERGY_ROWS;
    long long grid = resident<T, VT, L>(sms);
    if (grid > items) grid = items;
    k_energy_csr<T, VT, L><<<(int)grid, 256, 0, s>>>(h, static_cast<const V*>(psi), w, w32, partials, ticket,
                                                     step);
}

// The grid energy_launch uses: resident CTAs, at most one per row item.
template <typename T, typename VT, int L>
int energy_csr_grid_t(const HamView& h, int sms) {
    const long long items = (h.D + ENERGY_ROWS - 1) / ENERGY_ROWS;
    long long grid = resident<T, VT, L>(sms);
    return (int)(grid > items ? items : grid);
}

template <typename T, typename VT>
int energy_dispatch(int lanes, const HamView& h, const void* psi, double2* w, float2* w32, double* partials,
                    unsigned* ticket, DevStep* step, int sms, cudaStream_t s) {
    switch (lanes) {
        case 4: energy_launch<T, VT, 4>(h, psi, w, w32, partials, ticket, step, sms, s); return 1;
        case 8: energy_launch<T, VT, 8>(h, psi, w, w32, partials, ticket, step, sms, s); return 1;
        case 16: energy_launch<T, VT, 16>(h, psi, w, w32, partials, ticket, step, sms, s); return 1;
        case 32: energy_launch<T, VT, 32>(h, psi, w, w32, partials, ticket, step, sms, s); return 1;
        default: return -1;
    }
}

}  // namespace

namespace {

template <typename T, typename VT>
void xell_launch(const HamView& h, const void* psi, double2* w, float2* w32, double* partials,
                 unsigned* ticket, DevStep* step, cudaStream_t s, int withhold) {
    using V = typename C2<T>::type;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_energy_xell_tma<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(XtSmem<T, VT>));
        attr = true;
    }
    k_energy_xell_tma<T, VT><<<h.xgrid, XT_THREADS, sizeof(XtSmem<T, VT>), s>>>(
        h, static_cast<const V*>(psi), w, w32, partials, ticket, step, withhold);
}

}  // namespace

int energy_csr_grid(const HamView& h, int psi_prec, int sms) {
    // the schedule launch_energy_csr takes: 32 lanes per row, values in
    // the state's precision
    return psi_prec == TQ_C128 ? energy_csr_grid_t<double, double, 32>(h, sms)
                               : energy_csr_grid_t<float, float, 32>(h, sms);
}

int launch_energy_xell(const HamView& h, const void* psi, int psi_prec, double2* w, float2* w32,
                       double* partials, unsigned* ticket, DevStep* step, cudaStream_t s, int withhold_chunk) {
    if (psi_prec == TQ_C128)
        xell_launch<double, double>(h, psi, w, w32, partials, ticket, step, s, withhold_chunk);
    else
        xell_launch<float, float>(h, psi, w, w32, partials, ticket, step, s, withhold_chunk);
    return 1;
}

// Grid of the staged XOR-ELL energy: resident blocks on `sms` SMs, at most
// one per row block.
int xell_grid(long long n_blocks, int prec, int sms) {
    int per = 0;
    if (prec == TQ_C128) {
        cudaFuncSetAttribute(k_energy_xell_tma<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(XtSmem<double, double>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_energy_xell_tma<double, double>, XT_THREADS,
                                                      sizeof(XtSmem<double, double>));
    } else {
        cudaFuncSetAttribute(k_energy_xell_tma<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(XtSmem<float, float>));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_energy_xell_tma<float, float>, XT_THREADS,
                                                      sizeof(XtSmem<float, float>));
    }
    long long g = (long long)(per < 1 ? 1 : per) * sms;
    if (g > n_blocks) g = n_blocks;
    return (int)(g < 1 ? 1 : g);
}

int xell_chunk_pairs() { return XT_CHUNK; }

int launch_energy_csr2(const HamView& h, const void* psi, int psi_prec, double2* w, float2* w32,
                       double* partials, unsigned* ticket, DevStep* step, int sms, cudaStream_t s,
                       int lanes) {
    if (psi_prec == TQ_C128)
        return energy_dispatch<double, double>(lanes, h, psi, w, w32, partials, ticket, step, sms, s);
    return energy_dispatch<float, float>(lanes, h, psi, w, w32, partials, ticket, step, sms, s);
}

int launch_energy_matrix_free(const HamView& h, const void* psi, int psi_prec, double* partials,
                              unsigned* ticket, DevStep* step, int sms, cudaStream_t s) {
    const long long blocks = (h.D + 255) / 256;                 // one row per thread
    const int grid = (int)(blocks < (long long)sms * 8 ? blocks : (long long)sms * 8);
    if (psi_prec == TQ_C128)
        k_energy_mf<double><<<grid, 256, 0, s>>>(h, static_cast<const double2*>(psi), partials, ticket, step);
    else
        k_energy_mf<float><<<grid, 256, 0, s>>>(h, static_cast<const float2*>(psi), partials, ticket, step);
    return 1;
}

int launch_pool_gradients(const PoolView& p, const double2* w, const float2* w32, const void* psi,
                          int prec, const DevStep* step, double* partials, unsigned* tickets, double* g,
                          int sms, cudaStream_t s) {
    const int n = p.n_gitems;
    const int grid = n < sms * 8 ? n : sms * 8;
    if (prec == TQ_C128)
        k_pool_grad<double, double2><<<grid, GRAD_TPB, 0, s>>>(p, w, static_cast<const double2*>(psi), step,
                                                               partials, tickets, g, p.gitems, n, p.gfirst);
    else
        k_pool_grad<float, float2><<<grid, GRAD_TPB, 0, s>>>(p, w32, static_cast<const float2*>(psi), step,
                                                             partials, tickets, g, p.gitems, n, p.gfirst);
    return 1;
}

int launch_select(const double* g, int M, double eps, int prec, DevStep* step, cudaStream_t s) {
    k_select<<<1, SELECT_BS, 0, s>>>(g, M, eps, prec, step);
    return 1;
}

int launch_apply_twice(const PoolView& p, const DevStep* step, const void* psi, int prec, void* z, cudaStream_t s) {
    const long long D = 1ll << p.nq;
    const int bs = 256;
    const int grid = (int)((D + bs - 1) / bs < 2048 ? (D + bs - 1) / bs : 2048);
    if (prec == TQ_C128)
        k_apply_twice<double><<<grid, bs, 0, s>>>(p, step, static_cast<const double2*>(psi), static_cast<double2*>(z), D);
    else
        k_apply_twice<float><<<grid, bs, 0, s>>>(p, step, static_cast<const float2*>(psi), static_cast<float2*>(z), D);
    return 1;
}

namespace {

template <int L>
int launch_line_spmv_l(const HamView& h, const void* z, double2* y0, double2* y1, double2* y2, const DevStep* gate,
                       int sms, cudaStream_t s) {
    const long long warps = (h.D + 32 / L - 1) / (32 / L);
    long long grid = (warps * 32 + 255) / 256;
    const long long cap = (long long)sms * 16;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (h.prec == TQ_C128)
        k_line_spmv<double, L><<<(int)grid, 256, 0, s>>>(h, static_cast<const double2*>(z), y0, y1, y2, gate);
    else
        k_line_spmv<float, L><<<(int)grid, 256, 0, s>>>(h, static_cast<const float2*>(z), y0, y1, y2, gate);
    return 1;
}

}  // namespace

// Lanes per row by the mean row length: the compensated sums are dependent
// chains, so long rows get more lanes (shorter chains).
int launch_line_spmv_gated(const HamView& h, const void* z, double2* y0, double2* y1, double2* y2,
                           const DevStep* gate, int sms, cudaStream_t s) {
    const long long per_row = h.D > 0 ? h.nnz / h.D : 0;
    if (per_row >= 192) return launch_line_spmv_l<32>(h, z, y0, y1, y2, gate, sms, s);
    if (per_row >= 48) return launch_line_spmv_l<16>(h, z, y0, y1, y2, gate, sms, s);
    return launch_line_spmv_l<8>(h, z, y0, y1, y2, gate, sms, s);
}


namespace {

// Blocks of the support line pass: enough for the largest support (D/2
// rows, a single excitation) at 32/L rows per warp, at most the resident
// blocks (so that the grid-stride loop runs in one wave) and at most 4 per
// SM (the partial slots).
template <typename T, int L>
int line_support_grid(long long D, int sms) {
    static int per = 0;
    if (per == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_line_support<T, L>, 256, 0);
        per = per < 1 ? 1 : (per > 4 ? 4 : per);
    }
    const long long rows = D / 2 > 0 ? D / 2 : 1;
    const long long warps = (rows + 32 / L - 1) / (32 / L);
    long long grid = (warps * 32 + 255) / 256;
    if (grid > (long long)sms * per) grid = (long long)sms * per;
    return grid < 1 ? 1 : (int)grid;
}

template <int L>
int launch_line_support_l(const HamView& h, const PoolView& p, const void* psi, DevStep* step, double* partials,
                          unsigned* ticket, int sms, cudaStream_t s) {
    const int grid = h.prec == TQ_C128 ? line_support_grid<double, L>(h.D, sms) : line_support_grid<float, L>(h.D, sms);
    if (h.prec == TQ_C128)
        k_line_support<double, L><<<grid, 256, 0, s>>>(h, p, static_cast<const double2*>(psi), step, partials, ticket);
    else
        k_line_support<float, L><<<grid, 256, 0, s>>>(h, p, static_cast<const float2*>(psi), step, partials, ticket);
    return 1;
}

}  // namespace

int line_support_partials(int sms) { return 5 * sms * 4; }

int launch_line_support(const HamView& h, const PoolView& p, const void* psi, DevStep* step, double* partials,
                        unsigned* ticket, int sms, cudaStream_t s) {
    const long long per_row = h.D > 0 ? h.nnz / h.D : 0;
    if (per_row >= 192) return launch_line_support_l<32>(h, p, psi, step, partials, ticket, sms, s);
    if (per_row >= 48) return launch_line_support_l<16>(h, p, psi, step, partials, ticket, sms, s);
    return launch_line_support_l<8>(h, p, psi, step, partials, ticket, sms, s);
}

int launch_line_dots(const void* z, const double2* w0, const double2* w1, const double2* w2, int prec, long long D,
                     double* partials, unsigned* ticket, DevStep* step, cudaStream_t s) {
    const int bs = 256;
    const int grid = (int)((D + bs - 1) / bs < 512 ? (D + bs - 1) / bs : 512);
    if (prec == TQ_C128)
        k_line_dots<double><<<grid, bs, 0, s>>>(static_cast<const double2*>(z), w0, w1, w2, D, partials, ticket, step);
    else
        k_line_dots<float><<<grid, bs, 0, s>>>(static_cast<const float2*>(z), w0, w1, w2, D, partials, ticket, step);
    return 1;
}

int launch_line_table(double2* sc, cudaStream_t s) {
    k_line_table<<<16, 256, 0, s>>>(sc);
    return 1;
}

int launch_line_search(DevStep* step, double theta_given, const double* theta_list, const double2* sc,
                       const int* rank, long long* se, unsigned* ticket, cudaStream_t s) {
    k_line_search<<<LS_BLOCKS, LS_BS, 0, s>>>(step, theta_given, theta_list, sc, rank, se, ticket);
    return 1;
}

__global__ void k_step_record(DevStep* step, double* rec, int n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int i = step->iter;
    if (i < n) {
        const bool bad = !step->converged && !(isfinite(step->norm2) && step->norm2 > 0.0);
        double* r = rec + 6 * (size_t)i;
        r[0] = step->energy;
        r[1] = step->max_grad;
        r[2] = step->converged ? 0.0 : step->theta;
        r[3] = (double)step->selected;
        r[4] = (double)step->converged;
        r[5] = bad ? 1.0 : 0.0;
    }
    step->iter = i + 1;
}

int launch_step_record(DevStep* step, double* rec, int n, cudaStream_t s) {
    k_step_record<<<1, 32, 0, s>>>(step, rec, n);
    return 1;
}

}  // namespace tq
