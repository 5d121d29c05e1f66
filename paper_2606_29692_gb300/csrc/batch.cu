// Many independent ADAPT trajectories (Sec. III-D loop) of uneven size,
// advanced together.
//
// Every trajectory t has its own Hamiltonian, pool, state, angle list and
// convergence test.  One iteration of all of them is four persistent
// launches, each spanning every trajectory through a static work table:
//   energy   items (t, row block): w_t = H_t psi_t, <psi|w>, <psi|psi>
//            (the trajectory's last item sums its items' parts);
//   grads    items (t, op, chunk): the chunk's part of 2 Re<w_t|A_k psi_t>;
//   select   one warp per t: g_t[k] (divided by <psi|psi>) summed from the
//            chunk parts in a fixed order, k*, max|g|, convergence, angle,
//            record, and the iteration counter advanced; the last block
//            numbers the active trajectories' energy items for the next
//            iteration (prefix counts);
//   update   items (t, tile): the fused Taylor-5 pair update with A_{k*}
//            and the partials of ||psi'||^2.
// The state is renormalised once, after the last iteration (items
// (t, chunk): psi /= ||psi||): every quantity an iteration computes is
// independent of the state's scale (the energy is <psi|H|psi>/<psi|psi>,
// each gradient is divided by <psi|psi>, and the Taylor-5 update is linear),
// so the per-step renormalisation of Sec. III-D changes only rounding.
// The energy launch runs over the numbered items only, which also spreads
// the remaining trajectories' items evenly over the persistent grid; the
// other launches skip finished trajectories by a flag read on the device.
// A gradient item only writes its part (no ticket, fence or finishing
// block): the op's sum waits for the select launch.  The energy items keep
// their ticket, whose end-of-item wait measured faster for the XOR-ELL
// schedule than running on.
// So the whole run (max length x four launches, then the renormalisation)
// is captured once into a CUDA graph and replayed without any host round
// trip.  The SpMV of the energy item runs over the CSR with a lanes-per-row
// schedule (4, 8, 16, 32) or over the XOR-ELL layout, chosen by an
// autotuner.
#include "dev.cuh"
#include "host_util.h"
#include "pair.cuh"
#include "grad.cuh"
#include "spmv.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace tq {

struct TrajDev {
    int nq, M, len, nch, chunk;
    int eoff, ecnt;          // energy items of this trajectory
    int pcnt;                // pair tiles (8 norm partials each)
    long long D;
    long long hf;
    long long nbase;         // first norm-partial slot
    const double* diag;
    const int* rowptr;
    const int* col;
    const void* val;
    const int* xptr;         // XOR-ELL: first pair of each 8-row block
    const uint32_t* xmask;
    const void* xval;        // 8 values per pair
    PoolView pool;
    void* psi;
    double2* w;              // H psi, float64 (complex128 states)
    float2* w32;             // H psi, float32 (complex64 states)
    const double* thetas;
    double* g;
    double* gpart;           // one partial per gradient item of this trajectory
    const int* gfirst;       // first gradient item of each op (M + 1, the pool's table)
    int gbase;               // first gradient item of this trajectory
    double* res_e;
    double* res_g;
    double* res_th;
    int* res_sel;
};

struct TrajState {
    double e_num, e_den, energy, max_grad, theta;
    int selected, converged, iter, active, do_update, updated;
    unsigned etick;
};

namespace {

// The energy launch runs over the energy items of the trajectories still
// active, numbered 0 .. P[n].x - 1 in trajectory order.  Entry
// P[t] = (first number of trajectory t, its first item's table index minus
// that number): item number j belongs to the t with P[t].x <= j < P[t + 1].x
// and is table item j + P[t].y.  `lo` is a t with P[lo].x <= j (0, or the t
// of the block's previous item, since a block's numbers only grow).
__device__ __forceinline__ int active_traj(const int2* __restrict__ P, int n, int lo, int j) {
    int hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(&P[mid].x) <= j) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int BT_BS = 256;
// An energy item is four 64-row blocks: each item pays a descriptor fetch,
// a block sum and a ticket, so longer items spend less on them.
constexpr int ROWS_PER_ITEM = 4 * ENERGY_ROWS;
constexpr int BT_UPT = 2;
constexpr int SCALE_U = 8;
constexpr int SEL_U = 4;

template <typename T> __device__ __forceinline__ double2 d2(typename C2<T>::type v) {
    return make_double2((double)v.x, (double)v.y);
}

template <typename T>
__global__ void kb_reset(const TrajDev* tr, TrajState* ts, const int4* items, int n_items) {
    using V = typename C2<T>::type;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const TrajDev& d = tr[w.x];
        V* psi = static_cast<V*>(d.psi);
        for (int i = threadIdx.x; i < w.z; i += blockDim.x) {
            const long long r = (long long)w.y + i;
            V v;
            v.x = r == d.hf ? 1 : 0;
            v.y = 0;
            psi[r] = v;
        }
        if (w.y == 0 && threadIdx.x == 0) {
            TrajState s{};
            s.active = d.len > 0;
            ts[w.x] = s;
        }
    }
}

// Energy item: ROWS_PER_ITEM rows of one trajectory.  Groups of LPR lanes
// take LPR consecutive rows each; per row the group strides over the
// non-zeros and reduces with an xor butterfly in the state's precision, and
// lane j of the group keeps row j's sum; each lane then finishes its row in
// float64 (diagonal, w, dots).
template <typename T, typename VT, int LPR>
__global__ void __launch_bounds__(BT_BS)
kb_energy(const TrajDev* tr, TrajState* ts, const int4* items, const int2* pre, int n, double* part) {
    using V = typename C2<T>::type;
    __shared__ double sh[2 * (BT_BS / 32)];
    __shared__ bool last;
    const int total = __ldg(&pre[n].x);
    int t = 0;
    for (int j = blockIdx.x; j < total; j += gridDim.x) {
        t = active_traj(pre, n, t, j);
        const int it = j + __ldg(&pre[t].y);
        const TrajDev& d = tr[t];
        const int4 w4 = items[it];
        const V* psi = static_cast<const V*>(d.psi);
        const VT* val = static_cast<const VT*>(d.val);
        double num = 0.0, den = 0.0;
        const long long end = (long long)w4.y + w4.z;
        for (long long r0 = w4.y; r0 < end; r0 += ENERGY_ROWS)
            energy_rows<T, VT, LPR>(d.rowptr, d.col, val, d.diag, psi, d.w, d.w32, r0,
                                    r0 + ENERGY_ROWS < end ? r0 + ENERGY_ROWS : end, num, den);
        double v[2] = {num, den};
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) {
            part[2 * it] = v[0];
            part[2 * it + 1] = v[1];
            __threadfence();
            last = atomicAdd(&ts[t].etick, 1u) == (unsigned)d.ecnt - 1;
        }
        __syncthreads();
        if (last) {
            double a, b;
            block_sum_pairs(part, d.eoff, d.ecnt, sh, a, b);
            if (threadIdx.x == 0) {
                ts[t].e_num = a;
                ts[t].e_den = b;
                ts[t].energy = a / b;
                ts[t].etick = 0u;
            }
        }
        __syncthreads();
    }
}

// The same energy item over the XOR-ELL layout: blocks of 8 rows, each
// X-mask present in a block stored once with its 8 values, so one pair's
// gathers read one aligned run of 8 amplitudes.  Warp w of the block takes
// 4 consecutive row blocks (32 rows); per block, lane l serves pair slot
// l >> 2 (of 8 pairs per round) and rows 2u, 2u + 1 (u = l & 3), whose two
// amplitudes (8R + 2u) ^ x and its bit-0 partner are one aligned 16-byte
// run for complex64.  Four rounds (32 pairs) are in flight per warp, and
// the next four rounds' masks and values load behind their gathers.  The
// slot sums are reduced in the warp and parked in shared memory; each lane
// then finishes one of the warp's 32 rows in float64.
template <typename T, typename VT>
__global__ void __launch_bounds__(BT_BS)
kbx_energy(const TrajDev* tr, TrajState* ts, const int4* items, const int2* pre, int n, double* part) {
    using V = typename C2<T>::type;
    using VT2 = typename C2<VT>::type;
    constexpr int K = 4;                       // rounds of 8 pairs in flight
    __shared__ double sh[2 * (BT_BS / 32)];
    __shared__ bool last;
    __shared__ T stash[BT_BS / 32][32][2];      // per warp, row: (re, im) of the off-diagonal sum
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, slot = lane >> 2, u = lane & 3;
    const int total = __ldg(&pre[n].x);
    int t = 0;
    for (int j = blockIdx.x; j < total; j += gridDim.x) {
        t = active_traj(pre, n, t, j);
        const int it = j + __ldg(&pre[t].y);
        const TrajDev& d = tr[t];
        const int4 w4 = items[it];
        const V* __restrict__ psi = static_cast<const V*>(d.psi);
        const VT2* __restrict__ xv = static_cast<const VT2*>(d.xval);
        const uint32_t dmask = (uint32_t)(d.D - 1);
        const long long r0 = w4.y, r1 = (long long)w4.y + w4.z;
        const long long B0 = r0 / XELL_ROWS + 4 * wid;   // the warp's first block
        double num = 0.0, den = 0.0;
        for (int j = 0; j < 4; ++j) {
            const long long R = B0 + j;
            T ax = T(0), ay = T(0), bx = T(0), by = T(0);
            if (R * XELL_ROWS < r1) {                    // warp-uniform
                const int pb = d.xptr[R], pe = d.xptr[R + 1];
                const uint32_t ru = (uint32_t)(R * XELL_ROWS + 2 * u);
                uint32_t x[K];
                VT2 a[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const int p = pb + slot + 8 * k;
                    x[k] = p < pe ? d.xmask[p] : 0u;
                    a[k] = p < pe ? xv[(size_t)p * (XELL_ROWS / 2) + u] : VT2{};
                }
                for (int q = pb; q < pe; q += 8 * K) {
                    V v0[K], v1[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const uint32_t c = (ru ^ x[k]) & dmask;
                        v0[k] = __ldg(psi + c);
                        v1[k] = __ldg(psi + (c ^ 1u));
                    }
                    const int qn = q + 8 * K;
                    uint32_t nx[K];
                    VT2 na[K];
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int p = qn + slot + 8 * k;
                        nx[k] = p < pe ? d.xmask[p] : 0u;
                        na[k] = p < pe ? xv[(size_t)p * (XELL_ROWS / 2) + u] : VT2{};
                    }
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        ax = fma((T)a[k].x, v0[k].x, ax);
                        ay = fma((T)a[k].x, v0[k].y, ay);
                        bx = fma((T)a[k].y, v1[k].x, bx);
                        by = fma((T)a[k].y, v1[k].y, by);
                    }
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        x[k] = nx[k];
                        a[k] = na[k];
                    }
                }
            }
            // the 8 slots' sums, fixed butterfly over lane bits 2..4
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o);
                ay += __shfl_xor_sync(0xffffffffu, ay, o);
                bx += __shfl_xor_sync(0xffffffffu, bx, o);
                by += __shfl_xor_sync(0xffffffffu, by, o);
            }
            if (slot == 0) {
                stash[wid][8 * j + 2 * u][0] = ax;
                stash[wid][8 * j + 2 * u][1] = ay;
                stash[wid][8 * j + 2 * u + 1][0] = bx;
                stash[wid][8 * j + 2 * u + 1][1] = by;
            }
        }
        __syncwarp();
        {
            const long long r = B0 * XELL_ROWS + lane;
            if (r < r1 && r < d.D) {
                const V pv = psi[r];
                const double prx = (double)pv.x, pry = (double)pv.y;
                const double dg = d.diag[r];
                const double wx = fma(dg, prx, (double)stash[wid][lane][0]);
                const double wy = fma(dg, pry, (double)stash[wid][lane][1]);
                if (d.w) d.w[r] = make_double2(wx, wy);
                if (d.w32) d.w32[r] = make_float2((float)wx, (float)wy);
                num += prx * wx + pry * wy;
                den += prx * prx + pry * pry;
            }
        }
        __syncwarp();
        double v[2] = {num, den};
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) {
            part[2 * it] = v[0];
            part[2 * it + 1] = v[1];
            __threadfence();
            last = atomicAdd(&ts[t].etick, 1u) == (unsigned)d.ecnt - 1;
        }
        __syncthreads();
        if (last) {
            double a, b;
            block_sum_pairs(part, d.eoff, d.ecnt, sh, a, b);
            if (threadIdx.x == 0) {
                ts[t].e_num = a;
                ts[t].e_den = b;
                ts[t].energy = a / b;
                ts[t].etick = 0u;
            }
        }
        __syncthreads();
    }
}

// Gradient item: (t, op, chunk of the op's support rows).
template <typename T>
__global__ void __launch_bounds__(GRAD_TPB)
kb_grad(const TrajDev* tr, const TrajState* ts, const int4* items, int n_items) {
    using V = typename C2<T>::type;
    __shared__ double sh[GRAD_TPB / 32];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w4 = items[it];          // (t, op, chunk, chunks of this op)
        const int t = w4.x, k = w4.y;
        if (!ts[t].active) continue;
        const TrajDev& d = tr[t];
        const SuppRec s = load_supp(d.pool, k);
        const uint32_t size = (uint32_t)(d.D >> s.m);
        const uint32_t u0 = (uint32_t)w4.z * GRAD_CHUNK;
        const uint32_t cnt = min((uint32_t)GRAD_CHUNK, size - u0);
        const T c0 = sizeof(T) == 4 ? (T)d.pool.fc0f[k] : (T)d.pool.fc0d[k];
        double v;
        if constexpr (sizeof(T) == 4)
            v = grad_item<T>(s, c0, d.w32, static_cast<const V*>(d.psi), u0, cnt, sh);
        else
            v = grad_item<T>(s, c0, d.w, static_cast<const V*>(d.psi), u0, cnt, sh);
        // the select launch sums the op's chunks (grad_item ends with a
        // barrier, so sh is free again)
        if (threadIdx.x == 0) d.gpart[it - d.gbase] = v;
    }
}

// Numbers the energy items of the active trajectories for the next energy
// launch (n + 1 entries, as active_traj reads them), in one block: thread i
// owns a run of consecutive trajectories.
__device__ void number_active(const TrajDev* tr, const TrajState* ts, int n, int2* pre) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = (n + blockDim.x - 1) / blockDim.x;
    const int a = min(n, (int)threadIdx.x * c), b = min(n, a + c);
    int own = 0;
    for (int t = a; t < b; ++t)
        if (__ldcg(&ts[t].active)) own += tr[t].ecnt;
    int inc = own;                             // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < wid) before += wsum[w];
        total += wsum[w];
    }
    int e = before + inc - own;                // exclusive prefix of this thread's run
    for (int t = a; t < b; ++t) {
        const TrajDev& d = tr[t];
        pre[t] = make_int2(e, d.eoff - e);
        if (__ldcg(&ts[t].active)) e += d.ecnt;
    }
    if (threadIdx.x == 0) pre[n] = make_int2(total, 0);
}

// One warp per trajectory: each gradient from its op's chunk partials
// (Eq. (5), divided by <psi|psi>), then choice, convergence, angle, record,
// and the iteration counter advanced.  The last block to finish numbers the
// next iteration's energy items.
__global__ void kb_select(const TrajDev* tr, TrajState* ts, int n, double eps, int prec, int2* pre,
                          unsigned* ticket) {
    __shared__ bool last;
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t < n) {
        TrajState& s = ts[t];
        if (!s.active) {
            if (lane == 0) s.do_update = 0;
        } else {
            const TrajDev& d = tr[t];
            const double inv = 1.0 / s.e_den;
            double m = 0.0;
            // the lane's ops k = lane + 32 j, four at a time so that their
            // bounds and first chunks load together; each op's chunks are
            // summed in item order (every op has at least one)
            for (int k0 = lane; k0 < d.M; k0 += 32 * SEL_U) {
                int f[SEL_U], e[SEL_U];
                double acc[SEL_U];
#pragma unroll
                for (int u = 0; u < SEL_U; ++u) {
                    const int k = k0 + 32 * u;
                    f[u] = k < d.M ? d.gfirst[k] : 0;
                    e[u] = k < d.M ? d.gfirst[k + 1] : 0;
                }
#pragma unroll
                for (int u = 0; u < SEL_U; ++u) acc[u] = k0 + 32 * u < d.M ? d.gpart[f[u]] : 0.0;
#pragma unroll
                for (int u = 0; u < SEL_U; ++u) {
                    const int k = k0 + 32 * u;
                    if (k < d.M) {
                        for (int i = f[u] + 1; i < e[u]; ++i) acc[u] += d.gpart[i];
                        const double g = 2.0 * acc[u] * inv;
                        d.g[k] = g;            // read back below by this lane only
                        m = fmax(m, fabs(g));
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            const double tau = prec == TQ_C128 ? 1e-9 * fmax(1.0, m) : 1e-5;
            int best = d.M;
            for (int k = lane; k < d.M; k += 32)
                if (fabs(d.g[k]) >= m - tau && k < best) best = k;
            for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
            if (lane == 0) {
                const int it = s.iter;
                s.selected = best < d.M ? best : 0;
                s.max_grad = m;
                s.converged = m < eps ? 1 : 0;
                s.theta = s.converged ? 0.0 : d.thetas[it];
                s.do_update = !s.converged;
                if (s.do_update) s.updated = 1;
                d.res_e[it] = s.energy;
                d.res_g[it] = m;
                d.res_sel[it] = s.selected;
                d.res_th[it] = s.theta;
                s.iter = it + 1;
                s.active = (!s.converged && it + 1 < d.len) ? 1 : 0;
                __threadfence();
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    number_active(tr, ts, n, pre);
    if (threadIdx.x == 0) *ticket = 0u;
}

template <typename T>
__global__ void __launch_bounds__(PAIR_BS)
kb_pair(const TrajDev* tr, const TrajState* ts, const int4* items, int n_items, double* npart) {
    constexpr int NW = PAIR_BS / 32;
    const int warp = threadIdx.x >> 5;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w4 = items[it];
        const int t = w4.x, tl = w4.y;
        const TrajState& s = ts[t];
        if (!s.do_update) continue;
        const TrajDev& d = tr[t];
        const OpRec<T> op = make_rec<T>(d.pool, s.selected);
        const T tp = pair_tile<T, BT_UPT>(op, s.theta, static_cast<typename C2<T>::type*>(d.psi),
                                          (uint32_t)tl, (uint32_t)(d.D >> 2));
        store_partial(npart + d.nbase + (long long)tl * NW + warp, tp);
    }
}

// The final renormalisation, items (t, chunk of rows).  ||psi||^2 is the
// sum of the norm partials of the trajectory's last update (a trajectory's
// slots are written only by its own updates).
template <typename T>
__global__ void kb_scale(const TrajDev* tr, const TrajState* ts, const int4* items, int n_items,
                         const double* npart) {
    using V = typename C2<T>::type;
    __shared__ double sh[256 / 32];
    __shared__ double norm2;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int4 w = items[it];
        const TrajState& s = ts[w.x];
        if (!s.updated) continue;           // never updated: still the normalised reference state
        const TrajDev& d = tr[w.x];
        double acc[1] = {0.0};
        const int slots = d.pcnt * (PAIR_BS / 32);
        for (int i = threadIdx.x; i < slots; i += blockDim.x) {
            const double* slot = npart + d.nbase + i;
            if constexpr (sizeof(T) == 4) {
                const float2 hl = *reinterpret_cast<const float2*>(slot);
                acc[0] += (double)hl.x + (double)hl.y;
            } else {
                acc[0] += *slot;
            }
        }
        block_sum<1>(acc, sh);
        if (threadIdx.x == 0) norm2 = acc[0];
        __syncthreads();
        // the factor is formed in float64 and applied in the state's precision
        const T sc = (T)(1.0 / sqrt(norm2));
        __syncthreads();                    // norm2 is rewritten by the next item
        V* psi = static_cast<V*>(d.psi) + w.y;
        // SCALE_U loads in flight per thread before their stores
        for (int i0 = threadIdx.x; i0 < w.z; i0 += SCALE_U * blockDim.x) {
            V v[SCALE_U];
#pragma unroll
            for (int u = 0; u < SCALE_U; ++u) {
                const int i = i0 + u * blockDim.x;
                v[u] = i < w.z ? psi[i] : V{};
            }
#pragma unroll
            for (int u = 0; u < SCALE_U; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < w.z) {
                    v[u].x *= sc;
                    v[u].y *= sc;
                    psi[i] = v[u];
                }
            }
        }
    }
}

template <typename K>
int resident_grid(K kernel, int bs, int sms) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bs, 0);
    return std::max(1, per) * sms;
}

}  // namespace
}  // namespace tq

using namespace tq;

struct tq_batch {
    int device = 0;     // the context's device, kept for freeing after the context
    tq_ctx* ctx = nullptr;
    int n = 0, prec = 0, max_len = 0, lpr = 32;
    double eps = 0.0;
    std::vector<TrajDev> td;
    TrajDev* d_td = nullptr;
    TrajState* d_ts = nullptr;
    int4 *eitems = nullptr, *gitems = nullptr, *pitems = nullptr, *sitems = nullptr;
    int n_e = 0, n_g = 0, n_p = 0, n_s = 0;
    double* epart = nullptr;
    double* npart = nullptr;
    int2* pre = nullptr;            // the active trajectories' energy items, numbered (n + 1 entries)
    int2* pre0 = nullptr;           // the same before the first iteration
    unsigned* nticket = nullptr;    // blocks of the select launch done
    std::vector<void*> allocs;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_lpr = -1;
    int grid_e[4] = {1, 1, 1, 1};   // energy, per lanes-per-row 4, 8, 16, 32
    int grid_x = 1;                 // energy over the XOR-ELL layout
    int grid_g = 1, grid_p = 1;
};

namespace {

template <typename T>
T* dalloc(tq_batch* b, size_t n) {
    T* p = static_cast<T*>(dev_alloc(std::max<size_t>(1, n) * sizeof(T)));
    b->allocs.push_back(p);
    return p;
}

template <typename T>
T* dupload(tq_batch* b, const std::vector<T>& v) {
    T* p = dalloc<T>(b, v.size());
    if (!v.empty()) TQ_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

template <typename T, typename VT>
int launch_energy(tq_batch* b, cudaStream_t s) {
    switch (b->lpr) {
        case TQ_SPMV_XELL:
            kbx_energy<T, VT><<<b->grid_x, BT_BS, 0, s>>>(b->d_td, b->d_ts, b->eitems, b->pre, b->n, b->epart);
            break;
        case 4: kb_energy<T, VT, 4><<<b->grid_e[0], BT_BS, 0, s>>>(b->d_td, b->d_ts, b->eitems, b->pre, b->n, b->epart); break;
        case 8: kb_energy<T, VT, 8><<<b->grid_e[1], BT_BS, 0, s>>>(b->d_td, b->d_ts, b->eitems, b->pre, b->n, b->epart); break;
        case 16: kb_energy<T, VT, 16><<<b->grid_e[2], BT_BS, 0, s>>>(b->d_td, b->d_ts, b->eitems, b->pre, b->n, b->epart); break;
        default: kb_energy<T, VT, 32><<<b->grid_e[3], BT_BS, 0, s>>>(b->d_td, b->d_ts, b->eitems, b->pre, b->n, b->epart); break;
    }
    return 1;
}

// Persistent grid sizes, computed once (no runtime query inside a capture).
template <typename T, typename VT>
void compute_grids(tq_batch* b) {
    const int sms = b->ctx->sm_count;
    b->grid_e[0] = std::min(b->n_e, resident_grid(kb_energy<T, VT, 4>, BT_BS, sms));
    b->grid_e[1] = std::min(b->n_e, resident_grid(kb_energy<T, VT, 8>, BT_BS, sms));
    b->grid_e[2] = std::min(b->n_e, resident_grid(kb_energy<T, VT, 16>, BT_BS, sms));
    b->grid_e[3] = std::min(b->n_e, resident_grid(kb_energy<T, VT, 32>, BT_BS, sms));
    b->grid_x = std::min(b->n_e, resident_grid(kbx_energy<T, VT>, BT_BS, sms));
    b->grid_g = std::min(b->n_g, resident_grid(kb_grad<T>, GRAD_TPB, sms));
    b->grid_p = std::min(b->n_p, resident_grid(kb_pair<T>, PAIR_BS, sms));
}

template <typename T>
int launch_reset(tq_batch* b, cudaStream_t s) {
    const int grid = std::min(b->n_s, b->ctx->sm_count * 8);
    kb_reset<T><<<std::max(1, grid), 256, 0, s>>>(b->d_td, b->d_ts, b->sitems, b->n_s);
    return 1;
}

// One iteration of every trajectory: four launches.
template <typename T, typename VT>
void enqueue_iteration(tq_batch* b, cudaStream_t s) {
    tq_ctx* c = b->ctx;
    launch(c, "batch_energy", s, [&] { return launch_energy<T, VT>(b, s); });
    launch(c, "batch_gradients", s, [&] {
        kb_grad<T><<<b->grid_g, GRAD_TPB, 0, s>>>(b->d_td, b->d_ts, b->gitems, b->n_g);
        return 1;
    });
    launch(c, "batch_select", s, [&] {
        kb_select<<<(b->n * 32 + 255) / 256, 256, 0, s>>>(b->d_td, b->d_ts, b->n, b->eps, b->prec, b->pre,
                                                          b->nticket);
        return 1;
    });
    launch(c, "batch_taylor5_pair", s, [&] {
        kb_pair<T><<<b->grid_p, PAIR_BS, 0, s>>>(b->d_td, b->d_ts, b->pitems, b->n_p, b->npart);
        return 1;
    });
}

template <typename T>
void enqueue_scale(tq_batch* b, cudaStream_t s) {
    launch(b->ctx, "batch_scale", s, [&] {
        kb_scale<T><<<std::min(b->n_s, b->ctx->sm_count * 8), 256, 0, s>>>(b->d_td, b->d_ts, b->sitems, b->n_s,
                                                                           b->npart);
        return 1;
    });
}

// Launches of one run after the reset.
long long run_launches(const tq_batch* b) { return b->max_len > 0 ? 4ll * b->max_len + 1 : 0; }

void enqueue_all(tq_batch* b, cudaStream_t s) {
    for (int i = 0; i < b->max_len; ++i) {
        if (b->prec == TQ_C128) enqueue_iteration<double, double>(b, s);
        else enqueue_iteration<float, float>(b, s);
    }
    if (b->max_len > 0) {
        if (b->prec == TQ_C128) enqueue_scale<double>(b, s);
        else enqueue_scale<float>(b, s);
    }
}

void reset(tq_batch* b, cudaStream_t s) {
    TQ_CUDA(cudaMemcpyAsync(b->pre, b->pre0, (size_t)(b->n + 1) * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    launch(b->ctx, "batch_reset", s, [&] {
        return b->prec == TQ_C128 ? launch_reset<double>(b, s) : launch_reset<float>(b, s);
    });
}

void drop_graph(tq_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_lpr = -1;
}

}  // namespace

extern "C" int tq_batch_create(tq_ctx* c, int n_traj, tq_ham* const* hams, tq_pool* const* pools,
                               const int* n_electrons, const int* mappings, const int* lengths,
                               const double* thetas, double eps, tq_batch** out) {
    API_BEGIN
    TQ_REQUIRE(c && hams && pools && n_electrons && mappings && lengths && thetas && out, "null argument");
    for (int i = 0; i < n_traj; ++i)
        TQ_REQUIRE(hams[i] && pools[i] && !hams[i]->sector && !pools[i]->sector,
                   "the trajectory batch works in the full space");
    TQ_REQUIRE(n_traj >= 1, "n_traj must be >= 1");
    TQ_REQUIRE(std::isfinite(eps) && eps >= 0.0, "eps must be finite and >= 0");
    *out = nullptr;
    TQ_CUDA(cudaSetDevice(c->device));
    auto* b = new tq_batch();
    try {
        b->ctx = c;
        b->device = c->device;
        b->n = n_traj;
        b->eps = eps;
        b->prec = hams[0]->prec;
        std::vector<int4> ei, gi, pi, si;
        long long nslots = 0, toff = 0;
        for (int t = 0; t < n_traj; ++t) {
            const tq_ham* h = hams[t];
            const tq_pool* p = pools[t];
            TQ_REQUIRE(h && p, "null Hamiltonian or pool handle");
            TQ_REQUIRE(h->prec == b->prec, "all Hamiltonians must share one precision");
            TQ_REQUIRE(h->nq == p->nq, "Hamiltonian and pool qubit counts differ");
            TQ_REQUIRE(lengths[t] >= 0, "negative trajectory length");
            for (int i = 0; i < lengths[t]; ++i)
                TQ_REQUIRE(std::isfinite(thetas[toff + i]), "non-finite angle");
            TrajDev d{};
            d.nq = h->nq;
            d.D = h->D;
            d.M = p->M;
            d.len = lengths[t];
            d.hf = (long long)hf_index(h->nq, n_electrons[t], mappings[t]);
            d.diag = h->view.diag;
            d.rowptr = h->view.rowptr;
            d.col = h->view.col;
            d.val = h->view.val;
            d.xptr = h->view.xptr;
            d.xmask = h->view.xmask;
            d.xval = h->view.xval;
            d.pool = p->view;
            d.chunk = 0;
            d.nch = 0;
            d.eoff = (int)ei.size();
            for (long long r = 0; r < d.D; r += ROWS_PER_ITEM)
                ei.push_back(make_int4(t, (int)r, (int)std::min<long long>(ROWS_PER_ITEM, d.D - r), 0));
            d.ecnt = (int)ei.size() - d.eoff;
            d.gbase = (int)gi.size();
            // the pool's own item table: op k's chunks are items gf[k] .. gf[k + 1] - 1
            std::vector<int> gf((size_t)d.M + 1);
            TQ_CUDA(cudaMemcpy(gf.data(), p->view.gfirst, gf.size() * sizeof(int), cudaMemcpyDeviceToHost));
            for (int k = 0; k < d.M; ++k) {
                const int nchunks = gf[k + 1] - gf[k];
                TQ_REQUIRE(gf[k] == (int)gi.size() - d.gbase && nchunks >= 1, "pool gradient table is inconsistent");
                for (int ch = 0; ch < nchunks; ++ch) gi.push_back(make_int4(t, k, ch, nchunks));
            }
            const int n_gitems_t = (int)gi.size() - d.gbase;
            const long long units = d.D >> 2;
            d.pcnt = (int)((units + PAIR_BS * BT_UPT - 1) / (PAIR_BS * BT_UPT));
            for (int tl = 0; tl < d.pcnt; ++tl) pi.push_back(make_int4(t, tl, 0, 0));
            d.nbase = nslots;
            nslots += (long long)d.pcnt * (PAIR_BS / 32);
            for (long long r = 0; r < d.D; r += 4096)
                si.push_back(make_int4(t, (int)r, (int)std::min<long long>(4096, d.D - r), 0));
            const size_t es = b->prec == TQ_C128 ? 16 : 8;
            d.psi = dalloc<unsigned char>(b, (size_t)d.D * es);
            if (b->prec == TQ_C128) d.w = dalloc<double2>(b, (size_t)d.D);
            else d.w32 = dalloc<float2>(b, (size_t)d.D);
            d.thetas = dupload(b, std::vector<double>(thetas + toff, thetas + toff + d.len));
            toff += d.len;
            d.g = dalloc<double>(b, d.M);
            d.gpart = dalloc<double>(b, (size_t)n_gitems_t);
            d.gfirst = p->view.gfirst;
            d.res_e = dalloc<double>(b, std::max(1, d.len));
            d.res_g = dalloc<double>(b, std::max(1, d.len));
            d.res_th = dalloc<double>(b, std::max(1, d.len));
            d.res_sel = dalloc<int>(b, std::max(1, d.len));
            b->max_len = std::max(b->max_len, d.len);
            b->td.push_back(d);
        }
        b->eitems = dupload(b, ei);
        b->gitems = dupload(b, gi);
        b->pitems = dupload(b, pi);
        b->sitems = dupload(b, si);
        b->n_e = (int)ei.size();
        b->n_g = (int)gi.size();
        b->n_p = (int)pi.size();
        b->n_s = (int)si.size();
        b->epart = dalloc<double>(b, 2 * ei.size());
        b->npart = dalloc<double>(b, (size_t)nslots);
        {
            // before the first iteration the active trajectories are those of length > 0
            std::vector<int2> p0((size_t)n_traj + 1);
            int e = 0;
            for (int t = 0; t < n_traj; ++t) {
                const TrajDev& d = b->td[t];
                p0[t] = make_int2(e, d.eoff - e);
                if (d.len > 0) e += d.ecnt;
            }
            p0[n_traj] = make_int2(e, 0);
            b->pre0 = dupload(b, p0);
            b->pre = dupload(b, p0);
            b->nticket = dalloc<unsigned>(b, 1);
            TQ_CUDA(cudaMemset(b->nticket, 0, sizeof(unsigned)));
        }
        b->d_td = dupload(b, b->td);
        b->d_ts = dalloc<TrajState>(b, n_traj);
        TQ_CUDA(cudaMemset(b->d_ts, 0, n_traj * sizeof(TrajState)));
        TQ_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        if (b->prec == TQ_C128) compute_grids<double, double>(b);
        else compute_grids<float, float>(b);
    } catch (...) {
        tq_batch_free(b);
        throw;
    }
    *out = b;
    API_END
}

extern "C" int tq_batch_set_schedule(tq_batch* b, int lanes_per_row) {
    API_BEGIN
    TQ_REQUIRE(b != nullptr, "batch is null");
    TQ_REQUIRE(lanes_per_row == TQ_SPMV_XELL || lanes_per_row == 4 || lanes_per_row == 8 || lanes_per_row == 16 ||
                   lanes_per_row == 32,
               "lanes_per_row must be TQ_SPMV_XELL, 4, 8, 16 or 32");
    b->lpr = lanes_per_row;
    API_END
}

extern "C" int tq_batch_autotune(tq_batch* b, int* lanes_per_row, double* best_ms) {
    API_BEGIN
    TQ_REQUIRE(b != nullptr, "batch is null");
    TQ_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = b->cap;
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    int best = b->lpr;
    float best_t = 1e30f;
    for (int l : {(int)TQ_SPMV_XELL, 4, 8, 16, 32}) {
        b->lpr = l;
        reset(b, s);
        auto one = [&] {
            launch(b->ctx, "autotune_batch_energy", s, [&] {
                return b->prec == TQ_C128 ? launch_energy<double, double>(b, s) : launch_energy<float, float>(b, s);
            });
        };
        one();
        TQ_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) one();
        TQ_CUDA(cudaEventRecord(e1, s));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (ms < best_t) {
            best_t = ms;
            best = l;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->lpr = best;
    if (lanes_per_row) *lanes_per_row = best;
    if (best_ms) *best_ms = best_t;
    API_END
}

extern "C" int tq_batch_run(tq_batch* b, int use_graph, void* stream) {
    API_BEGIN
    TQ_REQUIRE(b != nullptr, "batch is null");
    TQ_CUDA(cudaSetDevice(b->ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    reset(b, s);
    if (!use_graph) {
        enqueue_all(b, s);
        return TQ_OK;
    }
    if (!b->exec || b->graph_lpr != b->lpr) {
        drop_graph(b);
        // capture on the batch's own stream, after the reset so that no
        // host-side check inside a launch sees a capturing stream
        TQ_CUDA(cudaStreamSynchronize(s));
        const int tracing = b->ctx->tracing;
        b->ctx->tracing = 0;   // no event records inside the graph
        TQ_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_all(b, b->cap);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(b->cap, &g);
            if (g) cudaGraphDestroy(g);
            b->ctx->tracing = tracing;
            throw;
        }
        b->ctx->tracing = tracing;
        TQ_CUDA(cudaStreamEndCapture(b->cap, &b->graph));
        TQ_CUDA(cudaGraphInstantiate(&b->exec, b->graph, 0));
        b->graph_lpr = b->lpr;
        b->ctx->launches -= run_launches(b);   // counted again at each replay below
    }
    {
        Traced t(b->ctx, "batch_graph", s);
        TQ_CUDA(cudaGraphLaunch(b->exec, s));
    }
    b->ctx->launches += run_launches(b);
    API_END
}

extern "C" int tq_batch_results(const tq_batch* b, int* n_iter, int* converged, double* energy,
                                double* max_grad, int* selected, double* theta) {
    API_BEGIN
    TQ_REQUIRE(b != nullptr, "batch is null");
    TQ_CUDA(cudaSetDevice(b->ctx->device));
    TQ_CUDA(cudaDeviceSynchronize());
    std::vector<TrajState> hs(b->n);
    TQ_CUDA(cudaMemcpy(hs.data(), b->d_ts, b->n * sizeof(TrajState), cudaMemcpyDeviceToHost));
    long long off = 0;
    for (int t = 0; t < b->n; ++t) {
        const TrajDev& d = b->td[t];
        if (n_iter) n_iter[t] = hs[t].iter;
        if (converged) converged[t] = hs[t].converged;
        const size_t L = (size_t)d.len;
        if (L) {
            if (energy) TQ_CUDA(cudaMemcpy(energy + off, d.res_e, L * sizeof(double), cudaMemcpyDeviceToHost));
            if (max_grad) TQ_CUDA(cudaMemcpy(max_grad + off, d.res_g, L * sizeof(double), cudaMemcpyDeviceToHost));
            if (selected) TQ_CUDA(cudaMemcpy(selected + off, d.res_sel, L * sizeof(int), cudaMemcpyDeviceToHost));
            if (theta) TQ_CUDA(cudaMemcpy(theta + off, d.res_th, L * sizeof(double), cudaMemcpyDeviceToHost));
        }
        off += d.len;
    }
    API_END
}

extern "C" int tq_batch_state(const tq_batch* b, int t, void** dev_ptr, int* n_qubits) {
    API_BEGIN
    TQ_REQUIRE(b != nullptr, "batch is null");
    TQ_REQUIRE(t >= 0 && t < b->n, "trajectory index out of range");
    if (dev_ptr) *dev_ptr = b->td[t].psi;
    if (n_qubits) *n_qubits = b->td[t].nq;
    API_END
}

extern "C" int tq_batch_free(tq_batch* b) {
    if (!b) return TQ_OK;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    drop_graph(b);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
    (void)cudaGetLastError();   // a failure while freeing is not reported to later calls
    return TQ_OK;
}
