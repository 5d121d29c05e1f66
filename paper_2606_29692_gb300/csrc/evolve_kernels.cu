// Fifth-order Taylor state update, Sec. III-C, Eqs. (6)-(8):
//   v_0 = psi, v_k = A v_{k-1} (k = 1..5),
//   psi' = psi + theta v_1 + theta^2/2 v_2 + theta^3/6 v_3 + theta^4/24 v_4
//              + theta^5/120 v_5.
//
// Pair path (pool generators).  A pool generator has one X-mask x, so row r
// of A has its only candidate column at r ^ x, and the two-element set
// {r, r ^ x} is closed under A.  Each thread therefore owns whole pairs: it
// loads psi[r] and psi[r ^ x] once, runs the five products and the running
// sum in registers, and stores both once.  Pairs are enumerated by
// inserting a zero at the highest set bit hb of x; two consecutive
// representatives r0, r0 + 1 and their partners form two aligned
// two-element vectors, so every load and store is a 16-byte (complex64) or
// 2 x 16-byte (complex128) access, coalesced across the warp.  Values of A
// come from the generator's factored sign form (no matrix bytes are read).
// The float64 squared norm of psi' is reduced per tile in the same pass.
//
// CSR path (any operator).  The state is staged in shared memory, split
// over the CTAs of a thread-block cluster; the gather of v_{k-1} reads
// peer CTAs' shared memory through the cluster mapping, each product is
// followed by a cluster barrier, and the running sum lives in registers.
// Global memory is touched by the initial load, the CSR, and the final
// store only.  The float64 norm is reduced across the cluster and applied
// before the store when renormalisation is asked for.
#include "dev.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace tq {

namespace {

constexpr int PAIR_BS = 256;

__device__ __forceinline__ void load2(const float2* p, uint32_t i, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p + i);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void store2(float2* p, uint32_t i, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p + i) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void load2(const double2* p, uint32_t i, double2& a, double2& b) {
    a = p[i];
    b = p[i + 1];
}
__device__ __forceinline__ void store2(double2* p, uint32_t i, double2 a, double2 b) {
    p[i] = a;
    p[i + 1] = b;
}

template <typename V, typename T>
__device__ __forceinline__ V scal(T s, V v) {
    V o;
    o.x = s * v.x;
    o.y = s * v.y;
    return o;
}
template <typename V, typename T>
__device__ __forceinline__ void axpy(V& acc, T c, V v) {
    acc.x = fma(c, v.x, acc.x);
    acc.y = fma(c, v.y, acc.y);
}

// Five chained products on one closed pair (r, q = r ^ x) with
// s_r = A[r][q], s_q = A[q][r]; returns the accumulated pair in (ar, aq).
template <typename V, typename T>
__device__ __forceinline__ void chain_pair(T s_r, T s_q, const T (&cf)[6], V& ar, V& aq) {
    V vr = ar, vq = aq;
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        const V nr = scal(s_r, vq);   // (A v)[r] = A[r][q] v[q]
        const V nq = scal(s_q, vr);   // (A v)[q] = A[q][r] v[r]
        vr = nr;
        vq = nq;
        axpy(ar, cf[k], vr);
        axpy(aq, cf[k], vq);
    }
}

// complex64: the same chain on Blackwell's packed float32x2 pipe (one
// instruction per complex multiply-by-real or multiply-add, rounding as the
// scalar form).
__device__ __forceinline__ void chain_pair(float s_r, float s_q, const float (&cf)[6], float2& ar,
                                           float2& aq) {
    const float2 sr = make_float2(s_r, s_r), sq = make_float2(s_q, s_q);
    float2 vr = ar, vq = aq;
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        const float2 nr = __fmul2_rn(sr, vq);
        const float2 nq = __fmul2_rn(sq, vr);
        vr = nr;
        vq = nq;
        const float2 c = make_float2(cf[k], cf[k]);
        ar = __ffma2_rn(c, vr, ar);
        aq = __ffma2_rn(c, vq, aq);
    }
}

template <typename T>
__device__ __forceinline__ void taylor_coefs(double theta, T (&cf)[6]) {
    double c = 1.0;
    cf[0] = T(1);
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        c = c * theta / (double)k;
        cf[k] = (T)c;
    }
}

// theta^k / k! for k = 0..5 in the kernel's own precision: powers by
// multiplication and constant reciprocal factorials (no division).  The
// complex64 path stays entirely on the float32 pipes: float64 issues at
// about 1/57 of the float32 rate on this part.
template <typename T>
__device__ __forceinline__ void taylor_coefs_fast(double theta, T (&cf)[6]) {
    const T t = (T)theta;
    const T t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    cf[0] = T(1);
    cf[1] = t;
    cf[2] = t2 * T(0.5);
    cf[3] = t3 * T(1.0 / 6.0);
    cf[4] = t4 * T(1.0 / 24.0);
    cf[5] = t5 * T(1.0 / 120.0);
}

// Per-warp norm partial: float64 sum for complex128; for complex64 a
// TwoSum-compensated float32 warp sum stored as a (hi, lo) float pair in
// the 8-byte slot and widened to float64 by the reduction kernel.
__device__ __forceinline__ void store_partial(double* slot, double v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) *slot = v;
}
__device__ __forceinline__ void store_partial(double* slot, float v) {
    float hi = v, lo = 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, lo, o);
        float sum, err;
        two_sum(hi, oh, sum, err);
        hi = sum;
        lo = lo + ol + err;
    }
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2*>(slot) = make_float2(hi, lo);
}
__device__ __forceinline__ void store_nan_partial(double* slot, double) {
    if ((threadIdx.x & 31) == 0) *slot = __longlong_as_double(0x7ff8000000000000ll);
}
__device__ __forceinline__ void store_nan_partial(double* slot, float) {
    if ((threadIdx.x & 31) == 0) *reinterpret_cast<float2*>(slot) = make_float2(__int_as_float(0x7fc00000), 0.f);
}

// One pool generator as staged in shared memory: X-mask, the factored sign
// form (A[r][r^x] = c0 (-1)^{parity(col & z0)} if parity(col & d_i) == t_i
// for all i, else 0, with col = r ^ x), and the parities of
// {0, 1, x, x ^ 1} against (d0, d1, d2, z0) so that one set of popcounts at
// r0 gives the values of all four rows of a unit.
template <typename T>
struct OpRec {
    uint32_t x, z0, d0, d1, d2;
    int t;        // target parities (bits 0..2)
    int dcode;    // 4 x 4-bit parity codes of delta in {0, 1, x, x^1}
    T c0;
};

template <typename T>
__device__ __forceinline__ OpRec<T> make_rec(const PoolView& p, int k) {
    OpRec<T> o;
    o.x = p.x[k];
    o.z0 = p.fz0[k];
    o.d0 = p.fd[3 * k];
    o.d1 = p.fd[3 * k + 1];
    o.d2 = p.fd[3 * k + 2];
    o.t = p.ft[k];
    o.c0 = sizeof(T) == 4 ? (T)p.fc0f[k] : (T)p.fc0d[k];
    const uint32_t dl[4] = {0u, 1u, o.x, o.x ^ 1u};
    int code = 0;
    for (int j = 0; j < 4; ++j) {
        const uint32_t d = dl[j];
        const int c = parity32(d & o.d0) | (parity32(d & o.d1) << 1) | (parity32(d & o.d2) << 2) |
                      (parity32(d & o.z0) << 3);
        code |= c << (4 * j);
    }
    o.dcode = code;
    return o;
}

// Value A[row][col] given the parity code of col.
template <typename T>
__device__ __forceinline__ T rec_value(const OpRec<T>& o, int code) {
    return (code & 7) != o.t ? T(0) : ((code & 8) ? -o.c0 : o.c0);
}

template <typename T>
__device__ __forceinline__ int base_code(const OpRec<T>& o, uint32_t r) {
    return parity32(r & o.d0) | (parity32(r & o.d1) << 1) | (parity32(r & o.d2) << 2) |
           (parity32(r & o.z0) << 3);
}

template <typename T, int UPT>
__global__ void __launch_bounds__(PAIR_BS)
k_taylor5_pair(PoolView p, int n_states, typename C2<T>::type* psi, const int* kk,
               const double* th, int k_imm, double th_imm, double* partials,
               int tiles_per_state, const DevStep* gate) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    OpRec<T>* ops = reinterpret_cast<OpRec<T>*>(smem_raw);
    if (gate && gate->converged) return;
    // the vectorised pool layout, staged once per CTA
    for (int i = threadIdx.x; i < p.M; i += blockDim.x) ops[i] = make_rec<T>(p, i);
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    constexpr int NW = PAIR_BS / 32;
    constexpr int TU = PAIR_BS * UPT;           // units per tile
    const long long D = 1ll << p.nq;
    const uint32_t units = (uint32_t)(D >> 2);
    const unsigned total = (unsigned)n_states * (unsigned)tiles_per_state;
    const unsigned tps = (unsigned)tiles_per_state;
    unsigned tile = blockIdx.x;
    int b = (int)(tile / tps);
    int k = tile < total ? (kk ? kk[b] : k_imm) : 0;
    double theta = tile < total ? (th ? th[b] : th_imm) : 0.0;
    for (; tile < total; ) {
        const int tl = (int)(tile - (unsigned)b * tps);
        // prefetch the next tile's op index and angle
        const unsigned ntile = tile + gridDim.x;
        const int nb = (int)(ntile / tps);
        int nk = 0;
        double nth = 0.0;
        if (ntile < total) {
            nk = kk ? kk[nb] : k_imm;
            nth = th ? th[nb] : th_imm;
        }
        double* slot = partials + (size_t)tile * NW + warp;
        if (k < 0 || k >= p.M) {
            // invalid op index from device memory: leave the state untouched
            // and poison its norm so the caller sees it
            store_nan_partial(slot, T(0));
        } else {
            const OpRec<T> op = ops[k];
            const uint32_t x = op.x;
            const int hb = 31 - __clz(x);
            T cf[6];
            taylor_coefs_fast<T>(theta, cf);
            V* base = psi + (long long)b * D;
            V e0[UPT], e1[UPT], f0[UPT], f1[UPT];
            uint32_t r0s[UPT];
            bool ok[UPT];
#pragma unroll
            for (int j = 0; j < UPT; ++j) {
                const uint32_t u = (uint32_t)tl * TU + j * PAIR_BS + threadIdx.x;
                ok[j] = u < units;
                if (!ok[j]) continue;
                if (hb > 0) {
                    const uint32_t r0 = insert_zero(2u * u, hb);
                    r0s[j] = r0;
                    load2(base, r0, e0[j], e1[j]);
                    load2(base, (r0 ^ x) & ~1u, f0[j], f1[j]);
                } else {
                    const uint32_t r0 = 4u * u;
                    r0s[j] = r0;
                    load2(base, r0, e0[j], f0[j]);
                    load2(base, r0 + 2u, e1[j], f1[j]);
                }
            }
            T tpart = T(0);
#pragma unroll
            for (int j = 0; j < UPT; ++j) {
                if (!ok[j]) continue;
                const uint32_t r0 = r0s[j];
                if (hb > 0) {
                    // rows r0, r0+1 and partners q0 = r0^x, q0^1; their columns
                    // are r0 ^ {x, x^1, 0, 1}
                    const uint32_t q0 = r0 ^ x;
                    const int bc = base_code(op, r0);
                    const T s_r0 = rec_value(op, bc ^ ((op.dcode >> 8) & 15));    // col q0
                    const T s_r1 = rec_value(op, bc ^ ((op.dcode >> 12) & 15));   // col q0^1
                    const T s_q0 = rec_value(op, bc ^ (op.dcode & 15));           // col r0
                    const T s_q1 = rec_value(op, bc ^ ((op.dcode >> 4) & 15));    // col r0+1
                    V a0 = e0[j], a1 = e1[j];
                    V b0 = (q0 & 1u) ? f1[j] : f0[j];   // psi[q0]
                    V b1 = (q0 & 1u) ? f0[j] : f1[j];   // psi[q0 ^ 1]
                    chain_pair(s_r0, s_q0, cf, a0, b0);
                    chain_pair(s_r1, s_q1, cf, a1, b1);
                    tpart += a0.x * a0.x + a0.y * a0.y + a1.x * a1.x + a1.y * a1.y;
                    tpart += b0.x * b0.x + b0.y * b0.y + b1.x * b1.x + b1.y * b1.y;
                    store2(base, r0, a0, a1);
                    if (q0 & 1u) store2(base, q0 & ~1u, b1, b0);
                    else store2(base, q0 & ~1u, b0, b1);
                } else {
                    // x == 1: pairs (r0, r0+1) and (r0+2, r0+3)
                    const int b0c = base_code(op, r0), b2c = base_code(op, r0 + 2u);
                    const T s_r0 = rec_value(op, b0c ^ ((op.dcode >> 4) & 15));  // col r0+1
                    const T s_q0 = rec_value(op, b0c);                           // col r0
                    const T s_r1 = rec_value(op, b2c ^ ((op.dcode >> 4) & 15));  // col r0+3
                    const T s_q1 = rec_value(op, b2c);                           // col r0+2
                    chain_pair(s_r0, s_q0, cf, e0[j], f0[j]);
                    chain_pair(s_r1, s_q1, cf, e1[j], f1[j]);
                    tpart += e0[j].x * e0[j].x + e0[j].y * e0[j].y + f0[j].x * f0[j].x + f0[j].y * f0[j].y;
                    tpart += e1[j].x * e1[j].x + e1[j].y * e1[j].y + f1[j].x * f1[j].x + f1[j].y * f1[j].y;
                    store2(base, r0, e0[j], f0[j]);
                    store2(base, r0 + 2u, e1[j], f1[j]);
                }
            }
            store_partial(slot, tpart);
        }
        tile = ntile;
        b = nb;
        k = nk;
        theta = nth;
    }
}

// One warp per state: fixed-order float64 sum of the state's partials
// (float64 values for complex128; (hi, lo) float pairs for complex64).
template <bool PAIRS>
__global__ void k_norm_reduce(const double* partials, int n_states, int tiles,
                              double* norm2_out, double* step_norm2) {
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n_states) return;
    double s = 0.0;
    for (int t = lane; t < tiles; t += 32) {
        const double* slot = partials + (long long)w * tiles + t;
        if (PAIRS) {
            const float2 hl = *reinterpret_cast<const float2*>(slot);
            s += (double)hl.x + (double)hl.y;
        } else {
            s += *slot;
        }
    }
    s = warp_sum(s);
    if (lane == 0) {
        if (norm2_out) norm2_out[w] = s;
        if (step_norm2 && w == 0) *step_norm2 = s;
    }
}

template <typename V>
__global__ void k_scale(V* psi, long long D, const double* norm2, const DevStep* gate) {
    if (gate && gate->converged) return;
    const double sc = 1.0 / sqrt(*norm2);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride) {
        V v = psi[i];
        v.x = (decltype(v.x))((double)v.x * sc);
        v.y = (decltype(v.y))((double)v.y * sc);
        psi[i] = v;
    }
}

// ---------------------------------------------------------------- CSR path

template <typename T, typename VT, int RPT>
__global__ void __launch_bounds__(1024)
k_taylor5_csr_cluster(int nq, int csize, const int* __restrict__ rowptr,
                      const int* __restrict__ col, const VT* __restrict__ val, double theta,
                      typename C2<T>::type* psi, int renorm, double* norm2_out) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sv = reinterpret_cast<V*>(smem_raw);
    __shared__ double red[32];
    __shared__ double cta_part;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const long long D = 1ll << nq;
    const int per = (int)(D / csize);
    const int shift = 31 - __clz(per);
    const int bs = blockDim.x;
    const int row0 = rank * per;
    for (int i = threadIdx.x; i < per; i += bs) sv[i] = psi[row0 + i];
    T cf[6];
    taylor_coefs<T>(theta, cf);
    V acc[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int i = threadIdx.x + j * bs;
        acc[j] = i < per ? sv[i] : V{};   // written by this thread above
    }
    cl.sync();
    for (int step = 1; step <= 5; ++step) {
        V nv[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int i = threadIdx.x + j * bs;
            V s{};
            if (i < per) {
                const int r = row0 + i;
                const int e1 = rowptr[r + 1];
                for (int e = rowptr[r]; e < e1; ++e) {
                    const int c = col[e];
                    if ((unsigned)c >= (unsigned)D) continue;   // column outside the state
                    const V* src = cl.map_shared_rank(sv, c >> shift);
                    const V v = src[c & (per - 1)];
                    const T a = (T)val[e];
                    s.x = fma(a, v.x, s.x);
                    s.y = fma(a, v.y, s.y);
                }
            }
            nv[j] = s;
        }
        cl.sync();   // every CTA has finished reading v_{k-1}
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int i = threadIdx.x + j * bs;
            if (i < per) {
                sv[i] = nv[j];
                axpy(acc[j], cf[step], nv[j]);
            }
        }
        cl.sync();   // v_k visible cluster-wide
    }
    double part = 0.0;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int i = threadIdx.x + j * bs;
        if (i < per) part += (double)acc[j].x * acc[j].x + (double)acc[j].y * acc[j].y;
    }
    double v[1] = {part};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) cta_part = v[0];
    cl.sync();
    double total = 0.0;
    for (int q = 0; q < csize; ++q) total += *cl.map_shared_rank(&cta_part, q);
    const double sc = renorm ? 1.0 / sqrt(total) : 1.0;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int i = threadIdx.x + j * bs;
        if (i < per) {
            V o;
            o.x = (T)((double)acc[j].x * sc);
            o.y = (T)((double)acc[j].y * sc);
            psi[row0 + i] = o;
        }
    }
    if (rank == 0 && threadIdx.x == 0 && norm2_out) *norm2_out = total;
    cl.sync();   // peers may still read this CTA's shared memory
}

// Unfused fallback for states too large for a cluster: one pass per product,
// v and the running sum in global (L2-resident) buffers.
template <typename T, typename VT>
__global__ void k_csr_step(long long D, const int* __restrict__ rowptr,
                           const int* __restrict__ col, const VT* __restrict__ val,
                           const typename C2<T>::type* vin, typename C2<T>::type* vout,
                           typename C2<T>::type* acc, double coef) {
    using V = typename C2<T>::type;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < D; r += stride) {
        V s{};
        for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) {
            const int c = col[e];
            if ((unsigned long long)c >= (unsigned long long)D) continue;
            const V v = vin[c];
            const T a = (T)val[e];
            s.x = fma(a, v.x, s.x);
            s.y = fma(a, v.y, s.y);
        }
        vout[r] = s;
        V a = acc[r];
        axpy(a, (T)coef, s);
        acc[r] = a;
    }
}

template <typename V>
__global__ void k_copy(const V* a, V* b, long long D) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride) b[i] = a[i];
}

template <typename V>
__global__ void k_norm_partials(const V* a, long long D, double* partials) {
    __shared__ double sh[32];
    double s = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride)
        s += (double)a[i].x * a[i].x + (double)a[i].y * a[i].y;
    double v[1] = {s};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

template <typename V>
__global__ void k_finish(const V* acc, V* psi, long long D, const double* partials, int nparts,
                         int renorm, double* norm2_out) {
    __shared__ double total_sh;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nparts; ++i) t += partials[i];
        total_sh = t;
        if (blockIdx.x == 0 && norm2_out) *norm2_out = t;
    }
    __syncthreads();
    const double sc = renorm ? 1.0 / sqrt(total_sh) : 1.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride) {
        V v = acc[i];
        v.x = (decltype(v.x))((double)v.x * sc);
        v.y = (decltype(v.y))((double)v.y * sc);
        psi[i] = v;
    }
}

template <typename T, typename VT, int RPT>
cudaError_t launch_cluster(int nq, int csize, int bs, const int* rowptr, const int* col,
                           const VT* val, double theta, void* psi, int renorm, double* norm2,
                           cudaStream_t s) {
    using V = typename C2<T>::type;
    auto kern = k_taylor5_csr_cluster<T, VT, RPT>;
    const size_t smem = (size_t)((1ll << nq) / csize) * sizeof(V);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(bs);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (nclusters < 1) return cudaErrorInvalidConfiguration;
    return cudaLaunchKernelEx(&cfg, kern, nq, csize, rowptr, col, val, theta,
                              static_cast<V*>(psi), renorm, norm2);
}

template <typename T, typename VT>
cudaError_t dispatch_cluster(int nq, int csize, const int* rowptr, const int* col,
                             const VT* val, double theta, void* psi, int renorm,
                             double* norm2, cudaStream_t s) {
    const long long per = (1ll << nq) / csize;
    const int bs = (int)(per < 1024 ? (per < 32 ? 32 : per) : 1024);
    const int rpt = (int)((per + bs - 1) / bs);
    // rows per thread: at most 8 (complex64) or 4 (complex128), see the
    // slice size chosen in launch_taylor5_csr
    switch (rpt) {
        case 1: return launch_cluster<T, VT, 1>(nq, csize, bs, rowptr, col, val, theta, psi, renorm, norm2, s);
        case 2: return launch_cluster<T, VT, 2>(nq, csize, bs, rowptr, col, val, theta, psi, renorm, norm2, s);
        case 4: return launch_cluster<T, VT, 4>(nq, csize, bs, rowptr, col, val, theta, psi, renorm, norm2, s);
        case 8:
            if constexpr (sizeof(T) == 4)
                return launch_cluster<T, VT, 8>(nq, csize, bs, rowptr, col, val, theta, psi, renorm, norm2, s);
            return cudaErrorInvalidConfiguration;
        default: return cudaErrorInvalidConfiguration;
    }
}

template <typename T, typename VT>
int run_unfused(int nq, const int* rowptr, const int* col, const VT* val, double theta,
                void* psi, int renorm, double* acc_buf, double* v0_buf, double* v1_buf,
                double* partials, double* norm2, int sms, cudaStream_t s) {
    using V = typename C2<T>::type;
    const long long D = 1ll << nq;
    V* acc = reinterpret_cast<V*>(acc_buf);
    V* v0 = reinterpret_cast<V*>(v0_buf);
    V* v1 = reinterpret_cast<V*>(v1_buf);
    V* p = static_cast<V*>(psi);
    const int bs = 256;
    const int grid = sms * 4;
    k_copy<V><<<grid, bs, 0, s>>>(p, acc, D);
    k_copy<V><<<grid, bs, 0, s>>>(p, v0, D);
    double c = 1.0;
    for (int k = 1; k <= 5; ++k) {
        c = c * theta / (double)k;
        k_csr_step<T, VT><<<grid, bs, 0, s>>>(D, rowptr, col, val, v0, v1, acc, c);
        V* t = v0;
        v0 = v1;
        v1 = t;
    }
    k_norm_partials<V><<<grid, bs, 0, s>>>(acc, D, partials);
    k_finish<V><<<grid, bs, 0, s>>>(acc, p, D, partials, grid, renorm, norm2);
    return 9;
}

}  // namespace

namespace {

// Resident CTAs per SM for the pool table size (cached per 4 KB bucket).
template <typename T, int UPT>
int pair_grid(int M, int sms) {
    static int per_sm[32] = {0};
    const size_t smem = (size_t)M * sizeof(OpRec<T>);
    const int bucket = (int)std::min<size_t>(31, smem / 4096);
    if (per_sm[bucket] == 0) {
        cudaFuncSetAttribute(k_taylor5_pair<T, UPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_taylor5_pair<T, UPT>, PAIR_BS,
                                                      (size_t)(bucket + 1) * 4096);
        per_sm[bucket] = n < 1 ? 1 : n;
    }
    return per_sm[bucket] * sms;
}

template <typename T, int UPT>
int launch_pair(const PoolView& p, int n_states, void* psi, const int* k, const double* theta,
                int k_imm, double theta_imm, double* partials, const DevStep* gate, int sms,
                cudaStream_t s) {
    using V = typename C2<T>::type;
    const long long units = (1ll << p.nq) >> 2;
    const int tiles = (int)((units + PAIR_BS * UPT - 1) / (PAIR_BS * UPT));
    const long long total = (long long)n_states * tiles;
    if (total >= (1ll << 31)) return -1;   // caller splits such batches
    long long grid = pair_grid<T, UPT>(p.M, sms);
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    const size_t smem = (size_t)p.M * sizeof(OpRec<T>);
    k_taylor5_pair<T, UPT><<<(int)grid, PAIR_BS, smem, s>>>(p, n_states, static_cast<V*>(psi), k, theta,
                                                            k_imm, theta_imm, partials, tiles, gate);
    return 1;
}

}  // namespace

int taylor5_pair_parts(int nq, int upt) {
    const long long units = (1ll << nq) >> 2;
    const int tiles = (int)((units + PAIR_BS * upt - 1) / (PAIR_BS * upt));
    return tiles * (PAIR_BS / 32);
}

bool pair_upt_valid(int upt) { return upt == 1 || upt == 2 || upt == 4 || upt == 8; }

namespace {

template <typename T>
int dispatch_pair(int upt, const PoolView& p, int n_states, void* psi, const int* k, const double* theta,
                  int k_imm, double theta_imm, double* partials, const DevStep* gate, int sms,
                  cudaStream_t s) {
    switch (upt) {
        case 1: return launch_pair<T, 1>(p, n_states, psi, k, theta, k_imm, theta_imm, partials, gate, sms, s);
        case 2: return launch_pair<T, 2>(p, n_states, psi, k, theta, k_imm, theta_imm, partials, gate, sms, s);
        case 4: return launch_pair<T, 4>(p, n_states, psi, k, theta, k_imm, theta_imm, partials, gate, sms, s);
        case 8: return launch_pair<T, 8>(p, n_states, psi, k, theta, k_imm, theta_imm, partials, gate, sms, s);
        default: return -1;
    }
}

}  // namespace

int launch_taylor5_pair(const PoolView& p, int n_states, int prec, int upt, void* psi, const int* k,
                        const double* theta, int k_imm, double theta_imm, double* partials, int sms,
                        cudaStream_t s) {
    if (prec == TQ_C128)
        return dispatch_pair<double>(upt, p, n_states, psi, k, theta, k_imm, theta_imm, partials, nullptr, sms, s);
    return dispatch_pair<float>(upt, p, n_states, psi, k, theta, k_imm, theta_imm, partials, nullptr, sms, s);
}

int launch_taylor5_pair_gated(const PoolView& p, int prec, int upt, void* psi, const DevStep* step,
                              double* partials, int sms, cudaStream_t s) {
    if (prec == TQ_C128)
        return dispatch_pair<double>(upt, p, 1, psi, &step->selected, &step->theta, 0, 0.0, partials, step, sms, s);
    return dispatch_pair<float>(upt, p, 1, psi, &step->selected, &step->theta, 0, 0.0, partials, step, sms, s);
}

int launch_norm_reduce(const double* partials, int prec, int n_states, int tiles_per_state,
                       double* norm2_out, double* step_norm2, cudaStream_t s) {
    const int bs = 256;
    const int grid = (n_states * 32 + bs - 1) / bs;
    if (prec == TQ_C128)
        k_norm_reduce<false><<<grid, bs, 0, s>>>(partials, n_states, tiles_per_state, norm2_out, step_norm2);
    else
        k_norm_reduce<true><<<grid, bs, 0, s>>>(partials, n_states, tiles_per_state, norm2_out, step_norm2);
    return 1;
}

int launch_scale_gated(void* psi, int prec, long long D, const double* norm2, const DevStep* gate,
                       cudaStream_t s) {
    const int bs = 256;
    const int grid = (int)((D + bs - 1) / bs < 1024 ? (D + bs - 1) / bs : 1024);
    if (prec == TQ_C128)
        k_scale<double2><<<grid, bs, 0, s>>>(static_cast<double2*>(psi), D, norm2, gate);
    else
        k_scale<float2><<<grid, bs, 0, s>>>(static_cast<float2*>(psi), D, norm2, gate);
    return 1;
}

int launch_scale(void* psi, int prec, long long D, const double* norm2, cudaStream_t s) {
    return launch_scale_gated(psi, prec, D, norm2, nullptr, s);
}

int launch_taylor5_csr(int nq, int prec, const int* rowptr, const int* col, const void* val,
                       double theta, void* psi, int renorm, double* acc, double* v0, double* v1,
                       double* partials, double* norm2, int sms, cudaStream_t s) {
    const long long D = 1ll << nq;
    // slice per CTA: 64 KiB of shared memory, and at most 8 rows per thread
    // so that v_k and the running sum of each row fit in registers
    const long long per_max = prec == TQ_C128 ? 4096 : 8192;
    long long csize = D <= per_max ? 1 : D / per_max;
    if (csize <= 16) {
        cudaError_t e;
        if (prec == TQ_C128)
            e = dispatch_cluster<double, double>(nq, (int)csize, rowptr, col,
                                                 static_cast<const double*>(val), theta, psi, renorm, norm2, s);
        else
            e = dispatch_cluster<float, float>(nq, (int)csize, rowptr, col,
                                               static_cast<const float*>(val), theta, psi, renorm, norm2, s);
        if (e == cudaSuccess) return 1;
        cudaGetLastError();   // clear a refused cluster configuration; fall back below
    }
    if (prec == TQ_C128)
        return run_unfused<double, double>(nq, rowptr, col, static_cast<const double*>(val), theta, psi,
                                           renorm, acc, v0, v1, partials, norm2, sms, s);
    return run_unfused<float, float>(nq, rowptr, col, static_cast<const float*>(val), theta, psi, renorm,
                                     acc, v0, v1, partials, norm2, sms, s);
}

}  // namespace tq
