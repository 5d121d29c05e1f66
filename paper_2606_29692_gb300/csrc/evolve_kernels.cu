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
// over the CTAs of a thread-block cluster (up to 16); the gather of v_{k-1}
// reads peer CTAs' shared memory through the cluster mapping, L lanes share
// a row, each product is followed by a cluster barrier, and v_{k-1}, v_k
// and the running sum live in shared memory.  Global memory is touched by
// the initial load, the CSR (L2-resident after the first product), and the
// final store only.  The float64 norm is reduced across the cluster and
// applied before the store when renormalisation is asked for.
#include "dev.cuh"
#include "pair.cuh"

#include <cooperative_groups.h>

#include <algorithm>

namespace cg = cooperative_groups;

namespace tq {

namespace {

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
            const T tpart = pair_tile<T, UPT>(op, theta, psi + (long long)b * D, (uint32_t)tl, units);
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
__global__ void k_norm_reduce(const double* partials, int n_states, int tiles, const double* base,
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
        if (base) s = base[w] + s;   // a carried norm: base + the change
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

// One product v_k = A v_{k-1} over the CTA's rows, L lanes per row (each
// lane takes every L-th entry, four in flight, gathers from the owning
// CTA's shared memory through the cluster mapping), then the group's sum
// goes to v_k and, times theta^k/k!, to the running sum (the group's first
// lane; every row has one owner for all five products).
template <typename T, typename VT, int L>
__device__ __forceinline__ void csr_product(const cg::cluster_group& cl, int row0, int R, int shift, long long D,
                                            const int* __restrict__ rowptr, const int* __restrict__ col,
                                            const VT* __restrict__ val, T coef, const typename C2<T>::type* cur,
                                            typename C2<T>::type* nxt, typename C2<T>::type* acc) {
    using V = typename C2<T>::type;
    const int sub = threadIdx.x & (L - 1);
    const int g = threadIdx.x / L, G = blockDim.x / L;
    for (int rl0 = 0; rl0 < R; rl0 += G) {          // uniform trip count: the shuffles below see whole warps
        const int rl = rl0 + g;
        T sx = T(0), sy = T(0);
        if (rl < R) {
            const int r = row0 + rl;
            const int e1 = rowptr[r + 1];
            constexpr int U = 4;
            for (int e0 = rowptr[r] + sub; e0 < e1; e0 += U * L) {
                int c[U];
                T a[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int e = e0 + j * L;
                    const bool ok = e < e1;
                    c[j] = ok ? col[e] : -1;
                    a[j] = ok ? (T)val[e] : T(0);
                }
                V v[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    if ((unsigned)c[j] < (unsigned)D) {   // a column outside the state is a zero entry
                        const V* src = cl.map_shared_rank(cur, (unsigned)c[j] >> shift);
                        v[j] = src[c[j] & (R - 1)];
                    } else {
                        v[j] = V{};
                        a[j] = T(0);
                    }
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    sx = fma(a[j], v[j].x, sx);
                    sy = fma(a[j], v[j].y, sy);
                }
            }
        }
#pragma unroll
        for (int o = L / 2; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (rl < R && sub == 0) {
            V nv;
            nv.x = sx;
            nv.y = sy;
            nxt[rl] = nv;
            V a = acc[rl];
            axpy(a, coef, nv);
            acc[rl] = a;
        }
    }
}

// The fused update for any CSR operator (Eqs. (7)-(8)): the state split
// over the CTAs of one thread-block cluster, R = D / cluster rows each,
// staged in shared memory as v_{k-1}, v_k and the running sum.  Each of the
// five products gathers v_{k-1} from whichever CTA owns the column (local
// or distributed shared memory) and writes v_k locally; one cluster
// barrier per product.  The lanes per row follow the operator's mean row
// length (read on the device from rowptr[D]).  The float64 norm is pushed
// to every CTA's shared memory after the last product and, with
// renormalisation, applied before the single store.
template <typename T, typename VT>
__global__ void __launch_bounds__(1024)
k_taylor5_csr_cluster(int nq, const int* __restrict__ rowptr, const int* __restrict__ col,
                      const VT* __restrict__ val, double theta, typename C2<T>::type* psi, int renorm,
                      double* norm2_out) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ double cta_part;
    __shared__ double slots[16];
    __shared__ double scale_sh;
    cg::cluster_group cl = cg::this_cluster();
    const unsigned nb = cl.num_blocks(), rank = cl.block_rank();
    const long long D = 1ll << nq;
    const int R = (int)(D / nb);
    const int shift = 31 - __clz(R);
    V* vb0 = reinterpret_cast<V*>(smem_raw);
    V* vb1 = vb0 + R;
    V* acc = vb1 + R;
    const int row0 = (int)rank * R;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        const V v = psi[row0 + i];
        vb0[i] = v;
        acc[i] = v;
    }
    T cf[6];
    taylor_coefs<T>(theta, cf);
    const long long nnz = rowptr[D];
    const long long per_row = nnz / D;
    cl.sync();   // every CTA has started and staged its rows
    V* cur = vb0;
    V* nxt = vb1;
    for (int k = 1; k <= 5; ++k) {
        if (per_row >= 24)
            csr_product<T, VT, 32>(cl, row0, R, shift, D, rowptr, col, val, cf[k], cur, nxt, acc);
        else if (per_row >= 4)
            csr_product<T, VT, 8>(cl, row0, R, shift, D, rowptr, col, val, cf[k], cur, nxt, acc);
        else
            csr_product<T, VT, 1>(cl, row0, R, shift, D, rowptr, col, val, cf[k], cur, nxt, acc);
        cl.sync();   // v_k complete everywhere; nobody reads v_{k-1} any more
        V* t = cur;
        cur = nxt;
        nxt = t;
    }
    double part = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x)
        part += (double)acc[i].x * acc[i].x + (double)acc[i].y * acc[i].y;
    double v[1] = {part};
    block_sum<1>(v, red);
    if (threadIdx.x == 0) cta_part = v[0];
    __syncthreads();
    if (threadIdx.x < nb) *cl.map_shared_rank(&slots[rank], threadIdx.x) = cta_part;
    cl.sync();   // the pushes are visible; nothing reads a peer after this
    if (threadIdx.x == 0) {
        double total = 0.0;
        for (unsigned q = 0; q < nb; ++q) total += slots[q];
        scale_sh = renorm ? 1.0 / sqrt(total) : 1.0;
        if (rank == 0 && norm2_out) *norm2_out = total;
    }
    __syncthreads();
    const double sc = scale_sh;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        V o;
        o.x = (T)((double)acc[i].x * sc);
        o.y = (T)((double)acc[i].y * sc);
        psi[row0 + i] = o;
    }
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

template <typename T, typename VT>
cudaError_t launch_cluster(int nq, int csize, const int* rowptr, const int* col, const VT* val, double theta,
                           void* psi, int renorm, double* norm2, cudaStream_t s) {
    using V = typename C2<T>::type;
    auto kern = k_taylor5_csr_cluster<T, VT>;
    const size_t smem = (size_t)3 * ((1ll << nq) / csize) * sizeof(V);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (csize > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(1024);
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
    return cudaLaunchKernelEx(&cfg, kern, nq, rowptr, col, val, theta, static_cast<V*>(psi), renorm, norm2);
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
    return launch_norm_carry(partials, prec, n_states, tiles_per_state, nullptr, norm2_out, step_norm2, s);
}

int launch_norm_carry(const double* partials, int prec, int n_states, int tiles_per_state, const double* base,
                      double* norm2_out, double* step_norm2, cudaStream_t s) {
    const int bs = 256;
    const int grid = (n_states * 32 + bs - 1) / bs;
    if (prec == TQ_C128)
        k_norm_reduce<false><<<grid, bs, 0, s>>>(partials, n_states, tiles_per_state, base, norm2_out, step_norm2);
    else
        k_norm_reduce<true><<<grid, bs, 0, s>>>(partials, n_states, tiles_per_state, base, norm2_out, step_norm2);
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
    // rows per CTA: three vectors of them in shared memory (at most 192 KB);
    // about 1024 rows per CTA, up to a 16-CTA cluster; a cluster size the
    // device refuses falls back to half the CTAs with twice the rows
    const long long vb = prec == TQ_C128 ? 16 : 8;
    const long long rmax = (192ll << 10) / (3 * vb);
    for (long long csize = std::min<long long>(16, std::max<long long>(1, D / 1024)); csize >= 1; csize /= 2) {
        if (D / csize > rmax || D % csize != 0) break;
        cudaError_t e;
        if (prec == TQ_C128)
            e = launch_cluster<double, double>(nq, (int)csize, rowptr, col, static_cast<const double*>(val), theta,
                                               psi, renorm, norm2, s);
        else
            e = launch_cluster<float, float>(nq, (int)csize, rowptr, col, static_cast<const float*>(val), theta,
                                             psi, renorm, norm2, s);
        if (e == cudaSuccess) return 1;
        cudaGetLastError();   // clear a refused cluster configuration; try a smaller one
    }
    if (prec == TQ_C128)
        return run_unfused<double, double>(nq, rowptr, col, static_cast<const double*>(val), theta, psi,
                                           renorm, acc, v0, v1, partials, norm2, sms, s);
    return run_unfused<float, float>(nq, rowptr, col, static_cast<const float*>(val), theta, psi, renorm,
                                     acc, v0, v1, partials, norm2, sms, s);
}

}  // namespace tq
