// Hot-path kernels in a sector-restricted basis (fixed alpha and beta
// electron counts; a variant of the paper's 2^N formulation, not part of
// it).  Every pool generator maps the sector into itself, and restricted to
// it A_k pairs rows r, c with A[r][c] = s = +-1, A[c][r] = -s, or
// annihilates row r.  It is stored as one (column, sign) entry per row.
//
// On a pair A^2 = -I, so the Taylor-5 sum of Eqs. (6)-(8) is exactly
//   psi'_r = c5 psi_r + s5 s psi_c,   psi'_c = c5 psi_c - s5 s psi_r,
//   c5 = 1 - t^2/2 + t^4/24,  s5 = t - t^3/6 + t^5/120,
// the same five products and sum in closed form; annihilated rows keep psi.
#include "dev.cuh"
#include "pair.cuh"
#include "sector.cuh"

namespace tq {

namespace {

// (column, sign) of every (op, row): A_k[r][r ^ x_k] evaluated in qubit space
// and its column ranked in the sector.  *bad counts entries that would leave
// the sector (none for spin-conserving generators).
__global__ void k_sector_pool(PoolView p, const uint32_t* sq, const SectorSpec* sect, long long dim, int* scol,
                              signed char* ssgn, unsigned long long* bad) {
    const long long total = (long long)p.M * dim;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += stride) {
        const int k = (int)(i / dim);
        const long long r = i - (long long)k * dim;
        const uint32_t c = sq[r] ^ p.x[k];
        const double v = op_value<double>(p, k, c);
        int col = (int)r;
        signed char sg = 0;
        if (v != 0.0) {
            const long long rc = sector_rank(c, *sect);
            if (rc < 0) {
                atomicAdd(bad, 1ull);
            } else {
                col = (int)rc;
                sg = v > 0.0 ? 1 : -1;
            }
        }
        scol[i] = col;
        ssgn[i] = sg;
    }
}

constexpr int SECT_ROWS_PER_LANE = 4;
constexpr int SECT_WARP_ROWS = 32 * SECT_ROWS_PER_LANE;
constexpr int SECT_SMEM_THREADS = 128;
constexpr size_t SECT_SMEM_MAX = 48 * 1024;    // states up to this size go through shared memory

struct SectOp {
    int k;
    double th;
};

// op and angle of state b (or of the step record when `gate` is set)
__device__ __forceinline__ SectOp sector_op(long long b, const int* ks, const double* thetas, int k_fixed,
                                            double theta_fixed, const DevStep* gate) {
    SectOp o;
    o.k = gate ? gate->selected : (ks ? ks[b] : k_fixed);
    o.th = gate ? gate->theta : (thetas ? thetas[b] : theta_fixed);
    return o;
}

// c5 = 1 - t^2/2 + t^4/24, s5 = t - t^3/6 + t^5/120 in the state's
// precision, by Horner's rule with reciprocal factorials (no division)
template <typename T>
__device__ __forceinline__ void sector_coefs(double th, T& c5, T& s5) {
    const T t = (T)th, t2 = t * t;
    c5 = fma(t2, fma(t2, T(1.0 / 24.0), T(-0.5)), T(1));
    s5 = t * fma(t2, fma(t2, T(1.0 / 120.0), T(-1.0 / 6.0)), T(1));
}

// The pair (r, c) with A[r][c] = sg: psi'_r = c5 psi_r + s5 sg psi_c,
// psi'_c = c5 psi_c - s5 sg psi_r.
template <typename V, typename T>
__device__ __forceinline__ void sector_pair(V& vr, V& vc, T c5, T s5, int sg) {
    const T a = s5 * (T)sg;
    const V nr = {c5 * vr.x + a * vc.x, c5 * vr.y + a * vc.y};
    const V nc = {c5 * vc.x - a * vr.x, c5 * vc.y - a * vr.y};
    vr = nr;
    vc = nc;
}

// Taylor-5 on many sector states, one block per state, the state staged in
// shared memory: coalesced load, every pair updated in place by the thread
// of its smaller row, coalesced store of the whole state.  The block also
// finishes the state's float64 norm (warp partials in a fixed order) into
// norm2[b] and/or *step_norm2, so no reduction launch follows.
template <typename T>
__global__ void __launch_bounds__(SECT_SMEM_THREADS, 10)
k_taylor5_sector_smem(PoolView p, typename C2<T>::type* psi, const int* ks, const double* thetas, int k_fixed,
                      double theta_fixed, const DevStep* gate, double* norm2, double* step_norm2) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char sect_raw[];
    V* sm = reinterpret_cast<V*>(sect_raw);
    __shared__ T sc[2];
    __shared__ int sok;
    __shared__ double swarp[SECT_SMEM_THREADS / 32];
    if (gate && gate->converged) return;
    const long long b = blockIdx.x;
    const long long dim = p.sdim;
    const int t = threadIdx.x;
    // every thread reads the op (an integer broadcast); one thread checks the
    // angle and forms the float64 coefficients
    const int k = gate ? gate->selected : (ks ? ks[b] : k_fixed);
    const bool kok = k >= 0 && k < p.M;
    if (t == 0) {
        const double th = gate ? gate->theta : (thetas ? thetas[b] : theta_fixed);
        sok = kok && isfinite(th);
        if (sok) sector_coefs<T>(th, sc[0], sc[1]);
    }
    V* __restrict__ x = psi + b * dim;
    const int* __restrict__ col = p.scol + (long long)(kok ? k : 0) * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)(kok ? k : 0) * dim;
    // the state and this thread's table entries load together
    constexpr int J = 10;
    int cj[J], sj[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const long long r = t + (long long)j * SECT_SMEM_THREADS;
        cj[j] = 0;
        sj[j] = 0;
        if (r < dim) {
            sm[r] = x[r];
            cj[j] = col[r];
            sj[j] = sgn[r];
        }
    }
    for (long long r = t + (long long)J * SECT_SMEM_THREADS; r < dim; r += SECT_SMEM_THREADS) sm[r] = x[r];
    __syncthreads();
    if (!sok) {
        if (t == 0) {
            if (norm2) norm2[b] = nan("");
            if (step_norm2) *step_norm2 = nan("");
        }
        return;
    }
    const T c5 = sc[0], s5 = sc[1];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const long long r = t + (long long)j * SECT_SMEM_THREADS;
        if (sj[j] != 0 && r < cj[j]) sector_pair<V, T>(sm[r], sm[cj[j]], c5, s5, sj[j]);
    }
    for (long long r = t + (long long)J * SECT_SMEM_THREADS; r < dim; r += SECT_SMEM_THREADS) {
        const int sg = sgn[r];
        const int c = col[r];
        if (sg != 0 && r < c) sector_pair<V, T>(sm[r], sm[c], c5, s5, sg);
    }
    __syncthreads();
    T acc = T(0);
    for (long long r = t; r < dim; r += SECT_SMEM_THREADS) {
        const V v = sm[r];
        x[r] = v;
        acc += v.x * v.x + v.y * v.y;
    }
    store_partial(swarp + (t >> 5), acc);
    __syncthreads();
    // warp 0 combines the warp partials in a fixed tree
    if (t < 32) {
        constexpr int NW = SECT_SMEM_THREADS / 32;
        double n;
        if constexpr (sizeof(T) == 4) {
            const float2 hl = t < NW ? *reinterpret_cast<const float2*>(swarp + t) : make_float2(0.f, 0.f);
            float hi = hl.x, lo = hl.y;
#pragma unroll
            for (int o = NW / 2; o > 0; o >>= 1) {
                const float oh = __shfl_down_sync(0xffffffffu, hi, o);
                const float ol = __shfl_down_sync(0xffffffffu, lo, o);
                float sum, err;
                two_sum(hi, oh, sum, err);
                hi = sum;
                lo = lo + ol + err;
            }
            n = (double)hi + (double)lo;
        } else {
            n = t < NW ? swarp[t] : 0.0;
#pragma unroll
            for (int o = NW / 2; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
        }
        if (t == 0) {
            if (norm2) norm2[b] = n;
            if (step_norm2) *step_norm2 = n;
        }
    }
}

// The same for states too large for shared memory: warp w updates rows
// [t RW, (t+1) RW) of state b (w = b * tiles + t), rows strided by 32
// across lanes; the thread of row r handles the pair (r, c) when r < c.
// Loads of a lane's rows are issued together (its pairs are disjoint from
// every other thread's, so no store of another lane can alias them).
template <typename T>
__global__ void __launch_bounds__(256)
k_taylor5_sector(PoolView p, long long n_states, typename C2<T>::type* psi, const int* ks, const double* thetas,
                 int k_fixed, double theta_fixed, const DevStep* gate, double* partials, int tiles) {
    using V = typename C2<T>::type;
    if (gate && gate->converged) return;
    const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (w >= n_states * tiles) return;
    const int lane = threadIdx.x & 31;
    const long long b = w / tiles;
    const int t = (int)(w - b * tiles);
    const long long dim = p.sdim;
    // lane 0 reads the op and angle and forms the float64 coefficients
    int k = -1;
    T c5 = T(0), s5 = T(0);
    if (lane == 0) {
        const SectOp o = sector_op(b, ks, thetas, k_fixed, theta_fixed, gate);
        if (o.k >= 0 && o.k < p.M && isfinite(o.th)) {
            k = o.k;
            sector_coefs<T>(o.th, c5, s5);
        }
    }
    k = __shfl_sync(0xffffffffu, k, 0);
    c5 = __shfl_sync(0xffffffffu, c5, 0);
    s5 = __shfl_sync(0xffffffffu, s5, 0);
    if (k < 0) {
        store_nan_partial(partials + w, T(0));
        return;
    }
    V* __restrict__ x = psi + b * dim;
    const int* __restrict__ col = p.scol + (long long)k * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)k * dim;
    int c[SECT_ROWS_PER_LANE], sg[SECT_ROWS_PER_LANE];
    V vr[SECT_ROWS_PER_LANE], vc[SECT_ROWS_PER_LANE];
#pragma unroll
    for (int j = 0; j < SECT_ROWS_PER_LANE; ++j) {
        const long long r = (long long)t * SECT_WARP_ROWS + j * 32 + lane;
        const bool in = r < dim;
        c[j] = in ? col[r] : 0;
        sg[j] = in ? sgn[r] : 0;
        vr[j] = in ? x[r] : V{};
    }
#pragma unroll
    for (int j = 0; j < SECT_ROWS_PER_LANE; ++j) {
        const long long r = (long long)t * SECT_WARP_ROWS + j * 32 + lane;
        vc[j] = (sg[j] != 0 && r < c[j]) ? x[c[j]] : V{};
    }
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < SECT_ROWS_PER_LANE; ++j) {
        const long long r = (long long)t * SECT_WARP_ROWS + j * 32 + lane;
        if (r >= dim) continue;
        if (sg[j] == 0) {
            acc += vr[j].x * vr[j].x + vr[j].y * vr[j].y;
        } else if (r < c[j]) {
            sector_pair<V, T>(vr[j], vc[j], c5, s5, sg[j]);
            x[r] = vr[j];
            x[c[j]] = vc[j];
            acc += vr[j].x * vr[j].x + vr[j].y * vr[j].y + vc[j].x * vc[j].x + vc[j].y * vc[j].y;
        }
    }
    store_partial(partials + w, acc);
}

// g_k = 2 Re<w|A_k psi> / <psi|psi>: one block per op, fixed-order sums.
template <typename T>
__global__ void __launch_bounds__(256)
k_sector_grad(PoolView p, const double2* __restrict__ w, const typename C2<T>::type* __restrict__ psi,
              const DevStep* step, double* g) {
    __shared__ double sh[8];
    const int k = blockIdx.x;
    const long long dim = p.sdim;
    const int* __restrict__ col = p.scol + (long long)k * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)k * dim;
    double s = 0.0;
    for (long long r = threadIdx.x; r < dim; r += blockDim.x) {
        const int sg = sgn[r];
        if (sg == 0) continue;
        const typename C2<T>::type v = psi[col[r]];
        const double2 wr = w[r];
        s += (double)sg * (wr.x * (double)v.x + wr.y * (double)v.y);
    }
    double v[1] = {s};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) g[k] = 2.0 * v[0] / step->e_den;
}

// The line search's records {psi, u1 = A psi, u2 = A u1, 0} per sector row
// (u2 = -psi on the rows A does not annihilate: A^2 = -I on a pair), for
// the selected op, in the state's precision (exact: the entries are +-1).
template <typename T>
__global__ void k_apply_twice_sector(PoolView p, const DevStep* step, const typename C2<T>::type* psi,
                                     typename C2<T>::type* z) {
    using V = typename C2<T>::type;
    if (step->converged) return;
    const long long dim = p.sdim;
    const int k = step->selected;
    const int* __restrict__ col = p.scol + (long long)k * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)k * dim;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < dim; r += stride) {
        const int sg = sgn[r];
        const V vc = psi[col[r]], vr = psi[r];
        V* rec = z + 4 * r;
        rec[0] = vr;
        rec[1] = sg > 0 ? vc : (sg < 0 ? V{-vc.x, -vc.y} : V{T(0), T(0)});
        rec[2] = sg ? V{-vr.x, -vr.y} : V{T(0), T(0)};
        rec[3] = V{T(0), T(0)};
    }
}

}  // namespace

// states of up to SECT_SMEM_MAX bytes take the shared-memory kernel
bool sector_in_smem(long long dim, int prec) {
    return (size_t)dim * (prec == TQ_C128 ? 16 : 8) <= SECT_SMEM_MAX;
}

int sector_tiles(long long dim, int prec) {
    return sector_in_smem(dim, prec) ? SECT_SMEM_THREADS / 32 : (int)((dim + SECT_WARP_ROWS - 1) / SECT_WARP_ROWS);
}

int launch_sector_pool(const PoolView& p, const uint32_t* sq, const SectorSpec* sect, long long dim, int* scol,
                       signed char* ssgn, unsigned long long* bad, int sms, cudaStream_t s) {
    const long long total = (long long)p.M * dim;
    long long grid = (total + 255) / 256;
    if (grid > (long long)sms * 16) grid = (long long)sms * 16;
    k_sector_pool<<<(int)(grid < 1 ? 1 : grid), 256, 0, s>>>(p, sq, sect, dim, scol, ssgn, bad);
    return 1;
}

int launch_taylor5_sector(const PoolView& p, long long n_states, int prec, void* psi, const int* k,
                          const double* theta, int k_fixed, double theta_fixed, const DevStep* gate,
                          double* partials, double* norm2, double* step_norm2, cudaStream_t s) {
    if (sector_in_smem(p.sdim, prec)) {
        const size_t smem = (size_t)p.sdim * (prec == TQ_C128 ? 16 : 8);
        if (prec == TQ_C128)
            k_taylor5_sector_smem<double><<<(unsigned)n_states, SECT_SMEM_THREADS, smem, s>>>(
                p, static_cast<double2*>(psi), k, theta, k_fixed, theta_fixed, gate, norm2, step_norm2);
        else
            k_taylor5_sector_smem<float><<<(unsigned)n_states, SECT_SMEM_THREADS, smem, s>>>(
                p, static_cast<float2*>(psi), k, theta, k_fixed, theta_fixed, gate, norm2, step_norm2);
        return 1;
    }
    const int tiles = sector_tiles(p.sdim, prec);
    const long long warps = n_states * tiles;
    const long long grid = (warps * 32 + 255) / 256;
    if (prec == TQ_C128)
        k_taylor5_sector<double><<<(unsigned)grid, 256, 0, s>>>(p, n_states, static_cast<double2*>(psi), k, theta,
                                                                k_fixed, theta_fixed, gate, partials, tiles);
    else
        k_taylor5_sector<float><<<(unsigned)grid, 256, 0, s>>>(p, n_states, static_cast<float2*>(psi), k, theta,
                                                               k_fixed, theta_fixed, gate, partials, tiles);
    return 1;
}

int launch_sector_gradients(const PoolView& p, const double2* w, const void* psi, int prec, const DevStep* step,
                            double* g, cudaStream_t s) {
    if (prec == TQ_C128)
        k_sector_grad<double><<<p.M, 256, 0, s>>>(p, w, static_cast<const double2*>(psi), step, g);
    else
        k_sector_grad<float><<<p.M, 256, 0, s>>>(p, w, static_cast<const float2*>(psi), step, g);
    return 1;
}

int launch_apply_twice_sector(const PoolView& p, const DevStep* step, const void* psi, int prec, void* z,
                              cudaStream_t s) {
    const long long dim = p.sdim;
    const int grid = (int)((dim + 255) / 256 < 1024 ? (dim + 255) / 256 : 1024);
    if (prec == TQ_C128)
        k_apply_twice_sector<double><<<grid, 256, 0, s>>>(p, step, static_cast<const double2*>(psi),
                                                          static_cast<double2*>(z));
    else
        k_apply_twice_sector<float><<<grid, 256, 0, s>>>(p, step, static_cast<const float2*>(psi),
                                                         static_cast<float2*>(z));
    return 1;
}

}  // namespace tq
