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

// Taylor-5 on many sector states: warp w updates rows [t RW, (t+1) RW) of
// state b (w = b * tiles + t), rows strided by 32 across lanes.  The thread
// of row r handles the pair (r, c) when r < c, and leaves annihilated rows
// alone; every row adds |psi'_r|^2 to the warp's norm partial.  The op and
// angle come from k[b], theta[b], or (k_fixed, theta_fixed), or from the
// device step record when `gate` is set (skipped if it has converged).
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
    const int k = gate ? gate->selected : (ks ? ks[b] : k_fixed);
    const double th = gate ? gate->theta : (thetas ? thetas[b] : theta_fixed);
    if (k < 0 || k >= p.M || !isfinite(th)) {
        store_nan_partial(partials + w, T(0));
        return;
    }
    const double t2 = th * th;
    const T c5 = (T)(1.0 - t2 / 2.0 + t2 * t2 / 24.0);
    const T s5 = (T)(th * (1.0 - t2 / 6.0 + t2 * t2 / 120.0));
    V* __restrict__ x = psi + b * dim;
    const int* __restrict__ col = p.scol + (long long)k * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)k * dim;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < SECT_ROWS_PER_LANE; ++j) {
        const long long r = (long long)t * SECT_WARP_ROWS + j * 32 + lane;
        if (r >= dim) break;
        const int c = col[r];
        const int sg = sgn[r];
        const V vr = x[r];
        if (sg == 0) {
            acc += vr.x * vr.x + vr.y * vr.y;
        } else if (r < c) {
            const V vc = x[c];
            const T a = s5 * (T)sg;
            const V nr = {c5 * vr.x + a * vc.x, c5 * vr.y + a * vc.y};
            const V nc = {c5 * vc.x - a * vr.x, c5 * vc.y - a * vr.y};
            x[r] = nr;
            x[c] = nc;
            acc += nr.x * nr.x + nr.y * nr.y + nc.x * nc.x + nc.y * nc.y;
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

// u1 = A psi, u2 = A u1 = -psi on the rows A does not annihilate (A^2 = -I
// on a pair), for the selected op; float64 outputs.
template <typename T>
__global__ void k_apply_twice_sector(PoolView p, const DevStep* step, const typename C2<T>::type* psi, double2* u1,
                                     double2* u2) {
    if (step->converged) return;
    const long long dim = p.sdim;
    const int k = step->selected;
    const int* __restrict__ col = p.scol + (long long)k * dim;
    const signed char* __restrict__ sgn = p.ssgn + (long long)k * dim;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < dim; r += stride) {
        const int sg = sgn[r];
        const typename C2<T>::type vc = psi[col[r]], vr = psi[r];
        u1[r] = make_double2(sg * (double)vc.x, sg * (double)vc.y);
        u2[r] = sg ? make_double2(-(double)vr.x, -(double)vr.y) : make_double2(0.0, 0.0);
    }
}

}  // namespace

int sector_tiles(long long dim) { return (int)((dim + SECT_WARP_ROWS - 1) / SECT_WARP_ROWS); }

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
                          double* partials, cudaStream_t s) {
    const int tiles = sector_tiles(p.sdim);
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

int launch_apply_twice_sector(const PoolView& p, const DevStep* step, const void* psi, int prec, double2* u1,
                              double2* u2, cudaStream_t s) {
    const long long dim = p.sdim;
    const int grid = (int)((dim + 255) / 256 < 1024 ? (dim + 255) / 256 : 1024);
    if (prec == TQ_C128)
        k_apply_twice_sector<double><<<grid, 256, 0, s>>>(p, step, static_cast<const double2*>(psi), u1, u2);
    else
        k_apply_twice_sector<float><<<grid, 256, 0, s>>>(p, step, static_cast<const float2*>(psi), u1, u2);
    return 1;
}

}  // namespace tq
