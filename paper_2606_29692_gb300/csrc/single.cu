// Single-state Taylor-5 update with renormalisation in one launch
// (Sec. III-C, Eqs. (6)-(8); dividing by the float64 norm is the ADAPT
// driver's addition, not the paper's).
//
// A state of up to 2^16 amplitudes is split over the CTAs of one
// thread-block cluster.  Each thread loads whole pairs {r, r ^ x} (the
// enumeration of the full-state pair kernel), runs the five products and
// the running sum in registers, and keeps the results there.  Each CTA
// pushes its float64 sum of |psi'|^2 into every peer's shared memory, one
// hardware cluster barrier follows, and every CTA adds the sums in rank
// order, so all get the same total; each thread then scales and stores its
// amplitudes.
// Each amplitude is read once and written once, and nothing goes through
// global scratch: the update, the norm and the rescale are one kernel where
// the batched form needs three.
#include "dev.cuh"
#include "pair.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace tq {

namespace {

constexpr int SINGLE_BS = 256;
constexpr int SINGLE_MAX_CLUSTER = 16;
constexpr int SINGLE_MAX_UPT = 4;

// k, theta from the arguments, or from the ADAPT step record when `gate`
// is set (then a converged step leaves the state alone).  norm2_out, if
// set, receives ||psi'||^2 before the rescale.
template <typename T, int UPT>
__global__ void __launch_bounds__(SINGLE_BS)
k_taylor5_single(PoolView p, int k_imm, double th_imm, const DevStep* gate, typename C2<T>::type* psi,
                 int renorm, double* norm2_out) {
    using V = typename C2<T>::type;
    constexpr int NW = SINGLE_BS / 32;
    static_assert(NW == 8, "the partials' shuffle tree spans eight warps");
    __shared__ double red[NW];
    __shared__ double cta_part;
    __shared__ double slots[SINGLE_MAX_CLUSTER];   // every CTA's sum, pushed here by its owner
    __shared__ double scale_sh;
    cg::cluster_group cl = cg::this_cluster();
    // the same decision in every CTA of the cluster, before any barrier
    if (gate && gate->converged) return;
    const int k = gate ? gate->selected : k_imm;
    const double theta = gate ? gate->theta : th_imm;
    if (k < 0 || k >= p.M) {
        if (cl.block_rank() == 0 && threadIdx.x == 0 && norm2_out)
            *norm2_out = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    // every CTA of the cluster must be running before a peer writes into
    // its shared memory: arrive now, wait just before the writes
    asm volatile("barrier.cluster.arrive;\n" ::: "memory");
    const OpRec<T> op = make_rec<T>(p, k);
    const uint32_t x = op.x;
    const int hb = 31 - __clz(x);
    const uint32_t units = (uint32_t)((1ll << p.nq) >> 2);
    const uint32_t per = units / (uint32_t)cl.num_blocks();
    const uint32_t u0 = (uint32_t)cl.block_rank() * per;
    PairUnit<V> w[UPT];
    bool ok[UPT];
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
        const uint32_t i = j * SINGLE_BS + threadIdx.x;
        ok[j] = i < per;
        if (ok[j]) unit_load(psi, x, hb, u0 + i, w[j]);
    }
    // the coefficients: complex64 per thread on the float32 pipe; complex128
    // once per CTA, by thread 0 while the loads are in flight
    T cf[6];
    double c5 = 0.0, s5 = 0.0;
    if constexpr (sizeof(T) == 8) {
        __shared__ double coef_sh[8];
        if (threadIdx.x == 0) {
            double c[6];
            taylor_coefs_fast<double>(theta, c);
            closed_coefs(c, coef_sh[6], coef_sh[7]);
#pragma unroll
            for (int i = 0; i < 6; ++i) coef_sh[i] = c[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 6; ++i) cf[i] = coef_sh[i];
        c5 = coef_sh[6];
        s5 = coef_sh[7];
    } else {
        taylor_coefs_fast<T>(theta, cf);
    }
    T tpart = T(0);
#pragma unroll
    for (int j = 0; j < UPT; ++j)
        if (ok[j]) unit_update<T>(op, hb, cf, c5, s5, w[j], tpart);
    store_partial(&red[threadIdx.x >> 5], tpart);
    __syncthreads();
    if (threadIdx.x < 32) {
        // the warps' partials by a fixed shuffle tree (complex64: the
        // (hi, lo) float pairs widened first)
        double v = 0.0;
        if (threadIdx.x < NW) {
            if constexpr (sizeof(T) == 4) {
                const float2 hl = *reinterpret_cast<const float2*>(&red[threadIdx.x]);
                v = (double)hl.x + (double)hl.y;
            } else {
                v = red[threadIdx.x];
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) cta_part = v;
    }
    __syncthreads();
    // each CTA writes its sum into slot `rank` of every CTA (one thread per
    // peer); after the barrier every CTA adds its own slots in rank order,
    // so all get the same total and no CTA reads another's memory later
    const unsigned nb = cl.num_blocks(), rank = cl.block_rank();
    asm volatile("barrier.cluster.wait;\n" ::: "memory");
    if (threadIdx.x < nb) *cl.map_shared_rank(&slots[rank], threadIdx.x) = cta_part;
    cl.sync();   // the pushes are visible; nothing reads a peer after this
    if (threadIdx.x < 32) {
        // warp 0: the slots by a fixed shuffle tree (rank order pairs up
        // the same way in every CTA), then one thread takes the reciprocal
        // square root (the float64 pipe issues a warp instruction every 64
        // cycles on this part: no serial chains, no division)
        double t = threadIdx.x < nb ? slots[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) {
            scale_sh = renorm ? rsqrt(t) : 1.0;
            if (rank == 0 && norm2_out) *norm2_out = t;
        }
    }
    __syncthreads();
    if (renorm) {
        // complex64 scales in float32 (the amplitudes' own precision)
        const T sc = (T)scale_sh;
#pragma unroll
        for (int j = 0; j < UPT; ++j) {
            if (!ok[j]) continue;
            V* v[4] = {&w[j].a0, &w[j].a1, &w[j].b0, &w[j].b1};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i]->x *= sc;
                v[i]->y *= sc;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < UPT; ++j)
        if (ok[j]) unit_store(psi, x, hb, w[j]);
}

// Cluster size and units per thread for a state of 2^nq amplitudes: the
// fewest units per thread whose cluster fits; 0 when no configuration does.
int single_shape(int nq, int max_cluster, int* upt_out) {
    if (nq < 2) return 0;
    const long long units = (1ll << nq) >> 2;
    for (int upt = 1; upt <= SINGLE_MAX_UPT; upt *= 2) {
        long long cs = (units + (long long)SINGLE_BS * upt - 1) / ((long long)SINGLE_BS * upt);
        if (cs < 1) cs = 1;
        if (cs <= max_cluster) {
            *upt_out = upt;
            return (int)cs;
        }
    }
    return 0;
}

cudaLaunchConfig_t single_cfg(int csize, cudaStream_t s, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(csize);
    cfg.blockDim = dim3(SINGLE_BS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename T, int UPT>
bool single_launchable_t(int csize) {
    auto kern = k_taylor5_single<T, UPT>;
    cudaError_t e = cudaSuccess;
    if (csize > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = single_cfg(csize, 0, attr);
    int n = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) (void)cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

template <typename T>
bool single_launchable(int csize, int upt) {
    switch (upt) {
        case 1: return single_launchable_t<T, 1>(csize);
        case 2: return single_launchable_t<T, 2>(csize);
        case 4: return single_launchable_t<T, 4>(csize);
        default: return false;
    }
}

template <typename T, int UPT>
cudaError_t launch_single_t(const PoolView& p, int csize, int k, double theta, const DevStep* gate, void* psi,
                            int renorm, double* norm2, cudaStream_t s) {
    using V = typename C2<T>::type;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = single_cfg(csize, s, attr);
    return cudaLaunchKernelEx(&cfg, k_taylor5_single<T, UPT>, p, k, theta, gate, static_cast<V*>(psi), renorm,
                              norm2);
}

template <typename T>
cudaError_t dispatch_single(const PoolView& p, int csize, int upt, int k, double theta, const DevStep* gate,
                            void* psi, int renorm, double* norm2, cudaStream_t s) {
    switch (upt) {
        case 1: return launch_single_t<T, 1>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        case 2: return launch_single_t<T, 2>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        case 4: return launch_single_t<T, 4>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        default: return cudaErrorInvalidConfiguration;
    }
}

// Cluster size and units per thread that launch for this state size and
// precision (cached per size), or false when none does.
bool single_config(int nq, int prec, int* cs_out, int* upt_out) {
    static int cache[2][32][2] = {};   // [prec][nq] -> {cluster size, upt}; -1 none
    if (nq < 2 || nq >= 32) return false;
    int* e = cache[prec == TQ_C128 ? 1 : 0][nq];
    if (e[0] == 0) {
        e[0] = -1;
        for (int maxc = SINGLE_MAX_CLUSTER; maxc >= 1; maxc /= 2) {
            int upt = 0;
            const int cs = single_shape(nq, maxc, &upt);
            if (cs == 0) break;
            const bool ok = prec == TQ_C128 ? single_launchable<double>(cs, upt) : single_launchable<float>(cs, upt);
            if (ok) {
                e[0] = cs;
                e[1] = upt;
                break;
            }
        }
    }
    if (e[0] < 0) return false;
    *cs_out = e[0];
    *upt_out = e[1];
    return true;
}

}  // namespace

bool taylor5_single_ready(int nq, int prec) {
    int cs = 0, upt = 0;
    return single_config(nq, prec, &cs, &upt);
}

int launch_taylor5_single(const PoolView& p, int prec, int k, double theta, const DevStep* gate, void* psi,
                          int renorm, double* norm2, cudaStream_t s) {
    int cs = 0, upt = 0;
    if (!single_config(p.nq, prec, &cs, &upt)) return -1;
    const cudaError_t e = prec == TQ_C128
                              ? dispatch_single<double>(p, cs, upt, k, theta, gate, psi, renorm, norm2, s)
                              : dispatch_single<float>(p, cs, upt, k, theta, gate, psi, renorm, norm2, s);
    return e == cudaSuccess ? 1 : -1;
}

}  // namespace tq
