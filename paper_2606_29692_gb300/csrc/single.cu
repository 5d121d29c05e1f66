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
//
// Launched with programmatic stream serialisation: the kernel lets the next
// launch in its stream start at once, and waits (griddepcontrol.wait: until
// the previous grid in the stream has completed and its writes are
// visible) only before it reads the state or the step record.  Back-to-back
// calls then overlap one call's tail with the next one's set-up (operator
// record, coefficients) instead of paying a full launch each.
#include "dev.cuh"
#include "grad.cuh"
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
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // the step record is the previous kernel's output: wait for it first
    if (gate) asm volatile("griddepcontrol.wait;" ::: "memory");
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
    // the coefficients: complex64 per thread on the float32 pipe; complex128
    // once per CTA, by thread 0 (before the wait, or while the loads are in
    // flight)
    __shared__ double coef_sh[8];
    if (sizeof(T) == 8 && threadIdx.x == 0) {
        double c[6];
        taylor_coefs_fast<double>(theta, c);
        closed_coefs(c, coef_sh[6], coef_sh[7]);
#pragma unroll
        for (int i = 0; i < 6; ++i) coef_sh[i] = c[i];
    }
    if (!gate) asm volatile("griddepcontrol.wait;" ::: "memory");   // the state is the previous kernel's output
    PairUnit<V> w[UPT];
    bool ok[UPT];
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
        const uint32_t i = j * SINGLE_BS + threadIdx.x;
        ok[j] = i < per;
        if (ok[j]) unit_load(psi, x, hb, u0 + i, w[j]);
    }
    T cf[6];
    double c5 = 0.0, s5 = 0.0;
    if constexpr (sizeof(T) == 8) {
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

// complex128 with a generator whose entries are +-1 (A^2 = -I on its
// support S, A[q][r] = -A[r][q]): on each pair {r, q = r ^ x} of S the
// fifth-order series is c5 psi + s5 A psi, so
//   ||psi'||^2 = sum_{off S} |psi|^2 + (1 + g) sum_{S} |psi|^2,  g = c5^2 + s5^2 - 1,
// exactly, from the input state.  The norm is reduced first and the update
// and the rescale are then one pass, branch-free: each pair takes
// (C, S) = (sc c5, +-sc s5) on S and (sc, 0) off it (fma(0, psi_q, sc psi_r)
// is sc psi_r exactly), so a warp never runs both sides of a branch.
// 13 float64 operations per pair (squared norm with its weight, then the
// update) against about 20 for update, squared norm and rescale in turn: the
// float64 pipes of the cluster's 16 SMs bound this kernel.  Membership, signs
// and coefficients depend on indices only and are worked out before the
// wait for the previous grid.  Pairs are r (a zero inserted at x's highest
// bit) and q = r ^ x; a pair lies in S or outside it whole.
template <int PPT>
__global__ void __launch_bounds__(SINGLE_BS)
k_taylor5_single_closed(PoolView p, int k_imm, double th_imm, const DevStep* gate, double2* psi, int renorm,
                        double* norm2_out) {
    constexpr int NW = SINGLE_BS / 32;
    static_assert(NW == 8, "the partials' shuffle tree spans eight warps");
    __shared__ double red[NW];
    __shared__ double cta_part;
    __shared__ double slots[SINGLE_MAX_CLUSTER];
    __shared__ double coef_sh[3];    // c5, s5, 1 + g
    __shared__ double scale_sh[3];   // sc c5, sc s5, sc
    cg::cluster_group cl = cg::this_cluster();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (gate) asm volatile("griddepcontrol.wait;" ::: "memory");
    if (gate && gate->converged) return;
    const int k = gate ? gate->selected : k_imm;
    const double theta = gate ? gate->theta : th_imm;
    if (k < 0 || k >= p.M) {
        if (cl.block_rank() == 0 && threadIdx.x == 0 && norm2_out)
            *norm2_out = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    const bool need_norm = renorm || norm2_out;   // uniform
    if (need_norm) asm volatile("barrier.cluster.arrive;\n" ::: "memory");
    const SuppRec sr = load_supp(p, k);
    const uint32_t x = sr.x;
    const int c0neg = p.fc0f[k] < 0.0f;
    const int hb = 31 - __clz(x);
    const unsigned nb = cl.num_blocks(), rank = cl.block_rank();
    const uint32_t per = (uint32_t)(((1ll << p.nq) >> 1) / nb);
    uint32_t rr[PPT];
    bool ok[PPT], on[PPT], neg[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        const uint32_t i = j * SINGLE_BS + threadIdx.x;
        ok[j] = i < per;
        rr[j] = insert_zero(rank * per + i, hb);
        on[j] = in_support(sr, rr[j]);
        neg[j] = parity32((rr[j] ^ x) & sr.z0) != c0neg;   // A[r][q] = -1
    }
    if (threadIdx.x == 0) {
        double cf[6], c5, s5;
        taylor_coefs_fast<double>(theta, cf);
        closed_coefs(cf, c5, s5);
        const double t2 = theta * theta, t6 = t2 * t2 * t2;   // c5^2 + s5^2 - 1 in closed form
        coef_sh[0] = c5;
        coef_sh[1] = s5;
        coef_sh[2] = 1.0 + t6 * fma(t2, fma(t2, 1.0 / 14400.0, -1.0 / 960.0), 1.0 / 360.0);
    }
    if (!gate) asm volatile("griddepcontrol.wait;" ::: "memory");   // the state is the previous kernel's output
    double2 a[PPT], b[PPT];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        if (!ok[j]) continue;
        a[j] = psi[rr[j]];
        b[j] = psi[rr[j] ^ x];
    }
    __syncthreads();   // coef_sh
    if (need_norm) {
        const double won = coef_sh[2];
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            if (!ok[j]) continue;
            const double t = fma(a[j].x, a[j].x, fma(a[j].y, a[j].y, fma(b[j].x, b[j].x, b[j].y * b[j].y)));
            acc = fma(on[j] ? won : 1.0, t, acc);
        }
        acc = warp_sum(acc);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double w = threadIdx.x < NW ? red[threadIdx.x] : 0.0;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            if (threadIdx.x == 0) cta_part = w;
        }
        __syncthreads();
        asm volatile("barrier.cluster.wait;\n" ::: "memory");
        if (threadIdx.x < nb) *cl.map_shared_rank(&slots[rank], threadIdx.x) = cta_part;
        cl.sync();
    }
    if (threadIdx.x < 32) {
        // warp 0: the slots (at most 16) by a fixed shuffle tree, the same
        // in every CTA
        double t = need_norm && threadIdx.x < nb ? slots[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = SINGLE_MAX_CLUSTER / 2; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) {
            const double sc = renorm ? rsqrt(t) : 1.0;
            scale_sh[0] = sc * coef_sh[0];
            scale_sh[1] = sc * coef_sh[1];
            scale_sh[2] = sc;
            if (rank == 0 && norm2_out) *norm2_out = t;
        }
    }
    __syncthreads();
    const double C5 = scale_sh[0], S5 = scale_sh[1], sc = scale_sh[2];
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
        if (!ok[j] || (!on[j] && !renorm)) continue;
        const double C = on[j] ? C5 : sc;
        const double S = on[j] ? (neg[j] ? -S5 : S5) : 0.0;
        const double2 u = a[j], w = b[j];
        psi[rr[j]] = make_double2(fma(S, w.x, C * u.x), fma(S, w.y, C * u.y));
        psi[rr[j] ^ x] = make_double2(fma(-S, u.x, C * w.x), fma(-S, u.y, C * w.y));
    }
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

// attr: room for two attributes (the cluster shape and programmatic
// stream serialisation).
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
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cfg;
}

template <typename T, int UPT>
bool single_launchable_t(int csize) {
    auto kern = k_taylor5_single<T, UPT>;
    cudaError_t e = cudaSuccess;
    if (csize > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchAttribute attr[2];
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

// Cluster size and pairs per thread of the closed-form kernel: the fewest
// pairs per thread whose cluster fits; 0 when none does.
int closed_shape(int nq, int max_cluster, int* ppt_out) {
    if (nq < 1) return 0;
    const long long pairs = (1ll << nq) >> 1;
    for (int ppt = 1; ppt <= 8; ppt *= 2) {
        long long cs = (pairs + (long long)SINGLE_BS * ppt - 1) / ((long long)SINGLE_BS * ppt);
        if (cs < 1) cs = 1;
        if (cs <= max_cluster) {
            *ppt_out = ppt;
            return (int)cs;
        }
    }
    return 0;
}

template <int PPT>
bool closed_launchable_t(int csize) {
    auto kern = k_taylor5_single_closed<PPT>;
    cudaError_t e = cudaSuccess;
    if (csize > 8) e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = single_cfg(csize, 0, attr);
    int n = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) (void)cudaGetLastError();
    return e == cudaSuccess && n >= 1;
}

bool closed_launchable(int csize, int ppt) {
    switch (ppt) {
        case 1: return closed_launchable_t<1>(csize);
        case 2: return closed_launchable_t<2>(csize);
        case 4: return closed_launchable_t<4>(csize);
        case 8: return closed_launchable_t<8>(csize);
        default: return false;
    }
}

// Cluster size and pairs per thread that launch for this state size (cached
// per size), or false when none does.
bool closed_config(int nq, int* cs_out, int* ppt_out) {
    static int cache[32][2] = {};   // [nq] -> {cluster size, ppt}; -1 none
    if (nq < 1 || nq >= 32) return false;
    int* e = cache[nq];
    if (e[0] == 0) {
        e[0] = -1;
        for (int maxc = SINGLE_MAX_CLUSTER; maxc >= 1; maxc /= 2) {
            int ppt = 0;
            const int cs = closed_shape(nq, maxc, &ppt);
            if (cs == 0) break;
            if (closed_launchable(cs, ppt)) {
                e[0] = cs;
                e[1] = ppt;
                break;
            }
        }
    }
    if (e[0] < 0) return false;
    *cs_out = e[0];
    *ppt_out = e[1];
    return true;
}

template <int PPT>
cudaError_t launch_closed_t(const PoolView& p, int csize, int k, double theta, const DevStep* gate, void* psi,
                            int renorm, double* norm2, cudaStream_t s) {
    cudaLaunchAttribute attr[2];
    const cudaLaunchConfig_t cfg = single_cfg(csize, s, attr);
    return cudaLaunchKernelEx(&cfg, k_taylor5_single_closed<PPT>, p, k, theta, gate, static_cast<double2*>(psi),
                              renorm, norm2);
}

cudaError_t dispatch_closed(const PoolView& p, int csize, int ppt, int k, double theta, const DevStep* gate,
                            void* psi, int renorm, double* norm2, cudaStream_t s) {
    switch (ppt) {
        case 1: return launch_closed_t<1>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        case 2: return launch_closed_t<2>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        case 4: return launch_closed_t<4>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        case 8: return launch_closed_t<8>(p, csize, k, theta, gate, psi, renorm, norm2, s);
        default: return cudaErrorInvalidConfiguration;
    }
}

template <typename T, int UPT>
cudaError_t launch_single_t(const PoolView& p, int csize, int k, double theta, const DevStep* gate, void* psi,
                            int renorm, double* norm2, cudaStream_t s) {
    using V = typename C2<T>::type;
    cudaLaunchAttribute attr[2];
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

int launch_taylor5_single(const PoolView& p, int prec, bool unit_pool, int k, double theta, const DevStep* gate,
                          void* psi, int renorm, double* norm2, cudaStream_t s) {
    int cs = 0, upt = 0;
    if (prec == TQ_C128 && unit_pool && closed_config(p.nq, &cs, &upt)) {
        const cudaError_t e = dispatch_closed(p, cs, upt, k, theta, gate, psi, renorm, norm2, s);
        return e == cudaSuccess ? 1 : -1;
    }
    if (!single_config(p.nq, prec, &cs, &upt)) return -1;
    const cudaError_t e = prec == TQ_C128
                              ? dispatch_single<double>(p, cs, upt, k, theta, gate, psi, renorm, norm2, s)
                              : dispatch_single<float>(p, cs, upt, k, theta, gate, psi, renorm, norm2, s);
    return e == cudaSuccess ? 1 : -1;
}

}  // namespace tq
