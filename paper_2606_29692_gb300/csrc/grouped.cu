// Support-only batched Taylor-5 update for groups of states that share a
// generator (Sec. III-C, Eqs. (6)-(8)), in an interleaved layout.
//
// The support-only update reads and writes a generator's support S, and
// DRAM moves 32-byte sectors.  With one state per contiguous vector a
// sector holds 4 consecutive complex64 amplitudes of one state, and S
// fills only part of the sectors it touches.  Here G states that take the
// same generator (G = 4 complex64, 2 complex128: 32 bytes) are stored
// amplitude-major within their group: element (g, r, s) -- group g,
// amplitude r, state s < G -- sits at (g D + r) G + s.  A support row of
// the group is then one whole sector holding that row of all G states, so
// every touched sector is used in full.  Each state keeps its own angle and
// its own carried float64 squared norm; the products are those of the
// per-state support update (complex64: the packed float32 chain;
// complex128: the closed form c5 psi + s5 A psi on pairs with entries +-1),
// so each state's amplitudes equal what that update gives it.
//
// L lanes share a row (L = 1, 2 or G), each holding G / L of its states:
// one lane per row expands each support row once but carries every
// state's coefficients and amplitudes (many registers, few resident
// warps); more lanes per row repeat the row expansion but hold fewer
// registers, so more warps and loads are in flight per SM.
#include "dev.cuh"
#include "grad.cuh"
#include "pair.cuh"

namespace tq {

namespace {

constexpr int GR_BS = 256;
constexpr int GR_NW = GR_BS / 32;

template <typename T> struct GroupSize;
template <> struct GroupSize<float> { static constexpr int value = 4; };
template <> struct GroupSize<double> { static constexpr int value = 2; };

// SPL consecutive amplitudes of one row (SPL states of the group), moved
// with 16-byte accesses.
template <typename V, int SPL>
struct Slice {
    V a[SPL];
    __device__ __forceinline__ void load(const V* p) {
        if constexpr (sizeof(V) == 8 && SPL >= 2) {
#pragma unroll
            for (int i = 0; i < SPL / 2; ++i) {
                const float4 u = reinterpret_cast<const float4*>(p)[i];
                a[2 * i] = make_float2(u.x, u.y);
                a[2 * i + 1] = make_float2(u.z, u.w);
            }
        } else {
#pragma unroll
            for (int i = 0; i < SPL; ++i) a[i] = p[i];
        }
    }
    __device__ __forceinline__ void store(V* p) const {
        if constexpr (sizeof(V) == 8 && SPL >= 2) {
#pragma unroll
            for (int i = 0; i < SPL / 2; ++i)
                reinterpret_cast<float4*>(p)[i] = make_float4(a[2 * i].x, a[2 * i].y, a[2 * i + 1].x, a[2 * i + 1].y);
        } else {
#pragma unroll
            for (int i = 0; i < SPL; ++i) p[i] = a[i];
        }
    }
};

// c5^2 + s5^2 - 1 of the fifth-order series for A^2 = -I:
// theta^6/360 - theta^8/960 + theta^10/14400.
__device__ __forceinline__ double grouped_growth(double theta) {
    const double t2 = theta * theta, t6 = t2 * t2 * t2;
    return t6 * fma(t2, fma(t2, 1.0 / 14400.0, -1.0 / 960.0), 1.0 / 360.0);
}

template <typename T, int L>
constexpr int grouped_min_blocks() {
    return L == 1 ? 2 : (sizeof(T) == 4 ? (L == 2 ? 3 : 4) : 3);
}

// Persistent grid over groups.  kk: op index per group; th, norm2: per
// state (G per group; norm2 may be null).  A group's op index outside
// [0, M) leaves its states untouched and makes their norms NaN.
template <typename T, int PPT, int L>
__global__ void __launch_bounds__(GR_BS, grouped_min_blocks<T, L>())
k_taylor5_grouped(PoolView p, int n_groups, typename C2<T>::type* psi, const int* kk, const double* th,
                  double* norm2) {
    using V = typename C2<T>::type;
    constexpr int G = GroupSize<T>::value;
    constexpr int SPL = G / L;                    // states per lane
    constexpr uint32_t PB = GR_BS / L;            // pairs per sweep of the CTA
    __shared__ double red[2][GR_NW][G];           // per warp and state; complex64: (hi, lo) float pairs
    int rp = 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s0 = (threadIdx.x % L) * SPL;       // this lane's first state
    const uint32_t slot = threadIdx.x / L;
    const long long D = 1ll << p.nq;
    for (int g = blockIdx.x; g < n_groups; g += gridDim.x) {
        const int k = kk[g];
        const bool bad = k < 0 || k >= p.M;
        T delta[SPL];
#pragma unroll
        for (int j = 0; j < SPL; ++j) delta[j] = T(0);
        if (!bad) {
            T cf[SPL][6];
            double c5[SPL], s5[SPL], nsq[SPL];
#pragma unroll
            for (int j = 0; j < SPL; ++j) {
                taylor_coefs_fast<T>(th[(long long)g * G + s0 + j], cf[j]);
                c5[j] = s5[j] = nsq[j] = 0.0;
                if constexpr (sizeof(T) == 8) closed_coefs(cf[j], c5[j], s5[j]);
            }
            const SuppRec sr = load_supp(p, k);
            const RowExp rx = make_rowexp(sr, p.supp[k].z);
            const uint32_t x = sr.x, z0 = sr.z0;
            const T c0 = sizeof(T) == 4 ? (T)p.fc0f[k] : (T)p.fc0d[k];
            const bool unit = fabsf(p.fc0f[k]) == 1.0f;
            const bool c0neg = p.fc0f[k] < 0.0f;
            const uint32_t P = 1u << (p.nq - sr.m - 1);
            V* base = psi + (long long)g * D * G + s0;
            for (uint32_t i0 = slot; i0 < P; i0 += PB * PPT) {
                Slice<V, SPL> A[PPT], B[PPT];
                uint32_t rr[PPT];
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint32_t u = i0 + j * PB;
                    if (u >= P) continue;
                    const uint32_t r = expand_row(rx, u);
                    rr[j] = r;
                    A[j].load(base + (long long)r * G);
                    B[j].load(base + (long long)(r ^ x) * G);
                }
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    if (i0 + j * PB >= P) continue;
                    const uint32_t r = rr[j], q = r ^ x;
                    const int nr = parity32(q & z0), nq = parity32(r & z0);   // signs of A[r][q], A[q][r]
#pragma unroll
                    for (int t = 0; t < SPL; ++t) {
                        V ar = A[j].a[t], aq = B[j].a[t];
                        bool closed = false;
                        if constexpr (sizeof(T) == 8) {
                            if (unit && nr != nq) {
                                const int sgn = (nr != (int)c0neg) ? -1 : 1;
                                closed_pair_sign(sgn, -sgn, cf[t], c5[t], s5[t], ar, aq);
                                closed = true;
                                const V a = A[j].a[t], b = B[j].a[t];
                                nsq[t] = fma(a.x, a.x, fma(a.y, a.y, fma(b.x, b.x, fma(b.y, b.y, nsq[t]))));
                            }
                        }
                        if (!closed) {
                            chain_pair(nr ? -c0 : c0, nq ? -c0 : c0, cf[t], ar, aq);
                            const V a = A[j].a[t], b = B[j].a[t];
                            delta[t] += (ar.x - a.x) * (ar.x + a.x) + (ar.y - a.y) * (ar.y + a.y);
                            delta[t] += (aq.x - b.x) * (aq.x + b.x) + (aq.y - b.y) * (aq.y + b.y);
                        }
                        A[j].a[t] = ar;
                        B[j].a[t] = aq;
                    }
                    A[j].store(base + (long long)r * G);
                    B[j].store(base + (long long)q * G);
                }
            }
            if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int t = 0; t < SPL; ++t) delta[t] += grouped_growth(th[(long long)g * G + s0 + t]) * nsq[t];
            }
        }
        // the warp's partial per state: a shuffle tree over the lanes that
        // hold the same states (offsets >= L keep lane % L), after which
        // lanes 0..L-1 hold states lane * SPL + t
#pragma unroll
        for (int t = 0; t < SPL; ++t) {
            if constexpr (sizeof(T) == 4) {
                float hi = delta[t], lo = 0.f;
#pragma unroll
                for (int o = 16; o >= L; o >>= 1) {
                    const float oh = __shfl_down_sync(0xffffffffu, hi, o);
                    const float ol = __shfl_down_sync(0xffffffffu, lo, o);
                    float sum, err;
                    two_sum(hi, oh, sum, err);
                    hi = sum;
                    lo = lo + ol + err;
                }
                if (lane < L)
                    *reinterpret_cast<float2*>(&red[rp][warp][lane * SPL + t]) =
                        bad ? make_float2(__int_as_float(0x7fc00000), 0.f) : make_float2(hi, lo);
            } else {
                double v = delta[t];
#pragma unroll
                for (int o = 16; o >= L; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane < L) red[rp][warp][lane * SPL + t] = bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
            }
        }
        __syncthreads();
        // warp 0: lane w * G + st holds warp w's partial of state st, then a
        // fixed shuffle tree over the warps
        if (warp == 0) {
            const int w = lane / G, st = lane % G;
            if constexpr (sizeof(T) == 4) {
                float hi = 0.f, lo = 0.f;
                if (w < GR_NW) {
                    const float2 hl = *reinterpret_cast<const float2*>(&red[rp][w][st]);
                    hi = hl.x;
                    lo = hl.y;
                }
#pragma unroll
                for (int o = 16; o >= G; o >>= 1) {
                    const float oh = __shfl_down_sync(0xffffffffu, hi, o);
                    const float ol = __shfl_down_sync(0xffffffffu, lo, o);
                    float sum, err;
                    two_sum(hi, oh, sum, err);
                    hi = sum;
                    lo = lo + ol + err;
                }
                if (lane < G && norm2) norm2[(long long)g * G + lane] += (double)hi + (double)lo;
            } else {
                double v = w < GR_NW ? red[rp][w][st] : 0.0;
#pragma unroll
                for (int o = 16; o >= G; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (lane < G && norm2) norm2[(long long)g * G + lane] += v;
            }
        }
        rp ^= 1;
    }
}

template <typename T, int PPT, int L>
int launch_grouped_t(const PoolView& p, int n_groups, void* psi, const int* k, const double* theta, double* norm2,
                     int sms, cudaStream_t s) {
    using V = typename C2<T>::type;
    static int per_sm = 0;
    if (per_sm == 0) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_taylor5_grouped<T, PPT, L>, GR_BS, 0);
        per_sm = n < 1 ? 1 : n;
    }
    long long grid = (long long)per_sm * sms;
    if (grid > n_groups) grid = n_groups;
    if (grid < 1) grid = 1;
    k_taylor5_grouped<T, PPT, L><<<(int)grid, GR_BS, 0, s>>>(p, n_groups, static_cast<V*>(psi), k, theta, norm2);
    return 1;
}

template <typename T, int L>
int dispatch_ppt(int ppt, const PoolView& p, int n_groups, void* psi, const int* k, const double* theta,
                 double* norm2, int sms, cudaStream_t s) {
    switch (ppt) {
        case 1: return launch_grouped_t<T, 1, L>(p, n_groups, psi, k, theta, norm2, sms, s);
        case 2: return launch_grouped_t<T, 2, L>(p, n_groups, psi, k, theta, norm2, sms, s);
        case 4: return launch_grouped_t<T, 4, L>(p, n_groups, psi, k, theta, norm2, sms, s);
        default: return -1;
    }
}

}  // namespace

int grouped_size(int prec) { return prec == TQ_C128 ? 2 : 4; }

bool grouped_schedule_ok(int prec, int lanes, int ppt) {
    const bool lanes_ok = lanes == 1 || lanes == 2 || (lanes == 4 && prec != TQ_C128);
    return lanes_ok && (ppt == 1 || ppt == 2 || ppt == 4);
}

int launch_taylor5_grouped(const PoolView& p, int n_groups, int prec, int lanes, int ppt, void* psi, const int* k,
                           const double* theta, double* norm2, int sms, cudaStream_t s) {
    if (prec == TQ_C128) {
        if (lanes == 1) return dispatch_ppt<double, 1>(ppt, p, n_groups, psi, k, theta, norm2, sms, s);
        if (lanes == 2) return dispatch_ppt<double, 2>(ppt, p, n_groups, psi, k, theta, norm2, sms, s);
        return -1;
    }
    if (lanes == 1) return dispatch_ppt<float, 1>(ppt, p, n_groups, psi, k, theta, norm2, sms, s);
    if (lanes == 2) return dispatch_ppt<float, 2>(ppt, p, n_groups, psi, k, theta, norm2, sms, s);
    if (lanes == 4) return dispatch_ppt<float, 4>(ppt, p, n_groups, psi, k, theta, norm2, sms, s);
    return -1;
}

}  // namespace tq
