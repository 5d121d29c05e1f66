// Device code of the fused Taylor-5 pair update (Sec. III-C, Eqs. (6)-(8)),
// shared by the single, batched and trajectory-batch kernels.
#pragma once

#include "dev.cuh"

namespace tq {

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
__device__ __forceinline__ void taylor_coefs_typed(T t, T (&cf)[6]) {
    const T t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    cf[0] = T(1);
    cf[1] = t;
    cf[2] = t2 * T(0.5);
    cf[3] = t3 * T(1.0 / 6.0);
    cf[4] = t4 * T(1.0 / 24.0);
    cf[5] = t5 * T(1.0 / 120.0);
}
template <typename T>
__device__ __forceinline__ void taylor_coefs_fast(double theta, T (&cf)[6]) {
    taylor_coefs_typed<T>((T)theta, cf);
}

// c5 = cf0 - cf2 + cf4 and s5 = cf1 - cf3 + cf5 (the closed form below) with
// additions the compiler may not fuse with the products inside cf, so every
// kernel that uses them gets the same bits.
__device__ __forceinline__ void closed_coefs(const double (&cf)[6], double& c5, double& s5) {
    c5 = __dadd_rn(__dsub_rn(cf[0], cf[2]), cf[4]);
    s5 = __dadd_rn(__dsub_rn(cf[1], cf[3]), cf[5]);
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

// Fixed-order float64 sum of a CTA's warp partials (complex64: (hi, lo)
// float pairs in the 8-byte slots).
template <typename T, int NW>
__device__ __forceinline__ double sum_partials(const double* red) {
    double sum = 0.0;
    for (int w = 0; w < NW; ++w) {
        if constexpr (sizeof(T) == 4) {
            const float2 hl = *reinterpret_cast<const float2*>(&red[w]);
            sum += (double)hl.x + (double)hl.y;
        } else {
            sum += red[w];
        }
    }
    return sum;
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
    int unit;     // |c0| == 1: every entry of A is 0 or +-1
    int c0neg;    // c0 < 0
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
    o.unit = fabsf(p.fc0f[k]) == 1.0f;
    o.c0neg = p.fc0f[k] < 0.0f;
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

// Entry of A as an integer -1, 0, +1 (valid when op.unit).
template <typename T>
__device__ __forceinline__ int rec_sign(const OpRec<T>& o, int code) {
    if ((code & 7) != o.t) return 0;
    return ((code & 8) != 0) != (o.c0neg != 0) ? -1 : 1;
}

// s * v for s in {-1, 0, +1} with integer masks on the float64 bit
// patterns: bit-identical to the float64 product, and no float64
// instruction (this part issues float64 at about 1/57 of float32).
__device__ __forceinline__ double2 sign_apply(int s, double2 v) {
    const unsigned long long keep = s != 0 ? ~0ull : 0ull;
    const unsigned long long flip = s < 0 ? 0x8000000000000000ull : 0ull;
    return make_double2(__longlong_as_double((__double_as_longlong(v.x) & keep) ^ flip),
                        __longlong_as_double((__double_as_longlong(v.y) & keep) ^ flip));
}

// The five-product chain of complex128 pairs with entries of A in
// {-1, 0, +1}: only the accumulation uses the float64 pipe.
__device__ __forceinline__ void chain_pair_sign(int s_r, int s_q, const double (&cf)[6], double2& ar,
                                                double2& aq) {
    double2 vr = ar, vq = aq;
#pragma unroll
    for (int k = 1; k <= 5; ++k) {
        const double2 nr = sign_apply(s_r, vq);
        const double2 nq = sign_apply(s_q, vr);
        vr = nr;
        vq = nq;
        ar.x = fma(cf[k], vr.x, ar.x);
        ar.y = fma(cf[k], vr.y, ar.y);
        aq.x = fma(cf[k], vq.x, aq.x);
        aq.y = fma(cf[k], vq.y, aq.y);
    }
}

template <typename T>
__device__ __forceinline__ int base_code(const OpRec<T>& o, uint32_t r) {
    return parity32(r & o.d0) | (parity32(r & o.d1) << 1) | (parity32(r & o.d2) << 2) |
           (parity32(r & o.z0) << 3);
}

// One tile of the pair update: units tl*TU .. tl*TU+TU-1 of a state at
// `base` (4 amplitudes per unit), generator `op`, angle theta.  Loads every
// unit of the thread first, then runs the five-product chains and stores.
// Returns the thread's float32 (complex64) or float64 sum of |psi'|^2.
// The same five products and sum in closed form for complex128 pairs whose
// 2x2 block of A is [[0, s], [-s, 0]], s = +-1 (every pool generator's, on
// its support): there A^2 = -I, so sum_k (theta A)^k / k! = c5 I + s5 A
// with c5 = cf0 - cf2 + cf4 and s5 = cf1 - cf3 + cf5; a pair A annihilates
// keeps psi.  Half the float64 work of the explicit chain, which still runs
// for any other sign pattern.
__device__ __forceinline__ void closed_pair_sign(int s_r, int s_q, const double (&cf)[6], double c5, double s5,
                                                 double2& ar, double2& aq) {
    if (s_r != 0 && s_q == -s_r) {
        const double2 tq = sign_apply(s_r, aq), tr = sign_apply(s_q, ar);
        const double2 vr = ar, vq = aq;
        ar = make_double2(fma(s5, tq.x, c5 * vr.x), fma(s5, tq.y, c5 * vr.y));
        aq = make_double2(fma(s5, tr.x, c5 * vq.x), fma(s5, tr.y, c5 * vq.y));
    } else if (s_r != 0 || s_q != 0) {
        chain_pair_sign(s_r, s_q, cf, ar, aq);
    }
}

// Four amplitudes of one unit of the pair enumeration: rows r0, r0 + 1 and
// their partners q0 = r0 ^ x, q0 ^ 1 (x > 1), or pairs (r0, r0 + 1) and
// (r0 + 2, r0 + 3) (x == 1).  After unit_update, a0/a1 hold rows r0/r0 + 1
// and b0/b1 rows q0/q0 ^ 1 (x > 1), or a0, b0, a1, b1 rows r0..r0 + 3.
template <typename V>
struct PairUnit {
    uint32_t r0;
    V a0, a1, b0, b1;
};

// Loads unit u (two aligned 2-element vectors).  hb: highest set bit of x.
template <typename V>
__device__ __forceinline__ void unit_load(const V* base, uint32_t x, int hb, uint32_t u, PairUnit<V>& w) {
    if (hb > 0) {
        const uint32_t r0 = insert_zero(2u * u, hb);
        w.r0 = r0;
        V f0, f1;
        load2(base, r0, w.a0, w.a1);
        load2(base, (r0 ^ x) & ~1u, f0, f1);
        const uint32_t q0 = r0 ^ x;
        w.b0 = (q0 & 1u) ? f1 : f0;   // psi[q0]
        w.b1 = (q0 & 1u) ? f0 : f1;   // psi[q0 ^ 1]
    } else {
        const uint32_t r0 = 4u * u;
        w.r0 = r0;
        load2(base, r0, w.a0, w.b0);
        load2(base, r0 + 2u, w.a1, w.b1);
    }
}

template <typename V>
__device__ __forceinline__ void unit_store(V* base, uint32_t x, int hb, const PairUnit<V>& w) {
    if (hb > 0) {
        const uint32_t q0 = w.r0 ^ x;
        store2(base, w.r0, w.a0, w.a1);
        if (q0 & 1u) store2(base, q0 & ~1u, w.b1, w.b0);
        else store2(base, q0 & ~1u, w.b0, w.b1);
    } else {
        store2(base, w.r0, w.a0, w.b0);
        store2(base, w.r0 + 2u, w.a1, w.b1);
    }
}

// The five products and the running sum (Eqs. (7)-(8)) on the unit's two
// pairs, in place; adds |psi'|^2 of its four amplitudes to tpart.
template <typename T>
__device__ __forceinline__ void unit_update(const OpRec<T>& op, int hb, const T (&cf)[6], double c5, double s5,
                                            PairUnit<typename C2<T>::type>& w, T& tpart);

template <typename T>
__device__ __forceinline__ void unit_update(const OpRec<T>& op, int hb, const T (&cf)[6],
                                            PairUnit<typename C2<T>::type>& w, T& tpart) {
    double c5 = 0.0, s5 = 0.0;
    if constexpr (sizeof(T) == 8) closed_coefs(cf, c5, s5);
    unit_update<T>(op, hb, cf, c5, s5, w, tpart);
}

// The same with the closed-form coefficients c5, s5 given (complex128).
template <typename T>
__device__ __forceinline__ void unit_update(const OpRec<T>& op, int hb, const T (&cf)[6], double c5, double s5,
                                            PairUnit<typename C2<T>::type>& w, T& tpart) {
    const uint32_t r0 = w.r0;
    if (hb > 0) {
        // rows r0, r0+1 and partners q0 = r0^x, q0^1; their columns are
        // r0 ^ {x, x^1, 0, 1}
        const int bc = base_code(op, r0);
        const int c_r0 = bc ^ ((op.dcode >> 8) & 15);    // col q0
        const int c_r1 = bc ^ ((op.dcode >> 12) & 15);   // col q0^1
        const int c_q0 = bc ^ (op.dcode & 15);           // col r0
        const int c_q1 = bc ^ ((op.dcode >> 4) & 15);    // col r0+1
        if constexpr (sizeof(T) == 8) {
            if (op.unit) {
                closed_pair_sign(rec_sign(op, c_r0), rec_sign(op, c_q0), cf, c5, s5, w.a0, w.b0);
                closed_pair_sign(rec_sign(op, c_r1), rec_sign(op, c_q1), cf, c5, s5, w.a1, w.b1);
            } else {
                chain_pair(rec_value(op, c_r0), rec_value(op, c_q0), cf, w.a0, w.b0);
                chain_pair(rec_value(op, c_r1), rec_value(op, c_q1), cf, w.a1, w.b1);
            }
        } else {
            chain_pair(rec_value(op, c_r0), rec_value(op, c_q0), cf, w.a0, w.b0);
            chain_pair(rec_value(op, c_r1), rec_value(op, c_q1), cf, w.a1, w.b1);
        }
        tpart += w.a0.x * w.a0.x + w.a0.y * w.a0.y + w.a1.x * w.a1.x + w.a1.y * w.a1.y;
        tpart += w.b0.x * w.b0.x + w.b0.y * w.b0.y + w.b1.x * w.b1.x + w.b1.y * w.b1.y;
    } else {
        // x == 1: pairs (r0, r0+1) and (r0+2, r0+3)
        const int b0c = base_code(op, r0), b2c = base_code(op, r0 + 2u);
        const T s_r0 = rec_value(op, b0c ^ ((op.dcode >> 4) & 15));  // col r0+1
        const T s_q0 = rec_value(op, b0c);                           // col r0
        const T s_r1 = rec_value(op, b2c ^ ((op.dcode >> 4) & 15));  // col r0+3
        const T s_q1 = rec_value(op, b2c);                           // col r0+2
        chain_pair(s_r0, s_q0, cf, w.a0, w.b0);
        chain_pair(s_r1, s_q1, cf, w.a1, w.b1);
        tpart += w.a0.x * w.a0.x + w.a0.y * w.a0.y + w.b0.x * w.b0.x + w.b0.y * w.b0.y;
        tpart += w.a1.x * w.a1.x + w.a1.y * w.a1.y + w.b1.x * w.b1.x + w.b1.y * w.b1.y;
    }
}

template <typename T, int UPT>
__device__ __forceinline__ T pair_tile(const OpRec<T>& op, double theta,
                                       typename C2<T>::type* base, uint32_t tl, uint32_t units) {
    using V = typename C2<T>::type;
    constexpr int TU = PAIR_BS * UPT;
    T cf[6];
    taylor_coefs_fast<T>(theta, cf);
    const uint32_t x = op.x;
    const int hb = 31 - __clz(x);
    PairUnit<V> w[UPT];
    bool ok[UPT];
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
        const uint32_t u = (uint32_t)tl * TU + j * PAIR_BS + threadIdx.x;
        ok[j] = u < units;
        if (ok[j]) unit_load(base, x, hb, u, w[j]);
    }
    T tpart = T(0);
#pragma unroll
    for (int j = 0; j < UPT; ++j) {
        if (!ok[j]) continue;
        unit_update<T>(op, hb, cf, w[j], tpart);
        unit_store(base, x, hb, w[j]);
    }
    return tpart;
}

}  // namespace tq
