// Kernels of the adjoint sweep for ADAPT-VQE with re-optimised angles (a
// standard extension of the paper's loop, Sec. III-D, which updates only the
// newest angle).  The ansatz is the product of the Taylor-5 factors of
// Eqs. (6)-(8); its energy gradient needs, per factor,
//   <chi | U'(theta) phi>,  U'(theta) = A sum_{m<=4} (theta A)^m / m!,
// and every pool generator has A^2 = -P (P: the rows A does not
// annihilate), so U'(theta) = c4 A - s4 P with c4 = 1 - theta^2/2 +
// theta^4/24 and s4 = theta - theta^3/6.
#include "dev.cuh"

namespace tq {

namespace {

__device__ __forceinline__ bool last_block_vqe(unsigned* ticket, unsigned nblocks) {
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == nblocks - 1;
    }
    __syncthreads();
    return is_last;
}

template <typename T>
__device__ __forceinline__ double cdot_re(typename C2<T>::type a, typename C2<T>::type b) {
    return (double)a.x * (double)b.x + (double)a.y * (double)b.y;
}

// Re<chi | (c4 A - s4 P) phi> over all rows, float64 sums in a fixed order
// (per block, then the last block over the block partials); writes
// 2 * sum / e_den.  Full-space pools read A's entries from the factored sign
// form, sector pools from their (column, sign) tables.
template <typename T>
__global__ void __launch_bounds__(256)
k_ansatz_dot(PoolView p, int k, double c4, double s4, const typename C2<T>::type* __restrict__ chi,
             const typename C2<T>::type* __restrict__ phi, long long D, double* partials, unsigned* ticket,
             const DevStep* step, double* out) {
    __shared__ double sh[8];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < D; r += stride) {
        long long c;
        double a;
        if (p.sdim) {
            a = (double)p.ssgn[(long long)k * p.sdim + r];
            c = p.scol[(long long)k * p.sdim + r];
        } else {
            c = r ^ (long long)p.x[k];
            a = op_value<double>(p, k, (uint32_t)c);
        }
        if (a != 0.0) acc += c4 * a * cdot_re<T>(chi[r], phi[c]) - s4 * cdot_re<T>(chi[r], phi[r]);
    }
    double v[1] = {acc};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
    if (last_block_vqe(ticket, gridDim.x)) {
        double t = 0.0;
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(partials + i);
        double u[1] = {t};
        block_sum<1>(u, sh);
        if (threadIdx.x == 0) {
            *out = 2.0 * u[0] / step->e_den;
            *ticket = 0u;
        }
    }
}

// chi = w - E psi (E from the step record), in the state's precision.
template <typename T>
__global__ void k_residual(const double2* __restrict__ w, const typename C2<T>::type* __restrict__ psi,
                           typename C2<T>::type* __restrict__ chi, long long D, const DevStep* step) {
    const double E = step->energy;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < D; r += stride) {
        const double2 wr = w[r];
        const typename C2<T>::type pr = psi[r];
        chi[r] = {(T)(wr.x - E * (double)pr.x), (T)(wr.y - E * (double)pr.y)};
    }
}

int small_grid(long long D, int sms) {
    long long g = (D + 255) / 256;
    if (g > (long long)sms * 4) g = (long long)sms * 4;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_ansatz_dot(const PoolView& p, int k, double c4, double s4, const void* chi, const void* phi, int prec,
                      long long D, double* partials, unsigned* ticket, const DevStep* step, double* grad_out,
                      int sms, cudaStream_t s) {
    const int grid = small_grid(D, sms);
    if (prec == TQ_C128)
        k_ansatz_dot<double><<<grid, 256, 0, s>>>(p, k, c4, s4, static_cast<const double2*>(chi),
                                                  static_cast<const double2*>(phi), D, partials, ticket, step, grad_out);
    else
        k_ansatz_dot<float><<<grid, 256, 0, s>>>(p, k, c4, s4, static_cast<const float2*>(chi),
                                                 static_cast<const float2*>(phi), D, partials, ticket, step, grad_out);
    return 1;
}

int launch_residual(const double2* w, const void* psi, void* chi, int prec, long long D, const DevStep* step,
                    cudaStream_t s) {
    const int grid = (int)((D + 255) / 256 < 2048 ? (D + 255) / 256 : 2048);
    if (prec == TQ_C128)
        k_residual<double><<<grid, 256, 0, s>>>(w, static_cast<const double2*>(psi), static_cast<double2*>(chi), D, step);
    else
        k_residual<float><<<grid, 256, 0, s>>>(w, static_cast<const float2*>(psi), static_cast<float2*>(chi), D, step);
    return 1;
}

}  // namespace tq
