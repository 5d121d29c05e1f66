// Pauli sum -> CSR compilation on the GPU (Sec. III-E step 3, "on-the-fly
// sparse compilation"), and basis-state initialisation.
//
// The operator is a sum of X-mask groups.  Row r of group x has exactly one
// candidate column, r ^ x, whose value is the group's term sum
//   v = sum_{p in group} c_p (-1)^{popcount((r ^ x) & z_p)}
// taken in the canonical (x, z) order.  Three passes:
//   count : one warp per row, lanes over groups, counts |v| > tol;
//   scan  : exclusive prefix sum -> rowptr (int64 accumulate, overflow check);
//   fill  : one warp per row recomputes the kept entries, compacts them into
//           shared memory with a ballot, sorts them by column (bitonic
//           network over the next power of two) and writes them.
// The X-mask 0 group (the diagonal) is kept apart in a float64 array.
//
// In a sector (h.sq, h.sect set) row r stands for qubit index h.sq[r] and
// the column of qubit index c is its sector rank; columns outside the
// sector (rank -1) are skipped.
#include "dev.cuh"
#include "sector.cuh"

#include <climits>

namespace tq {

namespace {

__device__ __forceinline__ double group_value(const HamView& h, int g, uint32_t col) {
    double v = 0.0;
    const int e = h.goff[g + 1];
    for (int t = h.goff[g]; t < e; ++t) {
        const double c = h.tc[t];
        v += parity32(col & h.tz[t]) ? -c : c;
    }
    return v;
}

__device__ __forceinline__ uint32_t row_index(const HamView& h, long long r) {
    return h.sq ? h.sq[r] : (uint32_t)r;
}
__device__ __forceinline__ long long col_position(const HamView& h, uint32_t c) {
    return h.sect ? sector_rank(c, *h.sect) : (long long)c;
}

__global__ void k_csr_count(HamView h, double tol, double amb_hi, int* counts,
                            unsigned long long* n_amb) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = warp; r < h.D; r += nwarps) {
        const uint32_t e = row_index(h, r);
        int cnt = 0, amb = 0;
        for (int g = lane; g < h.G; g += 32) {
            const uint32_t c = e ^ h.gx[g];
            if (col_position(h, c) < 0) continue;
            const double a = fabs(group_value(h, g, c));
            cnt += a > tol;
            amb += (a > tol) & (a <= amb_hi);
        }
        cnt = warp_sum_int(cnt);
        amb = warp_sum_int(amb);
        if (lane == 0) {
            counts[r] = cnt;
            if (amb) atomicAdd(n_amb, (unsigned long long)amb);
        }
    }
}

__global__ void k_diag(HamView h, double* diag) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < h.D; r += stride) {
        const uint32_t e = row_index(h, r);
        double v = 0.0;
        for (int t = 0; t < h.Kd; ++t) {
            const double c = h.dc[t];
            v += parity32(e & h.dz[t]) ? -c : c;
        }
        diag[r] = v;
    }
}

// Single-CTA exclusive scan: thread t owns a contiguous segment.
__global__ void k_scan(const int* counts, long long D, int* rowptr, long long* total,
                       int* max_row) {
    __shared__ long long part[1024];
    __shared__ int mx[1024];
    const int t = threadIdx.x, nt = blockDim.x;
    const long long seg = (D + nt - 1) / nt;
    const long long lo = t * seg, hi = lo + seg < D ? lo + seg : D;
    long long s = 0;
    int m = 0;
    for (long long i = lo; i < hi; ++i) {
        s += counts[i];
        m = counts[i] > m ? counts[i] : m;
    }
    part[t] = s;
    mx[t] = m;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        int mm = 0;
        for (int i = 0; i < nt; ++i) {
            const long long v = part[i];
            part[i] = run;
            run += v;
            mm = mx[i] > mm ? mx[i] : mm;
        }
        *total = run;
        *max_row = mm;
        if (run <= INT_MAX) rowptr[D] = (int)run;
    }
    __syncthreads();
    long long run = part[t];
    for (long long i = lo; i < hi; ++i) {
        if (run <= INT_MAX) rowptr[i] = (int)run;
        run += counts[i];
    }
}

template <typename VT>
__global__ void k_csr_fill(HamView h, double tol, int cap, int* col, VT* val) {
    extern __shared__ unsigned char smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t* skey = reinterpret_cast<uint32_t*>(smem) + (size_t)wid * cap;
    double* sval = reinterpret_cast<double*>(reinterpret_cast<uint32_t*>(smem) +
                                             (size_t)(blockDim.x >> 5) * cap) + (size_t)wid * cap;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = warp; r < h.D; r += nwarps) {
        const int start = h.rowptr[r];
        const int n = h.rowptr[r + 1] - start;
        if (n == 0) continue;
        const uint32_t e = row_index(h, r);
        int base = 0;
        for (int g0 = 0; g0 < h.G; g0 += 32) {
            const int g = g0 + lane;
            uint32_t c = 0;
            double v = 0.0;
            bool keep = false;
            if (g < h.G) {
                const uint32_t cq = e ^ h.gx[g];
                const long long pos = col_position(h, cq);
                if (pos >= 0) {
                    c = (uint32_t)pos;
                    v = group_value(h, g, cq);
                    keep = fabs(v) > tol;
                }
            }
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const int pos = base + __popc(ball & ((1u << lane) - 1u));
                skey[pos] = c;
                sval[pos] = v;
            }
            base += __popc(ball);
        }
        int P = 1;
        while (P < n) P <<= 1;
        for (int i = n + lane; i < P; i += 32) skey[i] = 0xffffffffu;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1) {
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int i = lane; i < P; i += 32) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const bool up = (i & k) == 0;
                        const uint32_t a = skey[i], b = skey[ixj];
                        if ((a > b) == up) {
                            skey[i] = b;
                            skey[ixj] = a;
                            const double tv = sval[i];
                            sval[i] = sval[ixj];
                            sval[ixj] = tv;
                        }
                    }
                }
                __syncwarp();
            }
        }
        for (int i = lane; i < n; i += 32) {
            col[start + i] = (int)skey[i];
            val[start + i] = (VT)sval[i];
        }
        __syncwarp();
    }
}

// XOR-ELL of the off-diagonal part (a second layout of the same entries):
// rows in blocks of XELL_ROWS = 8 (block R holds rows 8R .. 8R + 7).  For
// every X-mask group with a kept entry in any row of the block there is one
// pair: the mask x and the eight values H[8R + i][(8R + i) ^ x], written as
// zero where the CSR drop rule drops that entry.  The values are the CSR's
// (same group sums in the same order, same rounding), and the pairs of a
// block follow the canonical group order.  One warp per block, lanes over
// groups, as in the CSR passes.
__device__ __forceinline__ bool xell_values(const HamView& h, int g, long long R, double tol,
                                            double (&v)[XELL_ROWS]) {
    bool any = false;
#pragma unroll
    for (int i = 0; i < XELL_ROWS; ++i) {
        const long long r = R * XELL_ROWS + i;
        v[i] = 0.0;
        if (r < h.D) {
            const double a = group_value(h, g, (uint32_t)r ^ h.gx[g]);
            if (fabs(a) > tol) {
                v[i] = a;
                any = true;
            }
        }
    }
    return any;
}

__global__ void k_xell_count(HamView h, double tol, int* counts) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long R = warp; R < h.n_blocks; R += nwarps) {
        int cnt = 0;
        double v[XELL_ROWS];
        for (int g = lane; g < h.G; g += 32) cnt += xell_values(h, g, R, tol, v);
        cnt = warp_sum_int(cnt);
        if (lane == 0) counts[R] = cnt;
    }
}

template <typename VT>
__global__ void k_xell_fill(HamView h, double tol, uint32_t* xmask, VT* xval) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long R = warp; R < h.n_blocks; R += nwarps) {
        long long base = h.xptr[R];
        for (int g0 = 0; g0 < h.G; g0 += 32) {
            const int g = g0 + lane;
            double v[XELL_ROWS];
            const bool keep = g < h.G && xell_values(h, g, R, tol, v);
            const unsigned ball = __ballot_sync(0xffffffffu, keep);
            if (keep) {
                const long long pos = base + __popc(ball & ((1u << lane) - 1u));
                xmask[pos] = h.gx[g];
#pragma unroll
                for (int i = 0; i < XELL_ROWS; ++i) xval[pos * XELL_ROWS + i] = (VT)v[i];
            }
            base += __popc(ball);
        }
    }
}

// split[c] = first row block of CTA c: the smallest R with
// xptr[R] >= c * n_pairs / grid (pair-balanced contiguous ranges);
// split[grid] = n_blocks.
__global__ void k_xell_split(const int* xptr, long long n_blocks, int grid, int* split) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > grid) return;
    if (c == grid) {
        split[c] = (int)n_blocks;
        return;
    }
    const long long target = (long long)c * xptr[n_blocks] / grid;
    long long lo = 0, hi = n_blocks;        // first index in [0, n_blocks] with xptr >= target
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (xptr[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    split[c] = (int)lo;
}

__global__ void k_set_basis_c128(double2* psi, long long D, long long index) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride)
        psi[i] = make_double2(i == index ? 1.0 : 0.0, 0.0);
}
__global__ void k_set_basis_c64(float2* psi, long long D, long long index) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < D; i += stride)
        psi[i] = make_float2(i == index ? 1.0f : 0.0f, 0.0f);
}

int grid_for(long long work, int per_block, int sms, int max_per_sm) {
    long long g = (work + per_block - 1) / per_block;
    long long cap = (long long)sms * max_per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int launch_csr_count(const HamView& h, double tol, double amb_hi, int* counts,
                     unsigned long long* n_amb, int sms, cudaStream_t s) {
    const int bs = 256;
    k_csr_count<<<grid_for(h.D * 32, bs, sms, 8), bs, 0, s>>>(h, tol, amb_hi, counts, n_amb);
    return 1;
}

int launch_diag(const HamView& h, double* diag, int sms, cudaStream_t s) {
    const int bs = 256;
    k_diag<<<grid_for(h.D, bs, sms, 8), bs, 0, s>>>(h, diag);
    return 1;
}

int launch_scan(const int* counts, long long D, int* rowptr, long long* total, int* max_row,
                cudaStream_t s) {
    k_scan<<<1, 1024, 0, s>>>(counts, D, rowptr, total, max_row);
    return 1;
}

int launch_csr_fill(const HamView& h, double tol, int max_row, int* col, void* val, int prec,
                    int sms, cudaStream_t s) {
    int cap = 1;
    while (cap < max_row) cap <<= 1;
    if (cap < 32) cap = 32;
    // warps per block so that shared memory stays within 96 KB
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * cap * 12 > 96 * 1024) wpb >>= 1;
    const size_t smem = (size_t)wpb * cap * 12;
    const int bs = wpb * 32;
    const int grid = grid_for(h.D * 32, bs, sms, 8);
    if (prec == TQ_C128) {
        cudaFuncSetAttribute(k_csr_fill<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_csr_fill<double><<<grid, bs, smem, s>>>(h, tol, cap, col, static_cast<double*>(val));
    } else {
        cudaFuncSetAttribute(k_csr_fill<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_csr_fill<float><<<grid, bs, smem, s>>>(h, tol, cap, col, static_cast<float*>(val));
    }
    return 1;
}

int launch_xell_count(const HamView& h, double tol, int* counts, int sms, cudaStream_t s) {
    const int bs = 256;
    k_xell_count<<<grid_for(h.n_blocks * 32, bs, sms, 8), bs, 0, s>>>(h, tol, counts);
    return 1;
}

int launch_xell_fill(const HamView& h, double tol, uint32_t* xmask, void* xval, int prec, int sms,
                     cudaStream_t s) {
    const int bs = 256;
    const int grid = grid_for(h.n_blocks * 32, bs, sms, 8);
    if (prec == TQ_C128)
        k_xell_fill<double><<<grid, bs, 0, s>>>(h, tol, xmask, static_cast<double*>(xval));
    else
        k_xell_fill<float><<<grid, bs, 0, s>>>(h, tol, xmask, static_cast<float*>(xval));
    return 1;
}

int launch_xell_split(const int* xptr, long long n_blocks, int grid, int* split, cudaStream_t s) {
    k_xell_split<<<(grid + 1 + 255) / 256, 256, 0, s>>>(xptr, n_blocks, grid, split);
    return 1;
}

int launch_set_basis(void* psi, int prec, long long D, long long index, cudaStream_t s) {
    const int bs = 256;
    const int grid = (int)((D + bs - 1) / bs < 4096 ? (D + bs - 1) / bs : 4096);
    if (prec == TQ_C128)
        k_set_basis_c128<<<grid, bs, 0, s>>>(static_cast<double2*>(psi), D, index);
    else
        k_set_basis_c64<<<grid, bs, 0, s>>>(static_cast<float2*>(psi), D, index);
    return 1;
}

}  // namespace tq
