// Definitions of the helpers declared in api_internal.h.
#include "api_internal.h"

#include "dev.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace tq {
namespace api {




void* scratch(tq_ctx* c, int slot, size_t bytes) {
    if (c->scratch_bytes[slot] < bytes) {
        if (c->scratch[slot]) TQ_CUDA(cudaFree(c->scratch[slot]));
        c->scratch[slot] = nullptr;
        c->scratch_bytes[slot] = 0;
        c->scratch[slot] = dev_alloc(bytes);
        c->scratch_bytes[slot] = bytes;
    }
    return c->scratch[slot];
}

unsigned* tickets(tq_ctx* c, size_t n) {
    if (c->tickets_n < n) {
        if (c->tickets) TQ_CUDA(cudaFree(c->tickets));
        c->tickets = nullptr;
        c->tickets_n = 0;
        c->tickets = static_cast<unsigned*>(dev_alloc(n * sizeof(unsigned)));
        TQ_CUDA(cudaMemset(c->tickets, 0, n * sizeof(unsigned)));
        c->tickets_n = n;
    }
    return c->tickets;
}



size_t elem_bytes(int prec) { return prec == TQ_C128 ? 16 : 8; }

void check_prec(int prec) {
    TQ_REQUIRE(prec == TQ_C128 || prec == TQ_C64, "prec must be TQ_C128 or TQ_C64");
}


void set_device(const tq_ctx* c) { TQ_CUDA(cudaSetDevice(c->device)); }

// Build the CSR of a grouped Pauli sum into (rowptr, col, val); returns nnz.
long long build_csr(tq_ctx* c, HamView& h, double maxc, int prec, std::vector<void*>& allocs,
                    long long* n_amb, int* max_row) {
    const long long D = h.D;
    int* counts = static_cast<int*>(scratch(c, S_G, (size_t)D * sizeof(int)));
    int* rowptr = static_cast<int*>(dev_alloc((size_t)(D + 1) * sizeof(int)));
    allocs.push_back(rowptr);
    struct Out { long long total; int max_row; int pad; unsigned long long amb; };
    Out* dout = static_cast<Out*>(scratch(c, S_PART, sizeof(Out)));
    TQ_CUDA(cudaMemset(dout, 0, sizeof(Out)));
    const double tol = 1e-12 * maxc, amb_hi = 1e-9 * maxc;
    if (h.G > 0) {
        launch(c, "csr_count", 0, [&] { return launch_csr_count(h, tol, amb_hi, counts, &dout->amb, c->sm_count, 0); });
    } else {
        TQ_CUDA(cudaMemset(counts, 0, (size_t)D * sizeof(int)));
    }
    launch(c, "scan", 0, [&] { return launch_scan(counts, D, rowptr, &dout->total, &dout->max_row, 0); });
    Out hout;
    TQ_CUDA(cudaMemcpy(&hout, dout, sizeof(Out), cudaMemcpyDeviceToHost));
    if (hout.total >= 2147483647ll)
        throw Error(TQ_ENOMEM, "CSR has 2^31 or more non-zeros; int32 indices cannot address it");
    const long long nnz = hout.total;
    int* col = static_cast<int*>(dev_alloc((size_t)nnz * sizeof(int)));
    allocs.push_back(col);
    void* val = dev_alloc((size_t)nnz * (prec == TQ_C128 ? sizeof(double) : sizeof(float)));
    allocs.push_back(val);
    h.rowptr = rowptr;
    h.col = col;
    h.val = val;
    h.nnz = nnz;
    if (nnz > 0) launch(c, "csr_fill", 0, [&] { return launch_csr_fill(h, tol, hout.max_row, col, val, prec, c->sm_count, 0); });
    TQ_CUDA(cudaDeviceSynchronize());
    if (n_amb) *n_amb = (long long)hout.amb;
    if (max_row) *max_row = hout.max_row;
    return nnz;
}

// XOR-ELL form of the same off-diagonal entries (blocks of XELL_ROWS rows);
// returns the number of pairs.
long long build_xell(tq_ctx* c, HamView& h, double maxc, int prec, std::vector<void*>& allocs) {
    h.n_blocks = (h.D + XELL_ROWS - 1) / XELL_ROWS;
    const long long B = h.n_blocks;
    int* counts = static_cast<int*>(scratch(c, S_G, (size_t)B * sizeof(int)));
    int* xptr = static_cast<int*>(dev_alloc((size_t)(B + 1) * sizeof(int)));
    allocs.push_back(xptr);
    struct Out { long long total; int max_row; int pad; };
    Out* dout = static_cast<Out*>(scratch(c, S_PART, sizeof(Out)));
    TQ_CUDA(cudaMemset(dout, 0, sizeof(Out)));
    const double tol = 1e-12 * maxc;
    if (h.G > 0) {
        launch(c, "xell_count", 0, [&] { return launch_xell_count(h, tol, counts, c->sm_count, 0); });
    } else {
        TQ_CUDA(cudaMemset(counts, 0, (size_t)B * sizeof(int)));
    }
    launch(c, "scan", 0, [&] { return launch_scan(counts, B, xptr, &dout->total, &dout->max_row, 0); });
    Out hout;
    TQ_CUDA(cudaMemcpy(&hout, dout, sizeof(Out), cudaMemcpyDeviceToHost));
    if (hout.total >= 2147483647ll)
        throw Error(TQ_ENOMEM, "XOR-ELL has 2^31 or more pairs; int32 offsets cannot address it");
    const long long np = hout.total;
    // padded to whole copy chunks: the staged energy copies chunk by chunk
    const long long chunk = xell_chunk_pairs();
    const long long cap = std::max(1ll, (np + chunk - 1) / chunk) * chunk;
    const size_t vb = prec == TQ_C128 ? sizeof(double) : sizeof(float);
    uint32_t* xmask = static_cast<uint32_t*>(dev_alloc((size_t)cap * sizeof(uint32_t)));
    allocs.push_back(xmask);
    void* xval = dev_alloc((size_t)cap * XELL_ROWS * vb);
    allocs.push_back(xval);
    TQ_CUDA(cudaMemset(xmask + np, 0, (size_t)(cap - np) * sizeof(uint32_t)));
    TQ_CUDA(cudaMemset(static_cast<char*>(xval) + (size_t)np * XELL_ROWS * vb, 0,
                       (size_t)(cap - np) * XELL_ROWS * vb));
    h.xptr = xptr;
    h.xmask = xmask;
    h.xval = xval;
    h.n_pairs = np;
    if (np > 0) launch(c, "xell_fill", 0, [&] { return launch_xell_fill(h, tol, xmask, xval, prec, c->sm_count, 0); });
    // pair-balanced block ranges for the staged energy launch
    h.xgrid = xell_grid(B, prec, c->sm_count);
    int* split = static_cast<int*>(dev_alloc((size_t)(h.xgrid + 1) * sizeof(int)));
    allocs.push_back(split);
    h.xsplit = split;
    launch(c, "xell_split", 0, [&] { return launch_xell_split(xptr, B, h.xgrid, split, 0); });
    TQ_CUDA(cudaDeviceSynchronize());
    return np;
}

// A pool, Hamiltonian and state must describe the same space: the same
// qubit count, and either all the full space or all the same sector.
void check_space(const tq_pool* p, const tq_state* s) {
    TQ_REQUIRE(s->nq == p->nq, "state and pool qubit counts differ");
    TQ_REQUIRE(s->sector == p->sector, "state and pool differ in sector restriction");
    if (p->sector)
        TQ_REQUIRE(s->n_alpha == p->n_alpha && s->n_beta == p->n_beta, "state and pool sectors differ");
}
void check_space(const tq_ham* h, const tq_state* s) {
    TQ_REQUIRE(h->nq == s->nq, "state and Hamiltonian qubit counts differ");
    TQ_REQUIRE(h->sector == s->sector, "state and Hamiltonian differ in sector restriction");
    if (h->sector)
        TQ_REQUIRE(s->n_alpha == h->n_alpha && s->n_beta == h->n_beta, "state and Hamiltonian sectors differ");
}

void free_all(std::vector<void*>& allocs) {
    for (void* p : allocs)
        if (p) cudaFree(p);
    allocs.clear();
}



long long state_len(const tq_pool* p) { return p->sector ? p->view.sdim : 1ll << p->nq; }

// norm partials per state of the Taylor-5 launch for this pool
int update_tiles(const tq_pool* p, int prec, int upt) {
    return p->sector ? sector_tiles(p->view.sdim, prec) : taylor5_pair_parts(p->nq, upt);
}

// Taylor-5 on n states (ops and angles from k/theta arrays, or k_fixed and
// theta_fixed, or the step record when `gate` is set).  Returns true when
// the launch also wrote the float64 norms (norm2[i] and/or *step_norm2);
// otherwise they are in `part`, for launch_norm_reduce.
bool launch_update(tq_ctx* c, const tq_pool* p, long long n, int prec, int upt, void* psi, const int* k,
                   const double* theta, int k_fixed, double theta_fixed, const DevStep* gate, double* part,
                   double* norm2, double* step_norm2, cudaStream_t s) {
    if (p->sector) {
        launch(c, gate ? "taylor5_sector_gated" : "taylor5_sector", s, [&] {
            return launch_taylor5_sector(p->view, n, prec, psi, k, theta, k_fixed, theta_fixed, gate, part, norm2,
                                         step_norm2, s);
        });
        return sector_in_smem(p->view.sdim, prec);
    }
    if (gate) {
        launch(c, "taylor5_pair_gated", s, [&] { return launch_taylor5_pair_gated(p->view, prec, upt, psi, gate, part,
                                                  c->sm_count, s); });
    } else {
        launch(c, "taylor5_pair", s, [&] { return launch_taylor5_pair(p->view, (int)n, prec, upt, psi, k, theta, k_fixed,
                                                                      theta_fixed, part, c->sm_count, s); });
    }
    return false;
}



// Partials needed by energy + gradients (+ line search) on this problem.
size_t partials_needed(long long D, int n_gitems, int nq, int sms) {
    size_t n = (size_t)energy_grid(D, sms) * 2;
    n = std::max(n, (size_t)16 * sms);      // any persistent energy grid (at most 8 blocks per SM)
    n = std::max(n, (size_t)std::max(n_gitems, 0));
    n = std::max(n, (size_t)512 * 6);            // the line search's six dots per block
    n = std::max(n, (size_t)line_support_partials(sms));   // its support pass: five per block
    n = std::max(n, (size_t)taylor5_pair_parts(nq, 1));
    return n + 8;
}

void run_energy(tq_ctx* c, const tq_ham* h, const tq_state* psi, double* part, cudaStream_t s) {
    check_space(h, psi);
    TQ_REQUIRE(h->prec == psi->prec, "state and Hamiltonian precisions differ");
    double2* w = static_cast<double2*>(c->scratch[S_W0]);
    float2* w32 = psi->prec == TQ_C64 ? static_cast<float2*>(c->scratch[S_W32]) : nullptr;
    // a sector Hamiltonian has the CSR only
    const int lanes = c->spmv_lanes == TQ_SPMV_XELL && h->sector ? 8 : c->spmv_lanes;
    if (lanes == TQ_SPMV_XELL)
        launch(c, "energy_xell", s, [&] {
            return launch_energy_xell(h->view, psi->data, psi->prec, w, w32, part, c->tickets, c->step, s,
                                      (c->test_flags & TQ_TEST_WITHHOLD_CHUNK) ? 0 : -1);
        });
    else
        launch(c, "energy_csr", s, [&] { return launch_energy_csr2(h->view, psi->data, psi->prec, w, w32, part,
                                                                   c->tickets, c->step, c->sm_count, s, lanes); });
}

void run_gradients(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi, double* g,
                   double* part, cudaStream_t s) {
    check_space(p, psi);
    run_energy(c, h, psi, part, s);
    if (p->sector) {
        launch(c, "sector_gradients", s, [&] {
            return launch_sector_gradients(p->view, static_cast<double2*>(c->scratch[S_W0]), psi->data, psi->prec,
                                           c->step, g, s);
        });
        return;
    }
    launch(c, "pool_gradients", s, [&] {
        return launch_pool_gradients(p->view, static_cast<double2*>(c->scratch[S_W0]),
                                     static_cast<float2*>(c->scratch[S_W32]), psi->data, psi->prec, c->step,
                                     part, c->tickets + 16, g, c->sm_count, s);
    });
}

// Allocate (before any launch of the call) the scratch energy/gradients use.
double* prepare(tq_ctx* c, long long D, const tq_pool* p, int nq) {
    scratch(c, S_W0, (size_t)D * sizeof(double2));
    scratch(c, S_W32, (size_t)D * sizeof(float2));
    tickets(c, 16 + (size_t)(p ? p->M : 0) + 64);
    return static_cast<double*>(
        scratch(c, S_PART, partials_needed(D, p ? p->view.n_gitems : 0, nq, c->sm_count) * sizeof(double)));
}

// A kernel that gave up on a bounded wait left TQ_ETIMEOUT in the step's
// status word: clear it and report the failure.
void raise_status(tq_ctx* c, int status, cudaStream_t s) {
    if (status == TQ_OK) return;
    TQ_CUDA(cudaMemsetAsync(&c->step->status, 0, sizeof(int), s));
    TQ_CUDA(cudaStreamSynchronize(s));
    throw Error(status, "a kernel wait timed out; its results are invalid");
}


}  // namespace api
}  // namespace tq
