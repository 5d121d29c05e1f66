// C ABI of the library (declared in include/tq.h).  Argument checking,
// handle lifetime, device memory, and the launch sequences of each call.
#include "dev.cuh"
#include "host_util.h"
#include "grad.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

using namespace tq;

namespace {

thread_local std::string g_last_error;

template <typename T>
T* upload(std::vector<void*>& allocs, const std::vector<T>& v) {
    T* p = static_cast<T*>(dev_alloc(v.size() * sizeof(T)));
    allocs.push_back(p);
    if (!v.empty()) TQ_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

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

enum { S_PART = 0, S_W0, S_U1, S_U2, S_W1, S_W2, S_G, S_STAGE, S_W32, S_PHI, S_CHI, S_AG, S_HOSTB, S_REC,
       S_THETAS };

void run_energy(tq_ctx* c, const tq_ham* h, const tq_state* psi, double* part, cudaStream_t s);
double* prepare(tq_ctx* c, long long D, const tq_pool* p, int nq);

size_t elem_bytes(int prec) { return prec == TQ_C128 ? 16 : 8; }

void check_prec(int prec) {
    TQ_REQUIRE(prec == TQ_C128 || prec == TQ_C64, "prec must be TQ_C128 or TQ_C64");
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

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

}  // namespace

// ===================================================================== misc

namespace tq {
void set_last_error(const std::string& m) { g_last_error = m; }
}  // namespace tq

extern "C" const char* tq_last_error(void) { return g_last_error.c_str(); }
extern "C" int tq_version(void) { return 100; }

extern "C" int tq_ctx_create(int device, tq_ctx** out) {
    API_BEGIN
    TQ_REQUIRE(out != nullptr, "out is null");
    *out = nullptr;
    int n = 0;
    TQ_CUDA(cudaGetDeviceCount(&n));
    TQ_REQUIRE(device >= 0 && device < n, "device index out of range");
    TQ_CUDA(cudaSetDevice(device));
    auto* c = new tq_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete c;
        throw Error(TQ_ECUDA, cudaGetErrorString(e));
    }
    try {
        c->step = static_cast<DevStep*>(dev_alloc(sizeof(DevStep)));
        TQ_CUDA(cudaMemset(c->step, 0, sizeof(DevStep)));
        tickets(c, 4096);
        size_t fetch = 0;
        TQ_CUDA(cudaDeviceGetLimit(&fetch, cudaLimitMaxL2FetchGranularity));
        c->l2_fetch_default = (int)fetch;
        // the line search's sample table, filled before any call can read it
        c->line_sc = static_cast<double2*>(dev_alloc(4096 * sizeof(double2)));
        c->line_se = static_cast<double*>(dev_alloc((4096 + 64) * sizeof(double)));
        launch(c, "line_table", 0, [&] { return launch_line_table(c->line_sc, 0); });
        TQ_CUDA(cudaDeviceSynchronize());
    } catch (...) {
        tq_ctx_destroy(c);
        throw;
    }
    *out = c;
    API_END
}

extern "C" int tq_ctx_destroy(tq_ctx* c) {
    if (!c) return TQ_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (int i = 0; i < tq_ctx::kScratch; ++i)
        if (c->scratch[i]) cudaFree(c->scratch[i]);
    if (c->step) cudaFree(c->step);
    if (c->tickets) cudaFree(c->tickets);
    if (c->line_sc) cudaFree(c->line_sc);
    if (c->line_se) cudaFree(c->line_se);
    for (auto& s : c->aux)
        if (s) cudaStreamDestroy(s);
    for (auto& r : c->trace) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto& e : c->event_pool) cudaEventDestroy(e);
    delete c;
    return TQ_OK;
}

extern "C" int tq_ctx_launch_count(const tq_ctx* c, long long* launches) {
    API_BEGIN
    TQ_REQUIRE(c && launches, "null argument");
    *launches = c->launches;
    API_END
}

extern "C" int tq_ctx_set_pair_schedule(tq_ctx* c, int prec, int units_per_thread) {
    API_BEGIN
    TQ_REQUIRE(c != nullptr, "ctx is null");
    check_prec(prec);
    TQ_REQUIRE(pair_upt_valid(units_per_thread), "units_per_thread must be 1, 2, 4 or 8");
    c->pair_upt[prec] = units_per_thread;
    API_END
}

extern "C" int tq_ctx_set_l2_fetch(tq_ctx* c, int bytes) {
    API_BEGIN
    TQ_REQUIRE(c != nullptr, "ctx is null");
    TQ_REQUIRE(bytes == 0 || bytes == 32 || bytes == 64 || bytes == 128, "bytes must be 0, 32, 64 or 128");
    set_device(c);
    if (bytes == 0) bytes = c->l2_fetch_default;
    TQ_CUDA(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes));
    API_END
}

extern "C" int tq_ctx_get_l2_fetch(tq_ctx* c, int* bytes) {
    API_BEGIN
    TQ_REQUIRE(c && bytes, "null argument");
    set_device(c);
    size_t v = 0;
    TQ_CUDA(cudaDeviceGetLimit(&v, cudaLimitMaxL2FetchGranularity));
    *bytes = (int)v;
    API_END
}

extern "C" int tq_ctx_get_pair_schedule(const tq_ctx* c, int prec, int* units_per_thread) {
    API_BEGIN
    TQ_REQUIRE(c && units_per_thread, "null argument");
    check_prec(prec);
    *units_per_thread = c->pair_upt[prec];
    API_END
}

extern "C" int tq_autotune_pair(tq_ctx* c, const tq_pool* p, int prec, int n_states, int* best_upt,
                                double* best_ms) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the pair-kernel autotuner works on full-space pools");
    check_prec(prec);
    TQ_REQUIRE(n_states >= 1, "n_states must be >= 1");
    set_device(c);
    const long long D = 1ll << p->nq;
    const size_t sb = (size_t)D * elem_bytes(prec);
    const size_t parts = (size_t)n_states * taylor5_pair_parts(p->nq, 1);
    unsigned char* buf = static_cast<unsigned char*>(
        scratch(c, S_STAGE, (size_t)n_states * sb + (size_t)n_states * (sizeof(int) + sizeof(double)) +
                                parts * sizeof(double) + 256));
    void* psi = buf;
    int* dk = reinterpret_cast<int*>(buf + (size_t)n_states * sb);
    double* dth = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(dk + n_states) + 15) & ~(uintptr_t)15);
    double* part = dth + n_states;
    std::vector<int> hk(n_states);
    std::vector<double> hth(n_states);
    for (int b = 0; b < n_states; ++b) {
        hk[b] = (int)((b * 2654435761u) % (unsigned)p->M);
        hth[b] = 0.05 + 1e-4 * (b % 97);
    }
    TQ_CUDA(cudaMemset(psi, 0, (size_t)n_states * sb));
    TQ_CUDA(cudaMemcpy(dk, hk.data(), n_states * sizeof(int), cudaMemcpyHostToDevice));
    TQ_CUDA(cudaMemcpy(dth, hth.data(), n_states * sizeof(double), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    int best = c->pair_upt[prec];
    float best_t = 1e30f;
    const int cands[4] = {1, 2, 4, 8};
    for (int u : cands) {
        launch(c, "autotune_pair", 0, [&] { return launch_taylor5_pair(p->view, n_states, prec, u, psi, dk, dth, 0, 0.0, part, c->sm_count, 0); });
        TQ_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 5; ++r)
            launch(c, "autotune_pair", 0, [&] { return launch_taylor5_pair(p->view, n_states, prec, u, psi, dk, dth, 0, 0.0, part, c->sm_count, 0); });
        TQ_CUDA(cudaEventRecord(e1, 0));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 5.f;
        if (ms < best_t) {
            best_t = ms;
            best = u;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->pair_upt[prec] = best;
    if (best_upt) *best_upt = best;
    if (best_ms) *best_ms = best_t;
    API_END
}

extern "C" int tq_autotune_support(tq_ctx* c, const tq_pool* p, int prec, int n_states, int* best_ppt,
                                   double* best_ms) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the support-only update takes full-space pools");
    check_prec(prec);
    TQ_REQUIRE(n_states >= 1, "n_states must be >= 1");
    set_device(c);
    const long long D = 1ll << p->nq;
    const size_t sb = (size_t)D * elem_bytes(prec);
    size_t parts = 0;
    for (int u : {1, 2, 4, 8})
        parts = std::max(parts, (size_t)n_states * support_parts(support_tiles(p->nq, n_states, u, c->sm_count)));
    const int cands[8] = {1, 2, 4, 8, -1, -2, -4, -8};
    unsigned char* buf = static_cast<unsigned char*>(
        scratch(c, S_STAGE, (size_t)n_states * sb + (size_t)n_states * (sizeof(int) + 2 * sizeof(double)) +
                                parts * sizeof(double) + 256));
    void* psi = buf;
    int* dk = reinterpret_cast<int*>(buf + (size_t)n_states * sb);
    double* dth = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(dk + n_states) + 15) & ~(uintptr_t)15);
    double* dn = dth + n_states;
    double* part = dn + n_states;
    std::vector<int> hk(n_states);
    std::vector<double> hth(n_states);
    for (int b = 0; b < n_states; ++b) {
        hk[b] = (int)((b * 2654435761u) % (unsigned)p->M);
        hth[b] = 0.05 + 1e-4 * (b % 97);
    }
    TQ_CUDA(cudaMemset(psi, 0, (size_t)n_states * sb));
    TQ_CUDA(cudaMemset(dn, 0, (size_t)n_states * sizeof(double)));
    TQ_CUDA(cudaMemcpy(dk, hk.data(), n_states * sizeof(int), cudaMemcpyHostToDevice));
    TQ_CUDA(cudaMemcpy(dth, hth.data(), n_states * sizeof(double), cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    int best = c->supp_ppt[prec];
    float best_t = 1e30f;
    for (int u : cands) {
        const int tps = support_tiles(p->nq, n_states, u, c->sm_count);
        auto once = [&] {
            launch(c, "autotune_support", 0, [&] {
                return launch_taylor5_support(p->view, n_states, prec, u, psi, dk, dth, part, tps, dn, c->sm_count, 0);
            });
            if (tps > 1)
                launch(c, "autotune_support", 0, [&] {
                    return launch_norm_carry(part, prec, n_states, support_parts(tps), dn, dn, nullptr, 0);
                });
        };
        once();
        TQ_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 5; ++r) once();
        TQ_CUDA(cudaEventRecord(e1, 0));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 5.f;
        if (ms < best_t) {
            best_t = ms;
            best = u;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->supp_ppt[prec] = best;
    if (best_ppt) *best_ppt = best;
    if (best_ms) *best_ms = best_t;
    API_END
}

extern "C" int tq_ctx_set_spmv_schedule(tq_ctx* c, int lanes_per_row) {
    API_BEGIN
    TQ_REQUIRE(c != nullptr, "ctx is null");
    TQ_REQUIRE(lanes_per_row == TQ_SPMV_XELL || lanes_per_row == 4 || lanes_per_row == 8 ||
                   lanes_per_row == 16 || lanes_per_row == 32,
               "schedule must be 4, 8, 16 or 32 CSR lanes per row, or TQ_SPMV_XELL");
    c->spmv_lanes = lanes_per_row;
    API_END
}

extern "C" int tq_autotune_spmv(tq_ctx* c, const tq_ham* h, const tq_state* psi, int* best_lanes,
                                double* best_ms) {
    API_BEGIN
    TQ_REQUIRE(c && h && psi, "null argument");
    check_space(h, psi);
    TQ_REQUIRE(h->prec == psi->prec, "state and Hamiltonian precisions differ");
    set_device(c);
    double* part = prepare(c, h->D, nullptr, h->nq);
    cudaEvent_t e0, e1;
    TQ_CUDA(cudaEventCreate(&e0));
    TQ_CUDA(cudaEventCreate(&e1));
    int best = c->spmv_lanes;
    float best_t = 1e30f;
    for (int l : {4, 8, 16, 32, (int)TQ_SPMV_XELL}) {
        if (l == TQ_SPMV_XELL && h->sector) continue;   // a sector Hamiltonian has the CSR only
        c->spmv_lanes = l;
        run_energy(c, h, psi, part, 0);
        TQ_CUDA(cudaEventRecord(e0, 0));
        for (int r = 0; r < 3; ++r) run_energy(c, h, psi, part, 0);
        TQ_CUDA(cudaEventRecord(e1, 0));
        TQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms /= 3.f;
        if (ms < best_t) {
            best_t = ms;
            best = l;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->spmv_lanes = best;
    if (best_lanes) *best_lanes = best;
    if (best_ms) *best_ms = best_t;
    API_END
}

extern "C" int tq_ctx_set_test_flags(tq_ctx* c, int flags) {
    API_BEGIN
    TQ_REQUIRE(c != nullptr, "ctx is null");
    TQ_REQUIRE((flags & ~TQ_TEST_WITHHOLD_CHUNK) == 0, "unknown test flag");
    c->test_flags = flags;
    API_END
}

extern "C" int tq_ctx_trace(tq_ctx* c, int enable) {
    API_BEGIN
    TQ_REQUIRE(c != nullptr, "ctx is null");
    c->tracing = enable ? 1 : 0;
    API_END
}

extern "C" int tq_ctx_trace_report(tq_ctx* c, char* buf, size_t buf_size) {
    API_BEGIN
    TQ_REQUIRE(c && buf && buf_size > 0, "null argument");
    set_device(c);
    std::vector<std::string> names;
    std::vector<long long> counts;
    std::vector<double> ms;
    for (auto& r : c->trace) {
        TQ_CUDA(cudaEventSynchronize(r.stop));
        float t = 0.f;
        TQ_CUDA(cudaEventElapsedTime(&t, r.start, r.stop));
        size_t i = 0;
        while (i < names.size() && names[i] != r.name) ++i;
        if (i == names.size()) {
            names.push_back(r.name);
            counts.push_back(0);
            ms.push_back(0.0);
        }
        counts[i] += 1;
        ms[i] += t;
        c->event_pool.push_back(r.start);
        c->event_pool.push_back(r.stop);
    }
    c->trace.clear();
    std::string out;
    for (size_t i = 0; i < names.size(); ++i) {
        char line[256];
        snprintf(line, sizeof line, "%s %lld %.6f\n", names[i].c_str(), counts[i], ms[i]);
        out += line;
    }
    const size_t n = std::min(out.size(), buf_size - 1);
    std::memcpy(buf, out.data(), n);
    buf[n] = '\0';
    API_END
}

// ============================================================ host algebra

extern "C" int tq_pauli_hamiltonian(int n_spatial, const double* h1, const double* g2, double e_const,
                                    int mapping, long long* n_terms, uint64_t* x, uint64_t* z, double* c,
                                    long long capacity) {
    API_BEGIN
    TQ_REQUIRE(n_terms != nullptr, "n_terms is null");
    auto t = pauli_hamiltonian(n_spatial, h1, g2, e_const, mapping);
    *n_terms = (long long)t.size();
    if (x) {
        TQ_REQUIRE(z && c, "z and c must be given with x");
        TQ_REQUIRE(capacity >= (long long)t.size(), "capacity too small");
        for (size_t i = 0; i < t.size(); ++i) {
            x[i] = t[i].x;
            z[i] = t[i].z;
            c[i] = t[i].c;
        }
    }
    API_END
}

extern "C" int tq_pool_excitations(int n_spatial, int n_electrons, int* n_ops, int* idx4, int capacity) {
    API_BEGIN
    TQ_REQUIRE(n_ops != nullptr, "n_ops is null");
    auto ex = excitations(n_spatial, n_electrons);
    *n_ops = (int)ex.size();
    if (idx4) {
        TQ_REQUIRE(capacity >= (int)ex.size(), "capacity too small");
        for (size_t k = 0; k < ex.size(); ++k)
            for (int j = 0; j < 4; ++j) idx4[4 * k + j] = ex[k].idx[j];
    }
    API_END
}

extern "C" int tq_pauli_pool(int n_spatial, int n_electrons, int mapping, int capacity, uint64_t* x,
                             int* nterm, uint64_t* z, double* c) {
    API_BEGIN
    TQ_REQUIRE(x && nterm && z && c, "null output array");
    auto ex = excitations(n_spatial, n_electrons);
    TQ_REQUIRE(capacity >= (int)ex.size(), "capacity too small");
    const int N = 2 * n_spatial;
    for (size_t k = 0; k < ex.size(); ++k) {
        auto t = pauli_generator(ex[k], N, mapping);
        if (t.size() > 8) throw Error(TQ_ENUMERIC, "generator with more than 8 terms");
        x[k] = t.empty() ? 0 : t[0].x;
        nterm[k] = (int)t.size();
        for (int j = 0; j < 8; ++j) {
            z[8 * k + j] = j < (int)t.size() ? t[j].z : 0;
            c[8 * k + j] = j < (int)t.size() ? t[j].c : 0.0;
        }
    }
    API_END
}

extern "C" int tq_pool_support_forms(int n_spatial, int n_electrons, int mapping, int capacity, int* m,
                                     int* pivots, uint64_t* masks, int* target, int* rep_bit, int* rep_pos) {
    API_BEGIN
    TQ_REQUIRE(m && pivots && masks && target && rep_bit && rep_pos, "null output array");
    auto ex = excitations(n_spatial, n_electrons);
    TQ_REQUIRE(capacity >= (int)ex.size(), "capacity too small");
    const int N = 2 * n_spatial;
    for (size_t k = 0; k < ex.size(); ++k) {
        auto t = pauli_generator(ex[k], N, mapping);
        TQ_REQUIRE(!t.empty(), "empty generator");
        SignForm f = factor_generator(t);
        if (!f.ok) throw Error(TQ_ENUMERIC, "generator sign function does not factor");
        SupportForm sf = support_form(f, t[0].x);
        m[k] = sf.m;
        for (int i = 0; i < 3; ++i) {
            pivots[3 * k + i] = i < sf.m ? sf.p[i] : -1;
            masks[3 * k + i] = i < sf.m ? sf.e[i] : 0;
        }
        target[k] = sf.target;
        rep_bit[k] = sf.h;
        rep_pos[k] = sf.hp;
    }
    API_END
}

extern "C" int tq_hf_index(int n_qubits, int n_electrons, int mapping, long long* index) {
    API_BEGIN
    TQ_REQUIRE(index != nullptr, "index is null");
    TQ_REQUIRE(n_qubits >= 1 && n_qubits <= 2 * TQ_MAX_SPATIAL, "n_qubits out of range");
    *index = (long long)hf_index(n_qubits, n_electrons, mapping);
    API_END
}

// ============================================================ Hamiltonian

namespace {

// Pauli sum -> device Hamiltonian (diagonal, CSR, and outside a sector the
// XOR-ELL layout), over the full space or over a sector (`sect` non-null).
tq_ham* make_hamiltonian(tq_ctx* c, int n_spatial, const double* h1, const double* g2, double e_const,
                         int mapping, int prec, const SectorSpec* sect) {
    auto terms = pauli_hamiltonian(n_spatial, h1, g2, e_const, mapping);
    auto* h = new tq_ham();
    try {
        h->ctx = c;
        h->device = c->device;
        h->n_spatial = n_spatial;
        h->nq = 2 * n_spatial;
        h->prec = prec;
        h->mapping = mapping;
        h->D = sect ? sector_dim(sect->n, sect->na, sect->nb) : 1ll << h->nq;
        h->n_pauli = (long long)terms.size();
        std::vector<uint32_t> gx, tz, dz;
        std::vector<int> goff;
        std::vector<double> tc, dc;
        double maxc = 0.0;
        for (size_t i = 0; i < terms.size(); ++i) {
            maxc = std::max(maxc, std::fabs(terms[i].c));
            if (terms[i].x == 0) {
                dz.push_back((uint32_t)terms[i].z);
                dc.push_back(terms[i].c);
                continue;
            }
            if (gx.empty() || gx.back() != (uint32_t)terms[i].x) {
                gx.push_back((uint32_t)terms[i].x);
                goff.push_back((int)tz.size());
            }
            tz.push_back((uint32_t)terms[i].z);
            tc.push_back(terms[i].c);
        }
        goff.push_back((int)tz.size());
        HamView& v = h->view;
        v.nq = h->nq;
        v.prec = prec;
        v.D = h->D;
        v.G = (int)gx.size();
        v.gx = upload(h->allocs, gx);
        v.goff = upload(h->allocs, goff);
        v.tz = upload(h->allocs, tz);
        v.tc = upload(h->allocs, tc);
        v.Kd = (int)dz.size();
        v.dz = upload(h->allocs, dz);
        v.dc = upload(h->allocs, dc);
        size_t extra = 0;
        if (sect) {
            h->sector = 1;
            h->n_alpha = sect->na;
            h->n_beta = sect->nb;
            const auto basis = sector_basis(*sect);
            v.sq = upload(h->allocs, basis);
            v.sect = upload(h->allocs, std::vector<SectorSpec>{*sect});
            extra = basis.size() * 4 + sizeof(SectorSpec);
        }
        double* diag = static_cast<double*>(dev_alloc((size_t)h->D * sizeof(double)));
        h->allocs.push_back(diag);
        v.diag = diag;
        launch(c, "diag", 0, [&] { return launch_diag(v, diag, c->sm_count, 0); });
        h->nnz = build_csr(c, v, maxc, prec, h->allocs, &h->n_amb, &h->max_row);
        const long long np = sect ? 0 : build_xell(c, v, maxc, prec, h->allocs);
        const size_t vb = prec == TQ_C128 ? 8 : 4;
        h->bytes = (size_t)h->D * 8 + (size_t)(h->D + 1) * 4 + (size_t)h->nnz * (4 + vb) + extra +
                   (sect ? 0 : (size_t)(v.n_blocks + 1) * 4 + (size_t)np * (4 + XELL_ROWS * vb) + (size_t)(v.xgrid + 1) * 4) +
                   (gx.size() + goff.size() + tz.size() + dz.size()) * 4 + (tc.size() + dc.size()) * 8;
    } catch (...) {
        tq_ham_free(h);
        throw;
    }
    return h;
}

}  // namespace

extern "C" int tq_build_hamiltonian(tq_ctx* c, int n_spatial, const double* h1, const double* g2,
                                    double e_const, int mapping, int prec, tq_ham** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(std::isfinite(e_const), "e_const is not finite");
    TQ_REQUIRE(n_spatial >= 1 && 2 * n_spatial <= TQ_MAX_STATE_QUBITS,
               "n_spatial must give at most 26 qubits for a device Hamiltonian");
    set_device(c);
    *out = make_hamiltonian(c, n_spatial, h1, g2, e_const, mapping, prec, nullptr);
    API_END
}

extern "C" int tq_build_hamiltonian_sector(tq_ctx* c, int n_spatial, const double* h1, const double* g2,
                                           double e_const, int mapping, int prec, int n_alpha, int n_beta,
                                           tq_ham** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(std::isfinite(e_const), "e_const is not finite");
    TQ_REQUIRE(n_spatial >= 1 && 2 * n_spatial <= TQ_MAX_STATE_QUBITS,
               "n_spatial must give at most 26 qubits for a device Hamiltonian");
    const SectorSpec sp = make_sector_spec(n_spatial, n_alpha, n_beta, mapping);
    set_device(c);
    *out = make_hamiltonian(c, n_spatial, h1, g2, e_const, mapping, prec, &sp);
    API_END
}

extern "C" int tq_sector_dim(int n_spatial, int n_alpha, int n_beta, long long* dim) {
    API_BEGIN
    TQ_REQUIRE(dim != nullptr, "null argument");
    const SectorSpec sp = make_sector_spec(n_spatial, n_alpha, n_beta, TQ_JW);
    *dim = sector_dim(sp.n, sp.na, sp.nb);
    API_END
}

extern "C" int tq_sector_basis(int n_spatial, int n_alpha, int n_beta, int mapping, long long capacity,
                               unsigned* qubit_index) {
    API_BEGIN
    TQ_REQUIRE(qubit_index != nullptr, "null argument");
    const SectorSpec sp = make_sector_spec(n_spatial, n_alpha, n_beta, mapping);
    TQ_REQUIRE(capacity >= sector_dim(sp.n, sp.na, sp.nb), "capacity is smaller than the sector dimension");
    const auto b = sector_basis(sp);
    std::copy(b.begin(), b.end(), qubit_index);
    API_END
}

extern "C" int tq_ham_info(const tq_ham* h, int* n_qubits, int* prec, long long* nnz, long long* n_pauli,
                           long long* n_xgroups, long long* n_ambiguous, size_t* device_bytes) {
    API_BEGIN
    TQ_REQUIRE(h != nullptr, "ham is null");
    if (n_qubits) *n_qubits = h->nq;
    if (prec) *prec = h->prec;
    if (nnz) *nnz = h->nnz;
    if (n_pauli) *n_pauli = h->n_pauli;
    if (n_xgroups) *n_xgroups = h->view.G + (h->view.Kd > 0 ? 1 : 0);
    if (n_ambiguous) *n_ambiguous = h->n_amb;
    if (device_bytes) *device_bytes = h->bytes;
    API_END
}

extern "C" int tq_ham_csr(const tq_ham* h, const int** rowptr, const int** col, const void** val,
                          const double** diag) {
    API_BEGIN
    TQ_REQUIRE(h != nullptr, "ham is null");
    if (rowptr) *rowptr = h->view.rowptr;
    if (col) *col = h->view.col;
    if (val) *val = h->view.val;
    if (diag) *diag = h->view.diag;
    API_END
}

extern "C" int tq_ham_xell(const tq_ham* h, long long* n_blocks, long long* n_pairs, const int** xptr,
                           const unsigned** xmask, const void** xval) {
    API_BEGIN
    TQ_REQUIRE(h != nullptr, "ham is null");
    if (n_blocks) *n_blocks = h->view.n_blocks;
    if (n_pairs) *n_pairs = h->view.n_pairs;
    if (xptr) *xptr = h->view.xptr;
    if (xmask) *xmask = h->view.xmask;
    if (xval) *xval = h->view.xval;
    API_END
}

extern "C" int tq_ham_free(tq_ham* h) {
    if (!h) return TQ_OK;
    cudaSetDevice(h->device);
    free_all(h->allocs);
    delete h;
    (void)cudaGetLastError();   // a failure while freeing is not reported to later calls
    return TQ_OK;
}

// =================================================================== pool

namespace {

tq_pool* make_pool(tq_ctx* c, int n_spatial, int n_electrons, int mapping) {
    auto ex = excitations(n_spatial, n_electrons);
    TQ_REQUIRE(!ex.empty(), "the pool is empty for this electron count");
    auto* p = new tq_pool();
    try {
        p->ctx = c;
        p->device = c->device;
        p->n_spatial = n_spatial;
        p->n_electrons = n_electrons;
        p->nq = 2 * n_spatial;
        p->mapping = mapping;
        p->M = (int)ex.size();
        const int M = p->M;
        std::vector<uint32_t> x(M), z(8 * M, 0), fz0(M, 0), fd(3 * M, 0);
        std::vector<int> nterm(M), fok(M, 0), fm(M, 0), ft(M, 0);
        std::vector<float> cf(8 * M, 0.f), fc0f(M, 0.f);
        std::vector<int4> supp(M);
        std::vector<uint32_t> supe(3 * M, 0);
        std::vector<double> cd(8 * M, 0.0), fc0d(M, 0.0);
        p->idx4.resize(4 * M);
        p->terms.assign(8 * M, PauliTerm{0, 0, 0.0});
        for (int k = 0; k < M; ++k) {
            for (int j = 0; j < 4; ++j) p->idx4[4 * k + j] = ex[k].idx[j];
            auto t = pauli_generator(ex[k], p->nq, mapping);
            if (t.empty() || t.size() > 8) throw Error(TQ_ENUMERIC, "generator term count not in 1..8");
            x[k] = (uint32_t)t[0].x;
            nterm[k] = (int)t.size();
            for (size_t j = 0; j < t.size(); ++j) {
                if (t[j].x != t[0].x) throw Error(TQ_ENUMERIC, "generator with more than one X-mask");
                z[8 * k + j] = (uint32_t)t[j].z;
                cd[8 * k + j] = t[j].c;
                cf[8 * k + j] = (float)t[j].c;
                p->terms[8 * k + j] = t[j];
            }
            SignForm f = factor_generator(t);
            if (!f.ok) throw Error(TQ_ENUMERIC, "generator sign function does not factor");
            {
                fok[k] = 1;
                fm[k] = f.m;
                fz0[k] = (uint32_t)f.z0;
                for (int i = 0; i < 3; ++i) fd[3 * k + i] = (uint32_t)f.d[i];
                ft[k] = f.t;
                fc0d[k] = f.c0;
                fc0f[k] = (float)f.c0;
                SupportForm sf = support_form(f, t[0].x);
                supp[k] = make_int4(sf.m | (sf.target << 8), sf.p[0] | (sf.p[1] << 8) | (sf.p[2] << 16), sf.hp, sf.h);
                for (int i = 0; i < 3; ++i) supe[3 * k + i] = (uint32_t)sf.e[i];
            }
        }
        p->nterm = nterm;
        PoolView& v = p->view;
        v.M = M;
        v.nq = p->nq;
        v.x = upload(p->allocs, x);
        v.nterm = upload(p->allocs, nterm);
        v.z = upload(p->allocs, z);
        v.cf = upload(p->allocs, cf);
        v.cd = upload(p->allocs, cd);
        v.fok = upload(p->allocs, fok);
        v.fm = upload(p->allocs, fm);
        v.fz0 = upload(p->allocs, fz0);
        v.fd = upload(p->allocs, fd);
        v.ft = upload(p->allocs, ft);
        v.fc0f = upload(p->allocs, fc0f);
        v.fc0d = upload(p->allocs, fc0d);
        v.supp = upload(p->allocs, supp);
        v.supe = upload(p->allocs, supe);
        // gradient work items: (op, chunk of its support rows)
        std::vector<int2> gitems;
        std::vector<int> gfirst;
        for (int k = 0; k < M; ++k) {
            gfirst.push_back((int)gitems.size());
            const int m = supp[k].x & 0xff;
            const long long size = (1ll << p->nq) >> m;
            for (long long u = 0, ch = 0; u < size; u += GRAD_CHUNK, ++ch) gitems.push_back(make_int2(k, (int)ch));
        }
        gfirst.push_back((int)gitems.size());
        v.gitems = upload(p->allocs, gitems);
        v.gfirst = upload(p->allocs, gfirst);
        v.n_gitems = (int)gitems.size();
        for (int q = 0; q < 2; ++q) {
            p->csr_rowptr[q].assign(M, nullptr);
            p->csr_col[q].assign(M, nullptr);
            p->csr_val[q].assign(M, nullptr);
            p->csr_nnz[q].assign(M, -1);
        }
    } catch (...) {
        tq_pool_free(p);
        throw;
    }
    return p;
}

}  // namespace

extern "C" int tq_build_pool(tq_ctx* c, int n_spatial, int n_electrons, int mapping, tq_pool** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    TQ_REQUIRE(n_spatial >= 1 && 2 * n_spatial <= TQ_MAX_STATE_QUBITS, "n_spatial out of range");
    check_mapping(mapping);
    set_device(c);
    *out = make_pool(c, n_spatial, n_electrons, mapping);
    API_END
}

extern "C" int tq_build_pool_sector(tq_ctx* c, int n_spatial, int n_electrons, int mapping, int n_alpha,
                                    int n_beta, tq_pool** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    TQ_REQUIRE(n_spatial >= 1 && 2 * n_spatial <= TQ_MAX_STATE_QUBITS, "n_spatial out of range");
    const SectorSpec sp = make_sector_spec(n_spatial, n_alpha, n_beta, mapping);
    set_device(c);
    tq_pool* p = make_pool(c, n_spatial, n_electrons, mapping);
    try {
        const long long dim = sector_dim(sp.n, sp.na, sp.nb);
        std::vector<void*> tmp;
        const uint32_t* sq = upload(tmp, sector_basis(sp));
        const SectorSpec* dsp = upload(tmp, std::vector<SectorSpec>{sp});
        unsigned long long* bad = static_cast<unsigned long long*>(dev_alloc(sizeof(unsigned long long)));
        tmp.push_back(bad);
        int* scol = static_cast<int*>(dev_alloc((size_t)p->M * dim * sizeof(int)));
        p->allocs.push_back(scol);
        signed char* ssgn = static_cast<signed char*>(dev_alloc((size_t)p->M * dim));
        p->allocs.push_back(ssgn);
        unsigned long long hbad = 0;
        try {
            TQ_CUDA(cudaMemset(bad, 0, sizeof(unsigned long long)));
            launch(c, "sector_pool", 0, [&] { return launch_sector_pool(p->view, sq, dsp, dim, scol, ssgn, bad, c->sm_count, 0); });
            TQ_CUDA(cudaMemcpy(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost));
        } catch (...) {
            free_all(tmp);
            throw;
        }
        free_all(tmp);
        if (hbad) throw Error(TQ_ENUMERIC, "a pool generator leaves the sector");
        p->sector = 1;
        p->n_alpha = n_alpha;
        p->n_beta = n_beta;
        p->view.sdim = dim;
        p->view.scol = scol;
        p->view.ssgn = ssgn;
    } catch (...) {
        tq_pool_free(p);
        throw;
    }
    *out = p;
    API_END
}

namespace {

void write_families(const std::vector<int>& fam, int* family, int* order, int* n_families) {
    const int M = (int)fam.size();
    int K = 0;
    for (int f : fam) K = std::max(K, f + 1);
    if (family) std::copy(fam.begin(), fam.end(), family);
    if (order) {
        std::vector<int> o(M);
        for (int v = 0; v < M; ++v) o[v] = v;
        std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return fam[a] < fam[b]; });
        std::copy(o.begin(), o.end(), order);
    }
    if (n_families) *n_families = K;
}

}  // namespace

extern "C" int tq_pool_families(const tq_pool* p, int mode, int* family, int* order, int* n_families) {
    API_BEGIN
    TQ_REQUIRE(p != nullptr, "pool is null");
    write_families(pool_families(p->terms, p->nterm, mode), family, order, n_families);
    API_END
}

extern "C" int tq_pool_families_host(int n_spatial, int n_electrons, int mapping, int mode, int capacity,
                                     int* family, int* order, int* n_families) {
    API_BEGIN
    check_mapping(mapping);
    auto ex = excitations(n_spatial, n_electrons);
    TQ_REQUIRE(capacity >= (int)ex.size(), "capacity is smaller than the pool");
    std::vector<PauliTerm> terms(8 * ex.size(), PauliTerm{0, 0, 0.0});
    std::vector<int> nterm(ex.size());
    for (size_t k = 0; k < ex.size(); ++k) {
        auto t = pauli_generator(ex[k], 2 * n_spatial, mapping);
        TQ_REQUIRE(!t.empty() && t.size() <= 8, "generator term count not in 1..8");
        nterm[k] = (int)t.size();
        for (size_t j = 0; j < t.size(); ++j) terms[8 * k + j] = t[j];
    }
    write_families(pool_families(terms, nterm, mode), family, order, n_families);
    API_END
}

extern "C" int tq_pool_sector_table(const tq_pool* p, long long* dim, const int** col, const signed char** sgn) {
    API_BEGIN
    TQ_REQUIRE(p != nullptr, "pool is null");
    if (dim) *dim = p->view.sdim;
    if (col) *col = p->view.scol;
    if (sgn) *sgn = p->view.ssgn;
    API_END
}

extern "C" int tq_pool_info(const tq_pool* p, int* n_ops, int* n_qubits, int* idx4) {
    API_BEGIN
    TQ_REQUIRE(p != nullptr, "pool is null");
    if (n_ops) *n_ops = p->M;
    if (n_qubits) *n_qubits = p->nq;
    if (idx4) std::memcpy(idx4, p->idx4.data(), p->idx4.size() * sizeof(int));
    API_END
}

extern "C" int tq_pool_csr(tq_ctx* c, tq_pool* p, int k, int prec, const int** rowptr, const int** col,
                           const void** val, long long* nnz) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    check_prec(prec);
    TQ_REQUIRE(k >= 0 && k < p->M, "pool index out of range");
    const int q = prec == TQ_C128 ? 0 : 1;
    if (p->csr_nnz[q][k] < 0) {
        set_device(c);
        std::vector<void*> allocs;
        try {
            const int nt = p->nterm[k];
            std::vector<uint32_t> gx = {(uint32_t)p->terms[8 * k].x}, tz(nt);
            std::vector<int> goff = {0, nt};
            std::vector<double> tc(nt);
            double maxc = 0.0;
            for (int j = 0; j < nt; ++j) {
                tz[j] = (uint32_t)p->terms[8 * k + j].z;
                tc[j] = p->terms[8 * k + j].c;
                maxc = std::max(maxc, std::fabs(tc[j]));
            }
            HamView v{};
            v.nq = p->nq;
            v.prec = prec;
            v.D = 1ll << p->nq;
            v.G = 1;
            v.gx = upload(allocs, gx);
            v.goff = upload(allocs, goff);
            v.tz = upload(allocs, tz);
            v.tc = upload(allocs, tc);
            std::vector<void*> keep;
            const long long n = build_csr(c, v, maxc, prec, keep, nullptr, nullptr);
            free_all(allocs);
            for (void* ptr : keep) p->allocs.push_back(ptr);
            p->csr_rowptr[q][k] = v.rowptr;
            p->csr_col[q][k] = v.col;
            p->csr_val[q][k] = v.val;
            p->csr_nnz[q][k] = n;
        } catch (...) {
            free_all(allocs);
            throw;
        }
    }
    if (rowptr) *rowptr = p->csr_rowptr[q][k];
    if (col) *col = p->csr_col[q][k];
    if (val) *val = p->csr_val[q][k];
    if (nnz) *nnz = p->csr_nnz[q][k];
    API_END
}

extern "C" int tq_pool_free(tq_pool* p) {
    if (!p) return TQ_OK;
    cudaSetDevice(p->device);
    free_all(p->allocs);
    delete p;
    (void)cudaGetLastError();   // a failure while freeing is not reported to later calls
    return TQ_OK;
}

// ================================================================== state

extern "C" int tq_state_create(tq_ctx* c, int n_qubits, int prec, tq_state** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(n_qubits >= 1 && n_qubits <= TQ_MAX_STATE_QUBITS, "n_qubits out of range [1, 26]");
    set_device(c);
    auto* s = new tq_state();
    s->ctx = c;
    s->device = c->device;
    s->nq = n_qubits;
    s->prec = prec;
    s->D = 1ll << n_qubits;
    s->owned = 1;
    try {
        s->data = dev_alloc((size_t)s->D * elem_bytes(prec));
        TQ_CUDA(cudaMemset(s->data, 0, (size_t)s->D * elem_bytes(prec)));
    } catch (...) {
        delete s;
        throw;
    }
    *out = s;
    API_END
}

extern "C" int tq_state_wrap(tq_ctx* c, int n_qubits, int prec, void* dev_ptr, tq_state** out) {
    API_BEGIN
    TQ_REQUIRE(c && out && dev_ptr, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(n_qubits >= 1 && n_qubits <= TQ_MAX_STATE_QUBITS, "n_qubits out of range [1, 26]");
    TQ_REQUIRE(((uintptr_t)dev_ptr & 15u) == 0, "state pointer must be 16-byte aligned");
    auto* s = new tq_state();
    s->ctx = c;
    s->device = c->device;
    s->nq = n_qubits;
    s->prec = prec;
    s->D = 1ll << n_qubits;
    s->owned = 0;
    s->data = dev_ptr;
    *out = s;
    API_END
}

namespace {

tq_state* new_sector_state(tq_ctx* c, int n_spatial, int n_alpha, int n_beta, int prec) {
    const SectorSpec sp = make_sector_spec(n_spatial, n_alpha, n_beta, TQ_JW);
    auto* s = new tq_state();
    s->ctx = c;
    s->device = c->device;
    s->nq = 2 * n_spatial;
    s->prec = prec;
    s->D = sector_dim(sp.n, sp.na, sp.nb);
    s->sector = 1;
    s->n_spatial = n_spatial;
    s->n_alpha = n_alpha;
    s->n_beta = n_beta;
    return s;
}

}  // namespace

extern "C" int tq_state_create_sector(tq_ctx* c, int n_spatial, int n_alpha, int n_beta, int prec,
                                      tq_state** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(2 * n_spatial <= TQ_MAX_STATE_QUBITS, "n_spatial out of range");
    set_device(c);
    tq_state* s = new_sector_state(c, n_spatial, n_alpha, n_beta, prec);
    s->owned = 1;
    try {
        s->data = dev_alloc((size_t)s->D * elem_bytes(prec));
        TQ_CUDA(cudaMemset(s->data, 0, (size_t)s->D * elem_bytes(prec)));
    } catch (...) {
        delete s;
        throw;
    }
    *out = s;
    API_END
}

extern "C" int tq_state_wrap_sector(tq_ctx* c, int n_spatial, int n_alpha, int n_beta, int prec, void* dev_ptr,
                                    tq_state** out) {
    API_BEGIN
    TQ_REQUIRE(c && out && dev_ptr, "null argument");
    *out = nullptr;
    check_prec(prec);
    TQ_REQUIRE(2 * n_spatial <= TQ_MAX_STATE_QUBITS, "n_spatial out of range");
    TQ_REQUIRE(((uintptr_t)dev_ptr & 15u) == 0, "state pointer must be 16-byte aligned");
    tq_state* s = new_sector_state(c, n_spatial, n_alpha, n_beta, prec);
    s->data = dev_ptr;
    *out = s;
    API_END
}

extern "C" int tq_state_data(const tq_state* s, void** dev_ptr, int* n_qubits, int* prec) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "state is null");
    if (dev_ptr) *dev_ptr = s->data;
    if (n_qubits) *n_qubits = s->nq;
    if (prec) *prec = s->prec;
    API_END
}

extern "C" int tq_state_set_hf(tq_state* s, int n_electrons, int mapping, void* stream) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "state is null");
    set_device(s->ctx);
    long long idx;
    if (s->sector) {
        // the lowest determinant (spin orbitals P < n_electrons) has rank 0
        // in its sector, and is outside any other
        check_mapping(mapping);
        TQ_REQUIRE(n_electrons >= 0 && n_electrons <= s->nq, "n_electrons out of range");
        TQ_REQUIRE((n_electrons + 1) / 2 == s->n_alpha && n_electrons / 2 == s->n_beta,
                   "the lowest determinant is not in this state's sector");
        idx = 0;
    } else {
        idx = (long long)hf_index(s->nq, n_electrons, mapping);
    }
    check_launch(s->ctx, launch_set_basis(s->data, s->prec, s->D, idx, as_stream(stream)));
    API_END
}

extern "C" int tq_state_free(tq_state* s) {
    if (!s) return TQ_OK;
    if (s->owned && s->data) {
        cudaSetDevice(s->device);
        cudaFree(s->data);
    }
    delete s;
    (void)cudaGetLastError();   // a failure while freeing is not reported to later calls
    return TQ_OK;
}

// ================================================================ hot path

namespace {

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

}  // namespace

extern "C" int tq_evolve_taylor5(tq_ctx* c, const tq_pool* p, int k, double theta, tq_state* psi,
                                 int renormalize, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p && psi, "null argument");
    TQ_REQUIRE(k >= 0 && k < p->M, "pool index out of range");
    TQ_REQUIRE(std::isfinite(theta), "theta is not finite");
    check_space(p, psi);
    set_device(c);
    cudaStream_t s = as_stream(stream);
    const int upt = c->pair_upt[psi->prec];
    const int tiles = update_tiles(p, psi->prec, upt);
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)tiles * sizeof(double)));
    const bool fin = launch_update(c, p, 1, psi->prec, upt, psi->data, nullptr, nullptr, k, theta, nullptr, part,
                                   nullptr, renormalize ? &c->step->norm2 : nullptr, s);
    if (renormalize) {
        if (!fin)
            launch(c, "norm_reduce", s, [&] { return launch_norm_reduce(part, psi->prec, 1, tiles, nullptr, &c->step->norm2, s); });
        launch(c, "scale", s, [&] { return launch_scale(psi->data, psi->prec, psi->D, &c->step->norm2, s); });
    }
    API_END
}

extern "C" int tq_evolve_taylor5_csr(tq_ctx* c, int n_qubits, const int* rowptr, const int* col,
                                     const void* val, double theta, tq_state* psi, int renormalize,
                                     void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && rowptr && col && val && psi, "null argument");
    TQ_REQUIRE(std::isfinite(theta), "theta is not finite");
    TQ_REQUIRE(psi->nq == n_qubits, "state and operator qubit counts differ");
    set_device(c);
    const long long D = psi->D;
    const size_t vb = (size_t)D * elem_bytes(psi->prec);
    double* acc = static_cast<double*>(scratch(c, S_U1, vb));
    double* v0 = static_cast<double*>(scratch(c, S_U2, vb));
    double* v1 = static_cast<double*>(scratch(c, S_W1, vb));
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)c->sm_count * 4 * sizeof(double)));
    launch(c, "taylor5_csr", as_stream(stream), [&] { return launch_taylor5_csr(n_qubits, psi->prec, rowptr, col, val, theta, psi->data, renormalize,
                                       acc, v0, v1, part, &c->step->norm2, c->sm_count, as_stream(stream)); });
    API_END
}

namespace {

// Partials needed by energy + gradients (+ line search) on this problem.
size_t partials_needed(long long D, int n_gitems, int nq, int sms) {
    size_t n = (size_t)energy_grid(D, sms) * 2;
    n = std::max(n, (size_t)16 * sms);      // any persistent energy grid (at most 8 blocks per SM)
    n = std::max(n, (size_t)std::max(n_gitems, 0));
    n = std::max(n, (size_t)512 * 6);            // the line search's six dots per block
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

}  // namespace

extern "C" int tq_energy(tq_ctx* c, const tq_ham* h, const tq_state* psi, double* E, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && psi && E, "null argument");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    double* part = prepare(c, h->D, nullptr, h->nq);
    run_energy(c, h, psi, part, s);
    int status = 0;
    TQ_CUDA(cudaMemcpyAsync(E, &c->step->energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaMemcpyAsync(&status, &c->step->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    raise_status(c, status, s);
    API_END
}

extern "C" int tq_energy_matrix_free(tq_ctx* c, const tq_ham* h, const tq_state* psi, double* E,
                                     void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && psi && E, "null argument");
    TQ_REQUIRE(!h->sector, "the matrix-free energy works in the full space only");
    check_space(h, psi);
    set_device(c);
    cudaStream_t s = as_stream(stream);
    double* part = prepare(c, h->D, nullptr, h->nq);
    launch(c, "energy_matrix_free", s, [&] { return launch_energy_matrix_free(h->view, psi->data, psi->prec, part, c->tickets + 1,
                                              c->step, c->sm_count, s); });
    TQ_CUDA(cudaMemcpyAsync(E, &c->step->energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    API_END
}

extern "C" int tq_pool_gradients(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi, double* g,
                                 int g_on_device, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi && g, "null argument");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    double* gd = g_on_device ? g : static_cast<double*>(scratch(c, S_G, (size_t)p->M * sizeof(double)));
    double* part = prepare(c, h->D, p, p->nq);
    run_gradients(c, h, p, psi, gd, part, s);
    if (!g_on_device) {
        int status = 0;
        TQ_CUDA(cudaMemcpyAsync(g, gd, (size_t)p->M * sizeof(double), cudaMemcpyDeviceToHost, s));
        TQ_CUDA(cudaMemcpyAsync(&status, &c->step->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        TQ_CUDA(cudaStreamSynchronize(s));
        raise_status(c, status, s);
    }
    API_END
}

namespace {

// The device buffers of an ADAPT step, allocated before any of its launches
// (and before a graph capture of them).
struct AdaptBufs {
    double* g;
    void* z;           // {psi, A psi, A^2 psi, 0} per row
    double2 *w0, *w1, *w2;
    double* part;
};

AdaptBufs adapt_buffers(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi) {
    const long long D = h->D;
    AdaptBufs b;
    b.g = static_cast<double*>(scratch(c, S_G, (size_t)p->M * sizeof(double)));
    const size_t vb = (size_t)D * sizeof(double2);
    b.z = scratch(c, S_U1, 4 * (size_t)D * elem_bytes(psi->prec));
    b.w1 = static_cast<double2*>(scratch(c, S_W1, vb));
    b.w2 = static_cast<double2*>(scratch(c, S_W2, vb));
    b.part = prepare(c, D, p, p->nq);
    b.w0 = static_cast<double2*>(c->scratch[S_W0]);
    return b;
}

// The launches of one ADAPT step on s (no host synchronisation): energy and
// gradients, selection, the line search when the angle is not given (theta
// NaN and no theta_list), the update and the renormalisation.  theta_list
// (device, optional) gives step step->iter its angle.
void enqueue_adapt_step(tq_ctx* c, const AdaptBufs& b, const tq_ham* h, const tq_pool* p, tq_state* psi, double eps,
                        double theta, const double* theta_list, cudaStream_t s) {
    const long long D = h->D;
    run_gradients(c, h, p, psi, b.g, b.part, s);
    launch(c, "select", s, [&] { return launch_select(b.g, p->M, eps, psi->prec, c->step, s); });
    if (std::isnan(theta) && !theta_list) {
        if (p->sector)
            launch(c, "apply_twice_sector", s, [&] { return launch_apply_twice_sector(p->view, c->step, psi->data,
                                                                                      psi->prec, b.z, s); });
        else
            launch(c, "apply_twice", s, [&] { return launch_apply_twice(p->view, c->step, psi->data, psi->prec, b.z, s); });
        // H psi, H A psi and H A^2 psi from one pass with one arithmetic (w0
        // is rewritten: the gradients that read it have run)
        launch(c, "line_spmv_gated", s, [&] { return launch_line_spmv_gated(h->view, b.z, b.w0, b.w1, b.w2, c->step,
                                                                             c->sm_count, s); });
        launch(c, "line_dots", s, [&] { return launch_line_dots(b.z, b.w0, b.w1, b.w2, psi->prec, D, b.part,
                                                                c->tickets + 2, c->step, s); });
    }
    launch(c, "line_search", s, [&] { return launch_line_search(c->step, theta, theta_list, c->line_sc, c->line_se,
                                                                c->tickets + 3, s); });
    const int upt = c->pair_upt[psi->prec];
    const int tiles = update_tiles(p, psi->prec, upt);
    if (!launch_update(c, p, 1, psi->prec, upt, psi->data, nullptr, nullptr, 0, 0.0, c->step, b.part, nullptr,
                       &c->step->norm2, s))
        launch(c, "norm_reduce", s, [&] { return launch_norm_reduce(b.part, psi->prec, 1, tiles, nullptr,
                                                                    &c->step->norm2, s); });
    launch(c, "scale_gated", s, [&] { return launch_scale_gated(psi->data, psi->prec, D, &c->step->norm2, c->step, s); });
}

void check_adapt_args(const tq_ham* h, const tq_pool* p, const tq_state* psi, double eps) {
    TQ_REQUIRE(std::isfinite(eps) && eps >= 0.0, "eps must be finite and >= 0");
    check_space(h, psi);
    check_space(p, psi);
    TQ_REQUIRE(h->prec == psi->prec, "state and Hamiltonian precisions differ");
}

}  // namespace

extern "C" int tq_adapt_step(tq_ctx* c, const tq_ham* h, const tq_pool* p, tq_state* psi, double eps,
                             double theta, tq_adapt_result* out, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi && out, "null argument");
    check_adapt_args(h, p, psi, eps);
    TQ_REQUIRE(std::isnan(theta) || std::isfinite(theta), "theta must be finite or NaN");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    const AdaptBufs b = adapt_buffers(c, h, p, psi);
    enqueue_adapt_step(c, b, h, p, psi, eps, theta, nullptr, s);
    DevStep hs;
    TQ_CUDA(cudaMemcpyAsync(&hs, c->step, sizeof(DevStep), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    raise_status(c, hs.status, s);
    out->energy = hs.energy;
    out->max_grad = hs.max_grad;
    out->selected = hs.selected;
    out->converged = hs.converged;
    out->theta = hs.converged ? 0.0 : hs.theta;
    if (!hs.converged && !(std::isfinite(hs.norm2) && hs.norm2 > 0.0))
        throw Error(TQ_ENUMERIC, "non-finite or zero norm after the update");
    API_END
}

extern "C" int tq_adapt_run(tq_ctx* c, const tq_ham* h, const tq_pool* p, tq_state* psi, double eps,
                            const double* thetas, int n_iter, tq_adapt_result* results, int* n_done, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi && results && n_done, "null argument");
    check_adapt_args(h, p, psi, eps);
    TQ_REQUIRE(n_iter >= 0, "n_iter < 0");
    *n_done = 0;
    if (n_iter == 0) return TQ_OK;
    if (thetas)
        for (int i = 0; i < n_iter; ++i) TQ_REQUIRE(std::isfinite(thetas[i]), "thetas must be finite");
    set_device(c);
    // the run goes on a stream of the context, after the caller's work
    TQ_CUDA(cudaStreamSynchronize(as_stream(stream)));
    if (!c->aux[1]) TQ_CUDA(cudaStreamCreateWithFlags(&c->aux[1], cudaStreamNonBlocking));
    cudaStream_t s = c->aux[1];
    const AdaptBufs b = adapt_buffers(c, h, p, psi);
    double* rec = static_cast<double*>(scratch(c, S_REC, (size_t)n_iter * 6 * sizeof(double)));
    double* dth = nullptr;
    if (thetas) {
        dth = static_cast<double*>(scratch(c, S_THETAS, (size_t)n_iter * sizeof(double)));
        TQ_CUDA(cudaMemcpyAsync(dth, thetas, (size_t)n_iter * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    TQ_CUDA(cudaMemsetAsync(&c->step->iter, 0, sizeof(int), s));
    const double nan = std::nan("");
    // step 0 directly (it also settles every lazily set launch attribute),
    // then one step captured as a graph and replayed: no host round trip
    // between steps
    enqueue_adapt_step(c, b, h, p, psi, eps, nan, dth, s);
    launch(c, "step_record", s, [&] { return launch_step_record(c->step, rec, n_iter, s); });
    if (n_iter > 1) {
        if (c->tracing) {
            for (int i = 1; i < n_iter; ++i) {
                enqueue_adapt_step(c, b, h, p, psi, eps, nan, dth, s);
                launch(c, "step_record", s, [&] { return launch_step_record(c->step, rec, n_iter, s); });
            }
        } else {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            TQ_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            try {
                enqueue_adapt_step(c, b, h, p, psi, eps, nan, dth, s);
                launch(c, "step_record", s, [&] { return launch_step_record(c->step, rec, n_iter, s); });
            } catch (...) {
                cudaStreamEndCapture(s, &graph);
                if (graph) cudaGraphDestroy(graph);
                throw;
            }
            TQ_CUDA(cudaStreamEndCapture(s, &graph));
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            TQ_CUDA(ie);
            cudaError_t le = cudaSuccess;
            for (int i = 1; i < n_iter && le == cudaSuccess; ++i) le = cudaGraphLaunch(exec, s);
            cudaGraphExecDestroy(exec);
            TQ_CUDA(le);
        }
    }
    std::vector<double> hr((size_t)n_iter * 6);
    int status = 0;
    TQ_CUDA(cudaMemcpyAsync(hr.data(), rec, hr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaMemcpyAsync(&status, &c->step->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    raise_status(c, status, s);
    int done = n_iter;
    for (int i = 0; i < n_iter; ++i) {
        const double* r = &hr[6 * (size_t)i];
        results[i].energy = r[0];
        results[i].max_grad = r[1];
        results[i].theta = r[2];
        results[i].selected = (int)r[3];
        results[i].converged = (int)r[4];
        if (r[5] != 0.0) {
            *n_done = i + 1;
            throw Error(TQ_ENUMERIC, "non-finite or zero norm after the update of step " + std::to_string(i));
        }
        if (results[i].converged && done == n_iter) done = i + 1;
    }
    *n_done = done;
    API_END
}

// ===================================================== ADAPT-VQE (re-optimised)

namespace {

// E(theta) and dE/dtheta of psi(theta) = U_n ... U_1 psi0 (Taylor-5 factors,
// no renormalisation): forward states phi_0 .. phi_n kept in scratch, the
// energy pass over phi_n (w = H psi), chi = w - E psi, then per factor from
// the last: the gradient dot, and chi <- U_j(-theta_j) chi.  `grad` (host)
// may be null; `psi_out` (device, D amplitudes) receives phi_n if not null.
double ansatz_energy_grad(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, int n, const int* ops,
                          const double* th, double* grad, void* psi_out, cudaStream_t s) {
    check_space(p, psi0);
    check_space(h, psi0);
    TQ_REQUIRE(h->prec == psi0->prec, "state and Hamiltonian precisions differ");
    TQ_REQUIRE(n >= 0, "n_ops < 0");
    for (int j = 0; j < n; ++j) {
        TQ_REQUIRE(ops[j] >= 0 && ops[j] < p->M, "pool index out of range");
        TQ_REQUIRE(std::isfinite(th[j]), "theta is not finite");
    }
    const int prec = psi0->prec;
    const long long D = psi0->D;
    const size_t vb = (size_t)D * elem_bytes(prec);
    double* part = prepare(c, D, p, p->nq);
    unsigned char* phis = static_cast<unsigned char*>(scratch(c, S_PHI, (size_t)(n + 1) * vb));
    void* chi = scratch(c, S_CHI, vb);
    double* gdev = static_cast<double*>(scratch(c, S_AG, (size_t)std::max(n, 1) * sizeof(double)));
    const int upt = c->pair_upt[prec];
    TQ_CUDA(cudaMemcpyAsync(phis, psi0->data, vb, cudaMemcpyDeviceToDevice, s));
    for (int j = 0; j < n; ++j) {
        unsigned char* dst = phis + (size_t)(j + 1) * vb;
        TQ_CUDA(cudaMemcpyAsync(dst, phis + (size_t)j * vb, vb, cudaMemcpyDeviceToDevice, s));
        launch_update(c, p, 1, prec, upt, dst, nullptr, nullptr, ops[j], th[j], nullptr, part, nullptr, nullptr, s);
    }
    tq_state last = *psi0;
    last.owned = 0;
    last.data = phis + (size_t)n * vb;
    run_energy(c, h, &last, part, s);
    if (grad) {
        launch(c, "residual", s, [&] { return launch_residual(static_cast<double2*>(c->scratch[S_W0]), last.data, chi, prec,
                                                              D, c->step, s); });
        for (int j = n - 1; j >= 0; --j) {
            const double t = th[j], t2 = t * t;
            const double c4 = 1.0 - t2 / 2.0 + t2 * t2 / 24.0, s4 = t * (1.0 - t2 / 6.0);
            launch(c, "ansatz_dot", s, [&] {
                return launch_ansatz_dot(p->view, ops[j], c4, s4, chi, phis + (size_t)j * vb, prec, D, part,
                                         c->tickets + 4, c->step, gdev + j, c->sm_count, s);
            });
            launch_update(c, p, 1, prec, upt, chi, nullptr, nullptr, ops[j], -t, nullptr, part, nullptr, nullptr, s);
        }
    }
    double E = 0.0;
    int status = 0;
    TQ_CUDA(cudaMemcpyAsync(&E, &c->step->energy, sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaMemcpyAsync(&status, &c->step->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (grad && n > 0) TQ_CUDA(cudaMemcpyAsync(grad, gdev, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (psi_out) TQ_CUDA(cudaMemcpyAsync(psi_out, last.data, vb, cudaMemcpyDeviceToDevice, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    raise_status(c, status, s);
    return E;
}

// BFGS on f with gradient g: inverse-Hessian update, backtracking line
// search (Armijo, halving), restart along -g when the direction does not
// descend; stops when max |g_i| < gtol or after max_iter iterations.
// Returns f at the result; x is updated in place.
template <typename FG>
double bfgs(FG fg, std::vector<double>& x, double gtol, int max_iter, int* n_eval) {
    const size_t n = x.size();
    std::vector<double> g(n), gn(n), xn(n), d(n), sv(n), yv(n), Hy(n);
    std::vector<double> H(n * n, 0.0);
    for (size_t i = 0; i < n; ++i) H[i * n + i] = 1.0;
    double f = fg(x, g);
    int evals = 1;
    auto gmax = [](const std::vector<double>& v) {
        double m = 0.0;
        for (double e : v) m = std::max(m, std::fabs(e));
        return m;
    };
    for (int it = 0; it < max_iter && gmax(g) >= gtol; ++it) {
        double gd = 0.0;
        for (size_t i = 0; i < n; ++i) {
            double v = 0.0;
            for (size_t j = 0; j < n; ++j) v -= H[i * n + j] * g[j];
            d[i] = v;
            gd += v * g[i];
        }
        if (!(gd < 0.0)) {                         // not a descent direction: restart
            std::fill(H.begin(), H.end(), 0.0);
            for (size_t i = 0; i < n; ++i) H[i * n + i] = 1.0, d[i] = -g[i];
            gd = 0.0;
            for (size_t i = 0; i < n; ++i) gd -= g[i] * g[i];
        }
        double a = 1.0, fn = f;
        bool ok = false;
        for (int ls = 0; ls < 40; ++ls) {
            for (size_t i = 0; i < n; ++i) xn[i] = x[i] + a * d[i];
            fn = fg(xn, gn);
            ++evals;
            if (fn <= f + 1e-4 * a * gd) {
                ok = true;
                break;
            }
            a *= 0.5;
        }
        if (!ok) break;                            // no decrease along d: converged to rounding
        double sy = 0.0, yy = 0.0;
        for (size_t i = 0; i < n; ++i) {
            sv[i] = xn[i] - x[i];
            yv[i] = gn[i] - g[i];
            sy += sv[i] * yv[i];
            yy += yv[i] * yv[i];
        }
        if (sy > 1e-300) {
            if (it == 0) {                         // scale the first inverse Hessian
                std::fill(H.begin(), H.end(), 0.0);
                for (size_t i = 0; i < n; ++i) H[i * n + i] = sy / yy;
            }
            double yHy = 0.0;
            for (size_t i = 0; i < n; ++i) {
                double v = 0.0;
                for (size_t j = 0; j < n; ++j) v += H[i * n + j] * yv[j];
                Hy[i] = v;
                yHy += yv[i] * v;
            }
            const double rho = 1.0 / sy;
            for (size_t i = 0; i < n; ++i)
                for (size_t j = 0; j < n; ++j)
                    H[i * n + j] += -rho * (Hy[i] * sv[j] + sv[i] * Hy[j]) + (rho * rho * yHy + rho) * sv[i] * sv[j];
        }
        x = xn;
        g = gn;
        f = fn;
    }
    if (n_eval) *n_eval = evals;
    return f;
}

// The operator choice of the ADAPT step on host gradients (the tie rule of
// k_select): the lowest index within tau of max |g|.
int select_host(const std::vector<double>& g, int prec, double* gmax_out) {
    double gm = 0.0;
    for (double v : g) gm = std::max(gm, std::fabs(v));
    const double tau = prec == TQ_C128 ? 1e-9 * std::max(1.0, gm) : 1e-5;
    int k = 0;
    for (size_t i = 0; i < g.size(); ++i)
        if (std::fabs(g[i]) >= gm - tau) {
            k = (int)i;
            break;
        }
    *gmax_out = gm;
    return k;
}

}  // namespace

extern "C" int tq_ansatz_energy_grad(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, int n_ops,
                                     const int* ops, const double* thetas, double* E, double* grad, tq_state* psi_out,
                                     void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi0 && E, "null argument");
    TQ_REQUIRE(n_ops == 0 || (ops && thetas), "null argument");
    if (psi_out) {
        check_space(p, psi_out);
        TQ_REQUIRE(psi_out->prec == psi0->prec, "output state precision differs");
    }
    set_device(c);
    *E = ansatz_energy_grad(c, h, p, psi0, n_ops, ops, thetas, grad, psi_out ? psi_out->data : nullptr,
                            as_stream(stream));
    API_END
}

extern "C" int tq_adapt_vqe(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi0, double eps,
                            int max_ops, double gtol, int max_iter, int* n_ops, int* ops_out, double* thetas_out,
                            double* energies_out, tq_state* psi_out) {
    API_BEGIN
    TQ_REQUIRE(c && h && p && psi0 && n_ops && ops_out && thetas_out && energies_out, "null argument");
    TQ_REQUIRE(max_ops >= 0 && max_iter >= 0, "max_ops and max_iter must be >= 0");
    TQ_REQUIRE(std::isfinite(eps) && eps >= 0.0 && std::isfinite(gtol) && gtol > 0.0, "eps >= 0 and gtol > 0 required");
    check_space(p, psi0);
    check_space(h, psi0);
    set_device(c);
    cudaStream_t s = 0;
    const long long D = psi0->D;
    std::vector<int> ops;
    std::vector<double> th;
    std::vector<double> g(p->M);
    int count = 0;
    for (int it = 0; it < max_ops; ++it) {
        // psi(theta) and every pool gradient there
        void* work = scratch(c, S_STAGE, (size_t)D * elem_bytes(psi0->prec));
        ansatz_energy_grad(c, h, p, psi0, (int)ops.size(), ops.data(), th.data(), nullptr, work, s);
        tq_state cur = *psi0;
        cur.owned = 0;
        cur.data = work;
        double* gd = static_cast<double*>(scratch(c, S_G, (size_t)p->M * sizeof(double)));
        double* part = prepare(c, D, p, p->nq);
        run_gradients(c, h, p, &cur, gd, part, s);
        TQ_CUDA(cudaMemcpyAsync(g.data(), gd, (size_t)p->M * sizeof(double), cudaMemcpyDeviceToHost, s));
        TQ_CUDA(cudaStreamSynchronize(s));
        double gmax = 0.0;
        const int k = select_host(g, psi0->prec, &gmax);
        if (gmax < eps) break;
        ops.push_back(k);
        th.push_back(0.0);
        const double E = bfgs(
            [&](const std::vector<double>& x, std::vector<double>& gr) {
                return ansatz_energy_grad(c, h, p, psi0, (int)ops.size(), ops.data(), x.data(), gr.data(), nullptr, s);
            },
            th, gtol, max_iter, nullptr);
        ops_out[count] = k;
        energies_out[count] = E;
        ++count;
    }
    for (int j = 0; j < count; ++j) thetas_out[j] = th[j];
    *n_ops = count;
    if (psi_out) {
        check_space(p, psi_out);
        ansatz_energy_grad(c, h, p, psi0, count, ops.data(), th.data(), nullptr, psi_out->data, s);
    }
    API_END
}

// ================================================================ batched

extern "C" int tq_evolve_taylor5_batch(tq_ctx* c, const tq_pool* p, int n_states, int prec, void* psi,
                                       const int* k, const double* theta, double* norm2, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(n_states >= 0, "n_states < 0");
    check_prec(prec);
    if (n_states == 0) return TQ_OK;   // an empty batch is a no-op
    TQ_REQUIRE(psi && k && theta, "null argument");
    TQ_REQUIRE(((uintptr_t)psi & 15u) == 0, "psi must be 16-byte aligned");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    const int upt = c->pair_upt[prec];
    const int tiles = update_tiles(p, prec, upt);
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)n_states * tiles * sizeof(double)));
    const bool fin = launch_update(c, p, n_states, prec, upt, psi, k, theta, 0, 0.0, nullptr, part, norm2, nullptr, s);
    if (norm2 && !fin)
        launch(c, "norm_reduce", s, [&] { return launch_norm_reduce(part, prec, n_states, tiles, norm2, nullptr, s); });
    API_END
}

extern "C" int tq_evolve_taylor5_batch_support(tq_ctx* c, const tq_pool* p, int n_states, int prec, void* psi,
                                               const int* k, const double* theta, double* norm2, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the support-only update takes full-space pools (sector states: tq_evolve_taylor5_batch)");
    TQ_REQUIRE(n_states >= 0, "n_states < 0");
    check_prec(prec);
    if (n_states == 0) return TQ_OK;   // an empty batch is a no-op
    TQ_REQUIRE(psi && k && theta, "null argument");
    TQ_REQUIRE(((uintptr_t)psi & 15u) == 0, "psi must be 16-byte aligned");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    const int ppt = c->supp_ppt[prec];
    const int tps = support_tiles(p->nq, n_states, ppt, c->sm_count);
    const int parts = support_parts(tps);
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)n_states * parts * sizeof(double)));
    launch(c, "taylor5_support", s, [&] {
        return launch_taylor5_support(p->view, n_states, prec, ppt, psi, k, theta, part, tps, norm2, c->sm_count, s);
    });
    if (norm2 && tps > 1)
        launch(c, "norm_carry", s, [&] { return launch_norm_carry(part, prec, n_states, parts, norm2, norm2, nullptr, s); });
    API_END
}

extern "C" int tq_evolve_taylor5_batch_support_host(tq_ctx* c, const tq_pool* p, int n_states, int prec,
                                                    void* psi_host, const int* k_host, const double* theta_host,
                                                    double* norm2_host) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the support-only update takes full-space pools (sector states: tq_evolve_taylor5_batch)");
    TQ_REQUIRE(n_states >= 0, "n_states < 0");
    check_prec(prec);
    if (n_states == 0) return TQ_OK;   // an empty batch is a no-op
    TQ_REQUIRE(psi_host && k_host && theta_host, "null argument");
    TQ_REQUIRE(((uintptr_t)psi_host & 15u) == 0, "psi must be 16-byte aligned");
    set_device(c);
    // the kernel reads and writes the states where they are, over the
    // host link: they must be page-locked and mapped for this device
    cudaPointerAttributes attr{};
    const cudaError_t ae = cudaPointerGetAttributes(&attr, psi_host);
    if (ae != cudaSuccess) (void)cudaGetLastError();
    TQ_REQUIRE(ae == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr,
               "psi_host must be page-locked host memory mapped for the device (cudaHostAlloc / cudaHostRegister)");
    void* psi = attr.devicePointer;
    cudaStream_t s = c->aux[0];
    if (!s) TQ_CUDA(cudaStreamCreateWithFlags(&c->aux[0], cudaStreamNonBlocking));
    s = c->aux[0];
    const int ppt = c->supp_ppt[prec];
    const int tps = support_tiles(p->nq, n_states, ppt, c->sm_count);
    const int parts = support_parts(tps);
    unsigned char* buf = static_cast<unsigned char*>(
        scratch(c, S_HOSTB, (size_t)n_states * (sizeof(int) + 2 * sizeof(double)) + 64));
    int* dk = reinterpret_cast<int*>(buf);
    double* dth = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(dk + n_states) + 15) & ~(uintptr_t)15);
    double* dn = dth + n_states;
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)n_states * parts * sizeof(double)));
    TQ_CUDA(cudaMemcpyAsync(dk, k_host, (size_t)n_states * sizeof(int), cudaMemcpyHostToDevice, s));
    TQ_CUDA(cudaMemcpyAsync(dth, theta_host, (size_t)n_states * sizeof(double), cudaMemcpyHostToDevice, s));
    if (norm2_host)
        TQ_CUDA(cudaMemcpyAsync(dn, norm2_host, (size_t)n_states * sizeof(double), cudaMemcpyHostToDevice, s));
    double* n2 = norm2_host ? dn : nullptr;
    launch(c, "taylor5_support_host", s, [&] {
        return launch_taylor5_support(p->view, n_states, prec, ppt, psi, dk, dth, part, tps, n2, c->sm_count, s);
    });
    if (n2 && tps > 1)
        launch(c, "norm_carry", s, [&] { return launch_norm_carry(part, prec, n_states, parts, n2, n2, nullptr, s); });
    if (norm2_host)
        TQ_CUDA(cudaMemcpyAsync(norm2_host, dn, (size_t)n_states * sizeof(double), cudaMemcpyDeviceToHost, s));
    TQ_CUDA(cudaStreamSynchronize(s));
    API_END
}

extern "C" int tq_ctx_set_support_schedule(tq_ctx* c, int prec, int pairs_per_thread) {
    API_BEGIN
    TQ_REQUIRE(c, "null argument");
    check_prec(prec);
    TQ_REQUIRE(pair_upt_valid(std::abs(pairs_per_thread)), "pairs_per_thread must be +-1, +-2, +-4 or +-8");
    c->supp_ppt[prec] = pairs_per_thread;
    API_END
}

extern "C" int tq_evolve_taylor5_batch_host(tq_ctx* c, const tq_pool* p, int n_states, int prec,
                                            void* psi_host, const int* k_host, const double* theta_host,
                                            double* norm2_host) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(n_states >= 0, "n_states < 0");
    check_prec(prec);
    if (n_states == 0) return TQ_OK;   // an empty batch is a no-op
    TQ_REQUIRE(psi_host && k_host && theta_host, "null argument");
    set_device(c);
    for (auto& st : c->aux)
        if (!st) TQ_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    const long long D = state_len(p);
    const size_t sb = (size_t)D * elem_bytes(prec);
    // chunk of about 64 MiB of states per stream
    int chunk = (int)std::max<long long>(1, (64ll << 20) / (long long)sb);
    chunk = std::min(chunk, n_states);
    const int upt = c->pair_upt[prec];
    const int tiles = update_tiles(p, prec, upt);
    const size_t per_stream = (size_t)chunk * sb + (size_t)chunk * (sizeof(int) + 2 * sizeof(double)) +
                              (size_t)chunk * tiles * sizeof(double) + 256;
    unsigned char* stage = static_cast<unsigned char*>(scratch(c, S_STAGE, 3 * per_stream));
    for (int c0 = 0, it = 0; c0 < n_states; c0 += chunk, ++it) {
        const int n = std::min(chunk, n_states - c0);
        cudaStream_t s = c->aux[it % 3];
        unsigned char* base = stage + (size_t)(it % 3) * per_stream;
        void* dpsi = base;
        int* dk = reinterpret_cast<int*>(base + (size_t)chunk * sb);
        double* dth = reinterpret_cast<double*>(
            (reinterpret_cast<uintptr_t>(dk + chunk) + 15) & ~(uintptr_t)15);
        double* dn = dth + chunk;
        double* part = dn + chunk;
        TQ_CUDA(cudaMemcpyAsync(dpsi, static_cast<unsigned char*>(psi_host) + (size_t)c0 * sb, (size_t)n * sb,
                                cudaMemcpyHostToDevice, s));
        TQ_CUDA(cudaMemcpyAsync(dk, k_host + c0, (size_t)n * sizeof(int), cudaMemcpyHostToDevice, s));
        TQ_CUDA(cudaMemcpyAsync(dth, theta_host + c0, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
        const bool fin = launch_update(c, p, n, prec, upt, dpsi, dk, dth, 0, 0.0, nullptr, part,
                                       norm2_host ? dn : nullptr, nullptr, s);
        TQ_CUDA(cudaMemcpyAsync(static_cast<unsigned char*>(psi_host) + (size_t)c0 * sb, dpsi, (size_t)n * sb,
                                cudaMemcpyDeviceToHost, s));
        if (norm2_host) {
            if (!fin) launch(c, "norm_reduce", s, [&] { return launch_norm_reduce(part, prec, n, tiles, dn, nullptr, s); });
            TQ_CUDA(cudaMemcpyAsync(norm2_host + c0, dn, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    }
    for (auto& st : c->aux) TQ_CUDA(cudaStreamSynchronize(st));
    API_END
}
