// C ABI of the library (declared in include/tq.h): the context (schedules,
// autotuners, tracing), host-only algebra, and the Hamiltonian, pool and
// state objects.  The hot path is in api_path.cu, ADAPT-VQE in api_vqe.cu,
// the helpers they share in api_common.cu.
#include "api_internal.h"
#include "dev.cuh"
#include "grad.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

using namespace tq;
using namespace tq::api;

namespace {

thread_local std::string g_last_error;

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
        c->line_se = static_cast<long long*>(dev_alloc((4096 + 64) * sizeof(long long)));
        c->line_rank = static_cast<int*>(dev_alloc(4096 * sizeof(int)));
        {
            std::vector<int> rank(4096);
            line_rank_table(rank.data());
            TQ_CUDA(cudaMemcpy(c->line_rank, rank.data(), 4096 * sizeof(int), cudaMemcpyHostToDevice));
        }
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
    if (c->line_rank) cudaFree(c->line_rank);
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
                return launch_taylor5_support(p->view, n_states, prec, u, psi, dk, dth, part, tps, dn, c->sm_count, 0,
                                              0, c->tickets + TICKET_SUPPORT_SCHED);
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

extern "C" int tq_mapping_relabelled(int base_mapping, int n_qubits, const int* order, int* mapping_out) {
    API_BEGIN
    TQ_REQUIRE(order && mapping_out, "null argument");
    *mapping_out = register_relabelled(base_mapping, n_qubits, order);
    API_END
}

extern "C" int tq_pool_sector_order(int n_spatial, int n_electrons, int base_mapping, int low_bits,
                                    int* order_out) {
    API_BEGIN
    TQ_REQUIRE(order_out, "null argument");
    TQ_REQUIRE(n_spatial >= 1 && n_spatial <= TQ_MAX_SPATIAL, "n_spatial out of range [1, 15]");
    const auto o = pool_sector_order(n_spatial, n_electrons, base_mapping, low_bits);
    std::copy(o.begin(), o.end(), order_out);
    API_END
}

extern "C" int tq_mapping_linear(int base_mapping, int n_qubits, const unsigned long long* rows, int* mapping_out) {
    API_BEGIN
    TQ_REQUIRE(rows && mapping_out, "null argument");
    TQ_REQUIRE(n_qubits >= 1 && n_qubits <= 2 * TQ_MAX_SPATIAL, "n_qubits out of range [1, 30]");
    std::vector<uint64_t> r(rows, rows + n_qubits);
    *mapping_out = register_linear(base_mapping, n_qubits, r.data());
    API_END
}

extern "C" int tq_pool_sector_basis(int n_spatial, int n_electrons, int base_mapping, int low_bits,
                                    unsigned long long* rows_out) {
    API_BEGIN
    TQ_REQUIRE(rows_out, "null argument");
    TQ_REQUIRE(n_spatial >= 1 && n_spatial <= TQ_MAX_SPATIAL, "n_spatial out of range [1, 15]");
    const auto m = pool_sector_basis(n_spatial, n_electrons, base_mapping, low_bits);
    std::copy(m.begin(), m.end(), rows_out);
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
        p->unit = true;
        for (int k = 0; k < M; ++k) p->unit = p->unit && std::fabs(fc0d[k]) == 1.0;
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
