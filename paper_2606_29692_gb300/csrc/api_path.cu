// C ABI: the hot path (Taylor-5 updates, energy, gradients, the ADAPT
// step and run) and the batched updates.
#include "api_internal.h"
#include "dev.cuh"
#include "grad.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace tq;
using namespace tq::api;

// ================================================================ hot path


extern "C" int tq_evolve_taylor5(tq_ctx* c, const tq_pool* p, int k, double theta, tq_state* psi,
                                 int renormalize, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p && psi, "null argument");
    TQ_REQUIRE(k >= 0 && k < p->M, "pool index out of range");
    TQ_REQUIRE(std::isfinite(theta), "theta is not finite");
    check_space(p, psi);
    set_device(c);
    cudaStream_t s = as_stream(stream);
    if (!p->sector && taylor5_single_ready(p->nq, psi->prec)) {
        // one launch: update, norm and rescale in one thread-block cluster
        launch(c, "taylor5_single", s, [&] {
            return launch_taylor5_single(p->view, psi->prec, p->unit, k, theta, nullptr, psi->data, renormalize,
                                         renormalize ? &c->step->norm2 : nullptr, s);
        });
        return TQ_OK;
    }
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
    b.z = nullptr;
    b.w1 = b.w2 = nullptr;
    if (p->sector) {   // the record pass of a sector pool's line search
        b.z = scratch(c, S_U1, 4 * (size_t)D * elem_bytes(psi->prec));
        b.w1 = static_cast<double2*>(scratch(c, S_W1, vb));
        b.w2 = static_cast<double2*>(scratch(c, S_W2, vb));
    }
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
        if (p->sector) {
            launch(c, "apply_twice_sector", s, [&] { return launch_apply_twice_sector(p->view, c->step, psi->data,
                                                                                      psi->prec, b.z, s); });
            // H psi, H A psi and H A^2 psi from one pass with one arithmetic
            // (w0 is rewritten: the gradients that read it have run)
            launch(c, "line_spmv_gated", s, [&] { return launch_line_spmv_gated(h->view, b.z, b.w0, b.w1, b.w2,
                                                                                 c->step, c->sm_count, s); });
            launch(c, "line_dots", s, [&] { return launch_line_dots(b.z, b.w0, b.w1, b.w2, psi->prec, D, b.part,
                                                                    c->tickets + 2, c->step, s); });
        } else {
            // the rows of the chosen generator's support only
            launch(c, "line_support", s, [&] { return launch_line_support(h->view, p->view, psi->data, c->step,
                                                                          b.part, c->tickets + 2, c->sm_count, s); });
        }
    }
    launch(c, "line_search", s, [&] { return launch_line_search(c->step, theta, theta_list, c->line_sc, c->line_rank, c->line_se,
                                                                c->tickets + 3, s); });
    if (!p->sector && taylor5_single_ready(p->nq, psi->prec)) {
        // the update, its norm and the rescale in one launch
        launch(c, "taylor5_single_gated", s, [&] {
            return launch_taylor5_single(p->view, psi->prec, p->unit, 0, 0.0, c->step, psi->data, 1, &c->step->norm2, s);
        });
        return;
    }
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
        return launch_taylor5_support(p->view, n_states, prec, ppt, psi, k, theta, part, tps, norm2, c->sm_count, s,
                                      c->supp_ctas[prec], c->tickets + TICKET_SUPPORT_SCHED);
    });
    if (norm2 && tps > 1)
        launch(c, "norm_carry", s, [&] { return launch_norm_carry(part, prec, n_states, parts, norm2, norm2, nullptr, s); });
    API_END
}

extern "C" int tq_evolve_taylor5_batch_support_touch(tq_ctx* c, const tq_pool* p, int n_states, int prec,
                                                     void* psi, const int* k, double* norm2, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the support-only update takes full-space pools");
    TQ_REQUIRE(n_states >= 0, "n_states < 0");
    check_prec(prec);
    if (n_states == 0) return TQ_OK;
    TQ_REQUIRE(psi && k, "null argument");
    TQ_REQUIRE(((uintptr_t)psi & 15u) == 0, "psi must be 16-byte aligned");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    const int ppt = c->supp_ppt[prec] < 0 ? c->supp_ppt[prec] : -c->supp_ppt[prec];
    const int tps = support_tiles(p->nq, n_states, ppt, c->sm_count);
    const int parts = support_parts(tps);
    double* part = static_cast<double*>(scratch(c, S_PART, (size_t)n_states * parts * sizeof(double)));
    // theta is read by the tile set-up and not used: any finite values
    double* th = static_cast<double*>(scratch(c, S_HOSTB, (size_t)n_states * sizeof(double)));
    TQ_CUDA(cudaMemsetAsync(th, 0, (size_t)n_states * sizeof(double), s));
    launch(c, "taylor5_support_touch", s, [&] {
        return launch_taylor5_support_touch(p->view, n_states, prec, ppt, psi, k, th, part, tps, norm2, c->sm_count, s,
                                            c->supp_ctas[prec], c->tickets + TICKET_SUPPORT_SCHED);
    });
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
        return launch_taylor5_support(p->view, n_states, prec, ppt, psi, dk, dth, part, tps, n2, c->sm_count, s,
                                      c->supp_ctas[prec], c->tickets + TICKET_SUPPORT_SCHED);
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

extern "C" int tq_evolve_taylor5_batch_grouped(tq_ctx* c, const tq_pool* p, int n_groups, int prec, void* psi,
                                               const int* k, const double* theta, double* norm2, void* stream) {
    API_BEGIN
    TQ_REQUIRE(c && p, "null argument");
    TQ_REQUIRE(!p->sector, "the grouped update takes full-space pools");
    TQ_REQUIRE(n_groups >= 0, "n_groups < 0");
    check_prec(prec);
    if (n_groups == 0) return TQ_OK;   // an empty batch is a no-op
    TQ_REQUIRE(psi && k && theta, "null argument");
    TQ_REQUIRE(((uintptr_t)psi & 31u) == 0, "psi must be 32-byte aligned");
    set_device(c);
    cudaStream_t s = as_stream(stream);
    launch(c, "taylor5_grouped", s, [&] {
        return launch_taylor5_grouped(p->view, n_groups, prec, c->grouped_lanes[prec], c->grouped_ppt[prec], psi, k,
                                      theta, norm2,
                                      c->sm_count, s);
    });
    API_END
}

extern "C" int tq_ctx_set_grouped_schedule(tq_ctx* c, int prec, int lanes_per_row, int pairs_per_thread) {
    API_BEGIN
    TQ_REQUIRE(c, "null argument");
    check_prec(prec);
    TQ_REQUIRE(grouped_schedule_ok(prec, lanes_per_row, pairs_per_thread),
               "lanes_per_row must be 1, 2 or (complex64) 4 and pairs_per_thread 1, 2 or 4");
    c->grouped_lanes[prec] = lanes_per_row;
    c->grouped_ppt[prec] = pairs_per_thread;
    API_END
}

extern "C" int tq_ctx_set_support_occupancy(tq_ctx* c, int prec, int ctas_per_sm) {
    API_BEGIN
    TQ_REQUIRE(c, "null argument");
    check_prec(prec);
    TQ_REQUIRE(ctas_per_sm >= 0 && ctas_per_sm <= 32, "ctas_per_sm must be in [0, 32]");
    c->supp_ctas[prec] = ctas_per_sm;
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
