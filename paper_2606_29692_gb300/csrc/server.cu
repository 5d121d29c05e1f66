// Request loop with continuous batching over resident states and operators.
//
// Sessions (states) and Hamiltonians/pools stay in device memory.  Requests
// (evolve with a pool op and angle, energy, all gradients) are queued by any
// host thread; a server thread forms each tick from the queue in arrival
// order: at most one request per session (so a session's requests run in
// submission order), at most max_batch requests, and only while the scratch
// arena has room for the request's working memory (w = H psi, gradients and
// their partials): admission is by HBM footprint.  A tick is up to six
// launches, each covering every admitted request of its kind: energy SpMV,
// gradients, selection, the Taylor-5 pair update, its norm and the rescale.
// Work items are found by binary search over per-request prefix counts, so
// a tick costs one descriptor upload.  Ticks run in order on one stream; the
// host forms tick i+1 while tick i runs and posts completions when a tick's
// event has fired.  Every reduction is ordered per request, so a request's
// result does not depend on what else shares its tick.
#include "dev.cuh"
#include "grad.cuh"
#include "host_util.h"
#include "pair.cuh"
#include "spmv.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>

namespace tq {

struct ReqDev {
    long long D;
    void* psi;
    const double* diag;
    const int* rowptr;
    const int* col;
    const void* val;
    PoolView pool;
    double theta;
    double2* w64;
    float2* w32;
    double* g;
    double* gpart;
    unsigned* gtick;
    double energy, e_den, max_grad, norm2;
    int kind, M, k, argmax;
    unsigned etick;
    int pad;
};

namespace {

constexpr int SV_BS = 256;
constexpr int MAX_TICK = 2048;

// index block of a tick, in ints
struct Idx {
    int e_off[MAX_TICK + 1];   // energy items per E entry (prefix)
    int g_off[MAX_TICK + 1];   // gradient items per G entry (prefix)
    int g_pos[MAX_TICK];       // position of each G entry in E
    int p_off[MAX_TICK + 1];   // pair tiles per P entry (prefix)
    int p_base[MAX_TICK + 1];  // first norm-partial slot per P entry
};

__device__ __forceinline__ int find_req(const int* off, int n, int it) {
    int lo = 0, hi = n;   // off[0] = 0 <= it < off[n]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= it) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <typename T, typename VT, int L>
__global__ void __launch_bounds__(SV_BS)
ks_energy(ReqDev* E, const Idx* ix, int n, double* epart) {
    using V = typename C2<T>::type;
    __shared__ double sh[2 * (SV_BS / 32)];
    __shared__ bool last;
    const int total = ix->e_off[n];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int q = find_req(ix->e_off, n, it);
        ReqDev& d = E[q];
        const long long r0 = (long long)(it - ix->e_off[q]) * ENERGY_ROWS;
        const long long r1 = min(r0 + ENERGY_ROWS, d.D);
        double num = 0.0, den = 0.0;
        energy_rows<T, VT, L>(d.rowptr, d.col, static_cast<const VT*>(d.val), d.diag,
                              static_cast<const V*>(d.psi), d.w64, d.w32, r0, r1, num, den);
        double v[2] = {num, den};
        block_sum<2>(v, sh);
        if (threadIdx.x == 0) {
            epart[2 * it] = v[0];
            epart[2 * it + 1] = v[1];
            __threadfence();
            last = atomicAdd(&d.etick, 1u) == (unsigned)(ix->e_off[q + 1] - ix->e_off[q]) - 1;
        }
        __syncthreads();
        if (last) {
            double a, b;
            block_sum_pairs(epart, ix->e_off[q], ix->e_off[q + 1] - ix->e_off[q], sh, a, b);
            if (threadIdx.x == 0) {
                d.e_den = b;
                d.energy = a / b;
            }
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(GRAD_TPB)
ks_grad(ReqDev* E, const Idx* ix, int ng) {
    using V = typename C2<T>::type;
    __shared__ double sh[GRAD_TPB / 32];
    __shared__ bool last;
    const int total = ix->g_off[ng];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int j = find_req(ix->g_off, ng, it);
        ReqDev& d = E[ix->g_pos[j]];
        const int li = it - ix->g_off[j];
        const int2 kc = d.pool.gitems[li];
        const int k = kc.x;
        const SuppRec s = load_supp(d.pool, k);
        const uint32_t size = (uint32_t)(d.D >> s.m);
        const uint32_t u0 = (uint32_t)kc.y * GRAD_CHUNK;
        const uint32_t cnt = min((uint32_t)GRAD_CHUNK, size - u0);
        const T c0 = sizeof(T) == 4 ? (T)d.pool.fc0f[k] : (T)d.pool.fc0d[k];
        double v;
        if constexpr (sizeof(T) == 4) v = grad_item<T>(s, c0, d.w32, static_cast<const V*>(d.psi), u0, cnt, sh);
        else v = grad_item<T>(s, c0, d.w64, static_cast<const V*>(d.psi), u0, cnt, sh);
        const int f0 = d.pool.gfirst[k], f1 = d.pool.gfirst[k + 1];
        if (threadIdx.x == 0) {
            d.gpart[li] = v;
            __threadfence();
            last = atomicAdd(&d.gtick[k], 1u) == (unsigned)(f1 - f0) - 1;
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            double acc = 0.0;
            for (int i = f0; i < f1; ++i) acc += __ldcg(d.gpart + i);
            d.g[k] = 2.0 * acc / d.e_den;
        }
        __syncthreads();
    }
}

// One warp per gradient request: max |g| and the lowest index within tau of
// it (the ADAPT selection rule).
__global__ void ks_select(ReqDev* E, const Idx* ix, int ng, int prec) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= ng) return;
    ReqDev& d = E[ix->g_pos[j]];
    double m = 0.0;
    for (int k = lane; k < d.M; k += 32) m = fmax(m, fabs(d.g[k]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const double tau = prec == TQ_C128 ? 1e-9 * fmax(1.0, m) : 1e-5;
    int best = d.M;
    for (int k = lane; k < d.M; k += 32)
        if (fabs(d.g[k]) >= m - tau && k < best) best = k;
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) {
        d.max_grad = m;
        d.argmax = best < d.M ? best : 0;
    }
}

template <typename T>
__global__ void __launch_bounds__(PAIR_BS)
ks_pair(ReqDev* P, const Idx* ix, int np, double* npart) {
    constexpr int NW = PAIR_BS / 32;
    const int warp = threadIdx.x >> 5;
    const int total = ix->p_off[np];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        const int q = find_req(ix->p_off, np, it);
        ReqDev& d = P[q];
        const int tl = it - ix->p_off[q];
        const OpRec<T> op = make_rec<T>(d.pool, d.k);
        const T tp = pair_tile<T, 2>(op, d.theta, static_cast<typename C2<T>::type*>(d.psi), (uint32_t)tl,
                                     (uint32_t)(d.D >> 2));
        store_partial(npart + (long long)ix->p_base[q] + (long long)tl * NW + warp, tp);
    }
}

template <bool PAIRS>
__global__ void ks_norm(ReqDev* P, const Idx* ix, int np, const double* npart) {
    const int lane = threadIdx.x & 31;
    const int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= np) return;
    double acc = 0.0;
    for (int i = ix->p_base[q] + lane; i < ix->p_base[q + 1]; i += 32) {
        const double* slot = npart + i;
        if (PAIRS) {
            const float2 hl = *reinterpret_cast<const float2*>(slot);
            acc += (double)hl.x + (double)hl.y;
        } else {
            acc += *slot;
        }
    }
    acc = warp_sum(acc);
    if (lane == 0) P[q].norm2 = acc;
}

template <typename T>
__global__ void ks_scale(ReqDev* P, int np) {
    using V = typename C2<T>::type;
    for (int q = blockIdx.y; q < np; q += gridDim.y) {
        ReqDev& d = P[q];
        const double sc = 1.0 / sqrt(d.norm2);
        V* psi = static_cast<V*>(d.psi);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.D;
             i += (long long)gridDim.x * blockDim.x) {
            V v = psi[i];
            v.x = (T)((double)v.x * sc);
            v.y = (T)((double)v.y * sc);
            psi[i] = v;
        }
    }
}

template <typename K>
int resident(K kernel, int bs, int sms) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, bs, 0);
    return std::max(1, per) * sms;
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace tq

using namespace tq;

struct tq_server {
    int device = 0;     // the context's device, kept for freeing after the context
    tq_ctx* ctx = nullptr;
    int prec = TQ_C64;
    size_t budget = 0, states_bytes = 0;
    int max_batch = 0;
    size_t max_queue = 1 << 20;
    std::vector<const tq_ham*> hams;
    std::vector<const tq_pool*> pools;
    struct Session { int ham; void* psi; long long D; int nq; };
    std::vector<Session> sessions;
    std::vector<void*> allocs;
    unsigned char* arena = nullptr;    // per-request working memory
    size_t arena_bytes = 0;
    double* epart = nullptr;
    double* npart = nullptr;
    size_t epart_n = 0, npart_n = 0;
    cudaStream_t stream = nullptr;
    int grid_e = 1, grid_g = 1, grid_p = 1;
    struct Tick {
        std::vector<tq_request> reqs;
        std::vector<double> t_submit;
        std::vector<int> slot;        // index into E (>= 0) or ~index into P
        unsigned char* h = nullptr;   // pinned: E[MAX_TICK] | P[MAX_TICK] | Idx
        unsigned char* d = nullptr;
        cudaEvent_t done = nullptr;
        bool busy = false;
        int ne = 0, np = 0;
    } tick[2];
    int next = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::pair<tq_request, double>> queue;
    std::deque<tq_completion> done;
    std::thread worker;
    std::atomic<bool> running{false};
    std::atomic<bool> failed{false};
    long long ticks = 0, completed = 0, batched = 0;
    std::string error;
};

namespace {

constexpr size_t TICK_BYTES = 2 * MAX_TICK * sizeof(ReqDev) + sizeof(Idx);

ReqDev* tick_E(unsigned char* base) { return reinterpret_cast<ReqDev*>(base); }
ReqDev* tick_P(unsigned char* base) { return reinterpret_cast<ReqDev*>(base) + MAX_TICK; }
Idx* tick_I(unsigned char* base) { return reinterpret_cast<Idx*>(base + 2 * MAX_TICK * sizeof(ReqDev)); }

size_t work_bytes(const tq_server* s, int kind, long long D, const tq_pool* p) {
    if (kind == TQ_REQ_EVOLVE) return 0;
    size_t b = align256((size_t)D * (s->prec == TQ_C128 ? sizeof(double2) : sizeof(float2)));
    if (kind == TQ_REQ_GRADIENTS)
        b += align256((size_t)p->M * sizeof(double)) + align256((size_t)p->M * sizeof(unsigned)) +
             align256((size_t)p->view.n_gitems * sizeof(double));
    return b;
}

// Form a tick from the queue head (caller holds the lock).  Returns the
// number of admitted requests.
int form_tick(tq_server* s, tq_server::Tick& tk) {
    tk.reqs.clear();
    tk.t_submit.clear();
    tk.slot.clear();
    std::vector<char> taken(s->sessions.size(), 0);
    size_t arena_used = 0;
    long long e_items = 0, p_slots = 0;
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)tk.reqs.size() < s->max_batch;) {
        const tq_request& r = it->first;
        if (taken[r.session]) {   // later requests of a taken session keep their order
            ++it;
            continue;
        }
        taken[r.session] = 1;
        const auto& ss = s->sessions[r.session];
        const tq_pool* p = s->pools[ss.ham];
        const size_t wb = work_bytes(s, r.kind, ss.D, p);
        const long long ei = r.kind == TQ_REQ_EVOLVE ? 0 : (ss.D + ENERGY_ROWS - 1) / ENERGY_ROWS;
        const long long pt = r.kind == TQ_REQ_EVOLVE ? ((ss.D >> 2) + 2 * PAIR_BS - 1) / (2 * PAIR_BS) * (PAIR_BS / 32) : 0;
        if (arena_used + wb > s->arena_bytes || 2 * (e_items + ei) > (long long)s->epart_n ||
            p_slots + pt > (long long)s->npart_n)
            break;   // memory admission: wait for the next tick
        arena_used += wb;
        e_items += ei;
        p_slots += pt;
        tk.reqs.push_back(r);
        tk.t_submit.push_back(it->second);
        it = s->queue.erase(it);
    }
    return (int)tk.reqs.size();
}

template <typename T, typename VT>
void launch_tick(tq_server* s, tq_server::Tick& tk) {
    ReqDev* E = tick_E(tk.h);
    ReqDev* P = tick_P(tk.h);
    Idx* ix = tick_I(tk.h);
    int ne = 0, ng = 0, np = 0;
    ix->e_off[0] = ix->g_off[0] = ix->p_off[0] = ix->p_base[0] = 0;
    size_t arena_off = 0;
    tk.slot.assign(tk.reqs.size(), 0);
    for (size_t i = 0; i < tk.reqs.size(); ++i) {
        const tq_request& r = tk.reqs[i];
        const auto& ss = s->sessions[r.session];
        const tq_ham* hm = s->hams[ss.ham];
        const tq_pool* pl = s->pools[ss.ham];
        ReqDev d{};
        d.kind = r.kind;
        d.D = ss.D;
        d.M = pl->M;
        d.psi = ss.psi;
        d.diag = hm->view.diag;
        d.rowptr = hm->view.rowptr;
        d.col = hm->view.col;
        d.val = hm->view.val;
        d.pool = pl->view;
        d.k = r.op;
        d.theta = r.theta;
        if (r.kind == TQ_REQ_EVOLVE) {
            const int tiles = (int)(((d.D >> 2) + 2 * PAIR_BS - 1) / (2 * PAIR_BS));
            ix->p_off[np + 1] = ix->p_off[np] + tiles;
            ix->p_base[np + 1] = ix->p_base[np] + tiles * (PAIR_BS / 32);
            P[np] = d;
            tk.slot[i] = ~np;
            ++np;
            continue;
        }
        unsigned char* base = s->arena + arena_off;
        size_t off = align256((size_t)d.D * (s->prec == TQ_C128 ? 16 : 8));
        if (s->prec == TQ_C128) d.w64 = reinterpret_cast<double2*>(base);
        else d.w32 = reinterpret_cast<float2*>(base);
        if (r.kind == TQ_REQ_GRADIENTS) {
            d.g = reinterpret_cast<double*>(base + off);
            off += align256((size_t)d.M * sizeof(double));
            d.gtick = reinterpret_cast<unsigned*>(base + off);
            off += align256((size_t)d.M * sizeof(unsigned));
            d.gpart = reinterpret_cast<double*>(base + off);
            off += align256((size_t)pl->view.n_gitems * sizeof(double));
            ix->g_pos[ng] = ne;
            ix->g_off[ng + 1] = ix->g_off[ng] + pl->view.n_gitems;
            ++ng;
        }
        arena_off += off;
        ix->e_off[ne + 1] = ix->e_off[ne] + (int)((d.D + ENERGY_ROWS - 1) / ENERGY_ROWS);
        E[ne] = d;
        tk.slot[i] = ne;
        ++ne;
    }
    tk.ne = ne;
    tk.np = np;
    cudaStream_t st = s->stream;
    tq_ctx* c = s->ctx;
    ReqDev* dE = tick_E(tk.d);
    ReqDev* dP = tick_P(tk.d);
    Idx* dI = tick_I(tk.d);
    TQ_CUDA(cudaMemcpyAsync(dI, ix, sizeof(Idx), cudaMemcpyHostToDevice, st));
    if (ne) TQ_CUDA(cudaMemcpyAsync(dE, E, (size_t)ne * sizeof(ReqDev), cudaMemcpyHostToDevice, st));
    if (np) TQ_CUDA(cudaMemcpyAsync(dP, P, (size_t)np * sizeof(ReqDev), cudaMemcpyHostToDevice, st));
    for (int j = 0; j < ng; ++j)
        TQ_CUDA(cudaMemsetAsync(E[ix->g_pos[j]].gtick, 0, (size_t)E[ix->g_pos[j]].M * sizeof(unsigned), st));
    if (ne) {
        const int items = ix->e_off[ne];
        launch(c, "serve_energy", st, [&] {
            ks_energy<T, VT, 8><<<std::min(items, s->grid_e), SV_BS, 0, st>>>(dE, dI, ne, s->epart);
            return 1;
        });
    }
    if (ng) {
        const int items = ix->g_off[ng];
        launch(c, "serve_gradients", st, [&] {
            ks_grad<T><<<std::min(items, s->grid_g), GRAD_TPB, 0, st>>>(dE, dI, ng);
            return 1;
        });
        launch(c, "serve_select", st, [&] {
            ks_select<<<(ng * 32 + 255) / 256, 256, 0, st>>>(dE, dI, ng, s->prec);
            return 1;
        });
    }
    if (np) {
        const int items = ix->p_off[np];
        launch(c, "serve_taylor5_pair", st, [&] {
            ks_pair<T><<<std::min(items, s->grid_p), PAIR_BS, 0, st>>>(dP, dI, np, s->npart);
            return 1;
        });
        launch(c, "serve_norm", st, [&] {
            ks_norm<sizeof(T) == 4><<<(np * 32 + 255) / 256, 256, 0, st>>>(dP, dI, np, s->npart);
            return 1;
        });
        launch(c, "serve_scale", st, [&] {
            ks_scale<T><<<dim3(16, std::min(np, 1024)), 256, 0, st>>>(dP, np);
            return 1;
        });
    }
    if (ne) TQ_CUDA(cudaMemcpyAsync(E, dE, (size_t)ne * sizeof(ReqDev), cudaMemcpyDeviceToHost, st));
    if (np) TQ_CUDA(cudaMemcpyAsync(P, dP, (size_t)np * sizeof(ReqDev), cudaMemcpyDeviceToHost, st));
    TQ_CUDA(cudaEventRecord(tk.done, st));
    tk.busy = true;
}

void post_tick(tq_server* s, tq_server::Tick& tk) {
    const double t = now_s();
    ReqDev* E = tick_E(tk.h);
    ReqDev* P = tick_P(tk.h);
    std::lock_guard<std::mutex> lock(s->mu);
    for (size_t i = 0; i < tk.reqs.size(); ++i) {
        const tq_request& r = tk.reqs[i];
        const ReqDev& d = tk.slot[i] >= 0 ? E[tk.slot[i]] : P[~tk.slot[i]];
        tq_completion c{};
        c.tag = r.tag;
        c.kind = r.kind;
        c.session = r.session;
        c.status = TQ_OK;
        c.energy = r.kind == TQ_REQ_EVOLVE ? 0.0 : d.energy;
        c.max_grad = r.kind == TQ_REQ_GRADIENTS ? d.max_grad : 0.0;
        c.argmax = r.kind == TQ_REQ_GRADIENTS ? d.argmax : -1;
        c.norm2 = r.kind == TQ_REQ_EVOLVE ? d.norm2 : d.e_den;
        if (!std::isfinite(c.energy) || !std::isfinite(c.norm2)) c.status = TQ_ENUMERIC;
        c.t_submit = tk.t_submit[i];
        c.t_done = t;
        s->done.push_back(c);
    }
    s->completed += (long long)tk.reqs.size();
    s->batched += (long long)tk.reqs.size();
    s->ticks += 1;
    tk.busy = false;
    s->cv.notify_all();
}

void server_loop(tq_server* s) {
    try {
        TQ_CUDA(cudaSetDevice(s->ctx->device));
        while (s->running.load()) {
            // post finished ticks (in order)
            bool progressed = false;
            for (int k = 0; k < 2; ++k) {
                auto& tk = s->tick[(s->next + k) % 2];
                if (tk.busy && cudaEventQuery(tk.done) == cudaSuccess) {
                    post_tick(s, tk);
                    progressed = true;
                }
            }
            auto& tk = s->tick[s->next];
            if (!tk.busy) {
                int n = 0;
                {
                    std::unique_lock<std::mutex> lock(s->mu);
                    if (s->queue.empty() && !s->tick[(s->next + 1) % 2].busy)
                        s->cv.wait_for(lock, std::chrono::microseconds(200));
                    n = form_tick(s, tk);
                }
                if (n > 0) {
                    if (s->prec == TQ_C128) launch_tick<double, double>(s, tk);
                    else launch_tick<float, float>(s, tk);
                    s->next = (s->next + 1) % 2;
                    progressed = true;
                }
            }
            if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->error = e.what();
        s->failed = true;
        s->running = false;
        s->cv.notify_all();
    }
}

template <typename T, typename VT>
void compute_grids(tq_server* s) {
    const int sms = s->ctx->sm_count;
    s->grid_e = resident(ks_energy<T, VT, 8>, SV_BS, sms);
    s->grid_g = resident(ks_grad<T>, GRAD_TPB, sms);
    s->grid_p = resident(ks_pair<T>, PAIR_BS, sms);
}

}  // namespace

extern "C" int tq_server_create(tq_ctx* c, int prec, size_t hbm_budget, int max_batch, tq_server** out) {
    API_BEGIN
    TQ_REQUIRE(c && out, "null argument");
    TQ_REQUIRE(prec == TQ_C128 || prec == TQ_C64, "prec must be TQ_C128 or TQ_C64");
    TQ_REQUIRE(max_batch >= 1 && max_batch <= MAX_TICK, "max_batch must be in [1, 2048]");
    TQ_REQUIRE(hbm_budget >= (64u << 20), "hbm_budget must be at least 64 MiB");
    *out = nullptr;
    TQ_CUDA(cudaSetDevice(c->device));
    auto* s = new tq_server();
    try {
        s->ctx = c;
        s->device = c->device;
        s->prec = prec;
        s->budget = hbm_budget;
        s->max_batch = max_batch;
        for (auto& tk : s->tick) {
            TQ_CUDA(cudaMallocHost(&tk.h, TICK_BYTES));
            std::memset(tk.h, 0, TICK_BYTES);
            tk.d = static_cast<unsigned char*>(dev_alloc(TICK_BYTES));
            s->allocs.push_back(tk.d);
            TQ_CUDA(cudaEventCreateWithFlags(&tk.done, cudaEventDisableTiming));
        }
        TQ_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->epart_n = 2u << 20;
        s->npart_n = 4u << 20;
        s->epart = static_cast<double*>(dev_alloc(s->epart_n * sizeof(double)));
        s->npart = static_cast<double*>(dev_alloc(s->npart_n * sizeof(double)));
        s->allocs.push_back(s->epart);
        s->allocs.push_back(s->npart);
        if (prec == TQ_C128) compute_grids<double, double>(s);
        else compute_grids<float, float>(s);
    } catch (...) {
        tq_server_free(s);
        throw;
    }
    *out = s;
    API_END
}

extern "C" int tq_server_add_hamiltonian(tq_server* s, const tq_ham* h, const tq_pool* p, int* ham_id) {
    API_BEGIN
    TQ_REQUIRE(s && h && p && ham_id, "null argument");
    TQ_REQUIRE(!h->sector && !p->sector, "the request loop works in the full space");
    TQ_REQUIRE(!s->running.load(), "add Hamiltonians before tq_server_start");
    TQ_REQUIRE(h->prec == s->prec, "Hamiltonian precision differs from the server's");
    TQ_REQUIRE(h->nq == p->nq, "Hamiltonian and pool qubit counts differ");
    s->hams.push_back(h);
    s->pools.push_back(p);
    *ham_id = (int)s->hams.size() - 1;
    API_END
}

extern "C" int tq_server_add_session(tq_server* s, int ham_id, int n_electrons, int mapping, int* session_id) {
    API_BEGIN
    TQ_REQUIRE(s && session_id, "null argument");
    TQ_REQUIRE(!s->running.load(), "add sessions before tq_server_start");
    TQ_REQUIRE(ham_id >= 0 && ham_id < (int)s->hams.size(), "unknown Hamiltonian id");
    const tq_ham* h = s->hams[ham_id];
    const size_t bytes = align256((size_t)h->D * (s->prec == TQ_C128 ? 16 : 8));
    if (s->states_bytes + bytes > s->budget / 2)
        throw Error(TQ_EBUSY, "session states would exceed half of the server's HBM budget");
    TQ_CUDA(cudaSetDevice(s->ctx->device));
    void* psi = dev_alloc(bytes);
    s->allocs.push_back(psi);
    s->states_bytes += bytes;
    const long long idx = (long long)hf_index(h->nq, n_electrons, mapping);
    check_launch(s->ctx, launch_set_basis(psi, s->prec, h->D, idx, 0));
    TQ_CUDA(cudaDeviceSynchronize());
    s->sessions.push_back({ham_id, psi, h->D, h->nq});
    *session_id = (int)s->sessions.size() - 1;
    API_END
}

extern "C" int tq_server_start(tq_server* s) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "server is null");
    TQ_REQUIRE(!s->running.load(), "server already running");
    TQ_REQUIRE(!s->sessions.empty(), "no sessions");
    // the rest of the budget is the per-request working arena
    s->arena_bytes = s->budget - s->states_bytes;
    TQ_CUDA(cudaSetDevice(s->ctx->device));
    s->arena = static_cast<unsigned char*>(dev_alloc(s->arena_bytes));
    s->allocs.push_back(s->arena);
    // the largest single request must fit on its own
    for (size_t i = 0; i < s->sessions.size(); ++i) {
        const auto& ss = s->sessions[i];
        if (work_bytes(s, TQ_REQ_GRADIENTS, ss.D, s->pools[ss.ham]) > s->arena_bytes)
            throw Error(TQ_EBUSY, "a gradient request of session " + std::to_string(i) + " exceeds the arena");
    }
    s->running = true;
    s->worker = std::thread(server_loop, s);
    API_END
}

extern "C" int tq_server_submit(tq_server* s, const tq_request* r) {
    API_BEGIN
    TQ_REQUIRE(s && r, "null argument");
    TQ_REQUIRE(r->kind >= TQ_REQ_EVOLVE && r->kind <= TQ_REQ_GRADIENTS, "unknown request kind");
    TQ_REQUIRE(r->session >= 0 && r->session < (int)s->sessions.size(), "unknown session");
    if (r->kind == TQ_REQ_EVOLVE) {
        const auto& ss = s->sessions[r->session];
        TQ_REQUIRE(r->op >= 0 && r->op < s->pools[ss.ham]->M, "pool index out of range");
        TQ_REQUIRE(std::isfinite(r->theta), "theta is not finite");
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->failed) throw Error(TQ_ECUDA, "server stopped: " + s->error);
    if (s->queue.size() >= s->max_queue) throw Error(TQ_EBUSY, "request queue is full");
    s->queue.emplace_back(*r, now_s());
    s->cv.notify_all();
    API_END
}

extern "C" int tq_server_poll(tq_server* s, tq_completion* out, int max, int* n_out, int timeout_us) {
    API_BEGIN
    TQ_REQUIRE(s && out && n_out && max >= 1, "bad argument");
    *n_out = 0;
    std::unique_lock<std::mutex> lock(s->mu);
    if (s->done.empty() && timeout_us > 0)
        s->cv.wait_for(lock, std::chrono::microseconds(timeout_us), [&] { return !s->done.empty() || s->failed; });
    if (s->failed && s->done.empty()) throw Error(TQ_ECUDA, "server stopped: " + s->error);
    int n = 0;
    while (n < max && !s->done.empty()) {
        out[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = n;
    if (n == 0) throw Error(TQ_ETIMEOUT, "no completion within the timeout");
    API_END
}

extern "C" int tq_server_stats(const tq_server* s, long long* ticks, long long* completed, long long* queued) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "server is null");
    auto* m = const_cast<tq_server*>(s);
    std::lock_guard<std::mutex> lock(m->mu);
    if (ticks) *ticks = s->ticks;
    if (completed) *completed = s->completed;
    if (queued) *queued = (long long)s->queue.size();
    API_END
}

extern "C" int tq_server_session_state(const tq_server* s, int session, void** dev_ptr, int* n_qubits) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "server is null");
    TQ_REQUIRE(session >= 0 && session < (int)s->sessions.size(), "unknown session");
    if (dev_ptr) *dev_ptr = s->sessions[session].psi;
    if (n_qubits) *n_qubits = s->sessions[session].nq;
    API_END
}

extern "C" int tq_server_stop(tq_server* s) {
    API_BEGIN
    TQ_REQUIRE(s != nullptr, "server is null");
    if (s->running.exchange(false)) {
        s->cv.notify_all();
        if (s->worker.joinable()) s->worker.join();
    } else if (s->worker.joinable()) {
        s->worker.join();
    }
    TQ_CUDA(cudaSetDevice(s->ctx->device));
    TQ_CUDA(cudaStreamSynchronize(s->stream));
    for (auto& tk : s->tick)
        if (tk.busy) post_tick(s, tk);
    API_END
}

extern "C" int tq_server_free(tq_server* s) {
    if (!s) return TQ_OK;
    tq_server_stop(s);
    cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    for (auto& tk : s->tick) {
        if (tk.h) cudaFreeHost(tk.h);
        if (tk.done) cudaEventDestroy(tk.done);
    }
    if (s->stream) cudaStreamDestroy(s->stream);
    for (void* p : s->allocs) cudaFree(p);
    delete s;
    (void)cudaGetLastError();   // a failure while freeing is not reported to later calls
    return TQ_OK;
}
