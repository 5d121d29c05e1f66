// Host-side helpers shared by the C ABI translation units: status
// exceptions, argument checks, device allocation and traced launches.
#pragma once

#include <new>
#include <stdexcept>
#include <string>

#include "common.h"

namespace tq {

#define TQ_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            throw Error(e_ == cudaErrorMemoryAllocation ? TQ_ENOMEM : TQ_ECUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

#define TQ_REQUIRE(cond, msg)                              \
    do {                                                   \
        if (!(cond)) throw Error(TQ_EINVAL, (msg));        \
    } while (0)


// Brackets the launches made in its scope with events when tracing is on.
struct Traced {
    tq_ctx* c;
    cudaStream_t s;
    tq_trace_rec rec{};
    Traced(tq_ctx* ctx, const char* name, cudaStream_t st) : c(ctx), s(st) {
        if (!c->tracing) return;
        rec.name = name;
        rec.start = take();
        rec.stop = take();
        cudaEventRecord(rec.start, s);
    }
    ~Traced() {
        if (!c->tracing || !rec.start) return;
        cudaEventRecord(rec.stop, s);
        c->trace.push_back(rec);
    }
    cudaEvent_t take() {
        cudaEvent_t e = nullptr;
        if (!c->event_pool.empty()) {
            e = c->event_pool.back();
            c->event_pool.pop_back();
        } else {
            cudaEventCreate(&e);
        }
        return e;
    }
};

inline void check_launch(tq_ctx* c, int n) {
    c->launches += n;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error(TQ_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// Launch through `f` (which returns its launch count), traced under `name`.
// A launch error left pending by an unrelated earlier call (ours or another
// library's) is cleared first, so the check below reports this launch only.
template <typename F>
void launch(tq_ctx* c, const char* name, cudaStream_t s, F&& f) {
    (void)cudaGetLastError();
    Traced t(c, name, s);
    const int n = f();
    if (n < 0) throw Error(TQ_EINVAL, std::string(name) + ": problem too large for one launch");
    check_launch(c, n);
}

inline void* dev_alloc(size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Error(TQ_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    return p;
}


}  // namespace tq

#define API_BEGIN try {
#define API_END                                            \
    }                                                      \
    catch (const tq::Error& e) {                           \
        tq::set_last_error(e.what());                      \
        return e.code;                                     \
    }                                                      \
    catch (const std::bad_alloc&) {                        \
        tq::set_last_error("host allocation failed");      \
        return TQ_ENOMEM;                                  \
    }                                                      \
    catch (const std::exception& e) {                      \
        tq::set_last_error(e.what());                      \
        return TQ_ECUDA;                                   \
    }                                                      \
    return TQ_OK;
