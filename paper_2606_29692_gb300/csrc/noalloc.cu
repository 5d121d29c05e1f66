// Energy entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need
// an energy: a serving loop that pre-reserved all of its memory and must not
// stall on cudaMalloc/cudaFree (cudaFree synchronises the whole device), a
// host framework whose caching allocator already owns the device heap, or a
// plugin whose host forbids allocation after start-up.  For them this file
// keeps the energy reduction's scratch -- the per-CTA partial sums, the
// last-CTA ticket and the result record -- in one fixed array in device
// global memory, reserved when the library is loaded and held by every GPU
// that loads it until the process exits.  The caller passes the Hamiltonian's
// CSR and diagonal, the state and a device slot for the result; nothing is
// allocated or freed by the call.
#include "dev.cuh"

#include <mutex>

namespace {

// 64 KiB: the result record, the ticket, and up to 4064 CTA partial pairs.
constexpr size_t kScratchBytes = 64 * 1024;
constexpr size_t kStepOffset = 0;
constexpr size_t kTicketOffset = 256;
constexpr size_t kPartialsOffset = 512;
constexpr size_t kMaxPartialPairs = (kScratchBytes - kPartialsOffset) / (2 * sizeof(double));
static_assert(kMaxPartialPairs == 4064, "the documented limit of CTA partials");
static_assert(kStepOffset + sizeof(tq::DevStep) <= kTicketOffset, "the result record overlaps the ticket");
static_assert(kTicketOffset + sizeof(unsigned) <= kPartialsOffset, "the ticket overlaps the partials");

static __device__ __align__(256) unsigned char tq_energy_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool done = false;
    int sms = 0;
    unsigned char* scratch = nullptr;   // device address of tq_energy_scratch
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: resolve the array's device
// address (in host code its name is only a host-side stand-in) and the SM
// count used to size the grid.
int setup_device(int dev, DeviceSetup** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        tq::set_last_error("device index beyond the supported range");
        return TQ_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& d = g_setup[dev];
    if (!d.done) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, tq_energy_scratch);
        if (e != cudaSuccess) {
            tq::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return TQ_ECUDA;
        }
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) {
            tq::set_last_error(std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
            return TQ_ECUDA;
        }
        d.scratch = static_cast<unsigned char*>(p);
        d.sms = sms;
        d.done = true;
    }
    *out = &d;
    return TQ_OK;
}

}  // namespace

extern "C" int tq_energy_noalloc(int n_qubits, int prec, const int* rowptr, const int* col,
                                 const void* val, const double* diag, const void* psi,
                                 double* energy_out, void* stream) {
    using namespace tq;
    if (!rowptr || !col || !val || !diag || !psi || !energy_out) {
        tq::set_last_error("null argument");
        return TQ_EINVAL;
    }
    if (prec != TQ_C128 && prec != TQ_C64) {
        tq::set_last_error("prec must be TQ_C128 or TQ_C64");
        return TQ_EINVAL;
    }
    if (n_qubits < 1 || n_qubits > TQ_MAX_STATE_QUBITS) {
        tq::set_last_error("n_qubits out of range [1, 26]");
        return TQ_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        tq::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return TQ_ECUDA;
    }
    DeviceSetup* d = nullptr;
    int rc = setup_device(dev, &d);
    if (rc != TQ_OK) return rc;
    HamView h{};
    h.nq = n_qubits;
    h.prec = prec;
    h.D = 1ll << n_qubits;
    h.rowptr = rowptr;
    h.col = col;
    h.val = val;
    h.diag = diag;
    if ((size_t)energy_csr_grid(h, prec, d->sms) > kMaxPartialPairs) {
        tq::set_last_error("the reduction needs more CTA partials than the fixed scratch holds "
                          "(" + std::to_string(kMaxPartialPairs) + ")");
        return TQ_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevStep* step = reinterpret_cast<DevStep*>(d->scratch + kStepOffset);
    unsigned* ticket = reinterpret_cast<unsigned*>(d->scratch + kTicketOffset);
    double* partials = reinterpret_cast<double*>(d->scratch + kPartialsOffset);
    // the ticket must start at zero; an earlier call that failed part-way
    // could have left it otherwise
    e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        launch_energy_csr(h, psi, prec, nullptr, partials, ticket, step, d->sms, s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(energy_out, &step->energy, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        tq::set_last_error(std::string("tq_energy_noalloc: ") + cudaGetErrorString(e));
        return TQ_ECUDA;
    }
    return TQ_OK;
}
