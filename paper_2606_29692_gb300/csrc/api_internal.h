// Helpers shared by the translation units that implement the C ABI
// (api*.cu): context scratch, argument checks, the Hamiltonian layouts'
// builders, and the launch sequences several entry points share.  Not part
// of the ABI.
#pragma once

#include "common.h"
#include "host_util.h"

#include <vector>

namespace tq {
namespace api {

// Copies v to a new device array recorded in allocs.
template <typename T>
T* upload(std::vector<void*>& allocs, const std::vector<T>& v) {
    T* p = static_cast<T*>(dev_alloc(v.size() * sizeof(T)));
    allocs.push_back(p);
    if (!v.empty()) TQ_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
}

// Context scratch slots (grown on demand, kept until the context goes).
enum { S_PART = 0, S_W0, S_U1, S_U2, S_W1, S_W2, S_G, S_STAGE, S_W32, S_PHI, S_CHI, S_AG, S_HOSTB, S_REC,
       S_THETAS };
void* scratch(tq_ctx* c, int slot, size_t bytes);
// n zeroed tickets (every user leaves them zero).
unsigned* tickets(tq_ctx* c, size_t n);

size_t elem_bytes(int prec);
void check_prec(int prec);
inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
void set_device(const tq_ctx* c);

// A pool, Hamiltonian and state must describe the same space.
void check_space(const tq_pool* p, const tq_state* s);
void check_space(const tq_ham* h, const tq_state* s);
void free_all(std::vector<void*>& allocs);

// The CSR and XOR-ELL forms of a Hamiltonian's off-diagonal entries.
long long build_csr(tq_ctx* c, HamView& h, double maxc, int prec, std::vector<void*>& allocs,
                    long long* n_amb, int* max_row);
long long build_xell(tq_ctx* c, HamView& h, double maxc, int prec, std::vector<void*>& allocs);

// Amplitudes of one state of the pool's space.
long long state_len(const tq_pool* p);
// Norm partials per state of the Taylor-5 launch for this pool.
int update_tiles(const tq_pool* p, int prec, int upt);
// Taylor-5 on n states (ops and angles from k/theta, or k_fixed and
// theta_fixed, or the step record when gate is set).  Returns true when the
// launch also wrote the float64 norms; otherwise they are in part.
bool launch_update(tq_ctx* c, const tq_pool* p, long long n, int prec, int upt, void* psi, const int* k,
                   const double* theta, int k_fixed, double theta_fixed, const DevStep* gate, double* part,
                   double* norm2, double* step_norm2, cudaStream_t s);

// Partials needed by energy + gradients (+ line search) on this problem.
size_t partials_needed(long long D, int n_gitems, int nq, int sms);
// Allocates (before any launch of a call) the scratch energy and gradients use.
double* prepare(tq_ctx* c, long long D, const tq_pool* p, int nq);
void run_energy(tq_ctx* c, const tq_ham* h, const tq_state* psi, double* part, cudaStream_t s);
void run_gradients(tq_ctx* c, const tq_ham* h, const tq_pool* p, const tq_state* psi, double* g, double* part,
                   cudaStream_t s);
// Clears and reports TQ_ETIMEOUT left by a kernel's bounded wait.
void raise_status(tq_ctx* c, int status, cudaStream_t s);

}  // namespace api
}  // namespace tq
