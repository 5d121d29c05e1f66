// Internal declarations shared by the host code and the CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "tq.h"

namespace tq {

struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

// ---------------------------------------------------------------- host algebra

struct PauliTerm {
    uint64_t x, z;  // X^x Z^z, Z acting first
    double c;       // real coefficient of that product
};

struct Excitation {
    int idx[4];  // (i, a, -1, -1) or (i, j, a, b)
    int order;   // 1 single, 2 double
};

// Sign function of a pool generator in factored form:
//   A[r][r ^ x] = c0 * (-1)^{popcount(col & z0)} * prod_{i<m} [parity(col & d_i) == t_i]
// with col = r ^ x.  ok == 0 means "use the generic term sum".
struct SignForm {
    int ok;
    int m;
    double c0;
    uint64_t z0;
    uint64_t d[3];
    int t;
};

// Support of a generator, {r : A[r][r^x] != 0}, as an affine subspace in
// reduced form: m pivot bits p[0] < p[1] < p[2]; each mask e[i] contains
// pivot p[i] and no other pivot; row r is in the support iff
// parity(r & e[i]) == bit i of target for every i.  Support row u
// (0 <= u < 2^(N-m)) is u with zeros inserted at the pivots, each pivot bit
// then set to target_i xor parity(r & e[i]).  The support is closed under
// r -> r ^ x; h is the highest set bit of x that is not a pivot (one always
// exists) and hp its position among the free bits: pair u (0 <= u <
// 2^(N-m-1)) is support row insert_zero(u, hp), the member of its pair
// {r, r ^ x} whose bit h is 0.
struct SupportForm {
    int m;
    int p[3];
    uint64_t e[3];
    int target;
    int h, hp;
};
SupportForm support_form(const SignForm& f, uint64_t x);

void check_mapping(int mapping);
// Registers (or finds) the relabelled encoding base + order; returns its id.
int register_relabelled(int base, int N, const int* order);
int register_linear(int base, int N, const uint64_t* rows);
std::vector<uint64_t> pool_sector_basis(int n, int ne, int base, int low_bits);
// Qubit order whose lowest low_bits index bits are the qubits, picked one at
// a time, that leave the fewest touched segments over the pool's supports.
std::vector<int> pool_sector_order(int n, int ne, int base, int low_bits);
// Sets the thread-local reason returned by tq_last_error().
void set_last_error(const std::string& m);
std::vector<PauliTerm> pauli_hamiltonian(int n, const double* h1, const double* g2,
                                         double e_const, int mapping);
std::vector<Excitation> excitations(int n, int ne);
std::vector<PauliTerm> pauli_generator(const Excitation& ex, int N, int mapping);
uint64_t hf_index(int N, int ne, int mapping);
SignForm factor_generator(const std::vector<PauliTerm>& t);
// rows of B^-1 (occupation bit j = parity(qubit index & rows[j])) and the
// qubit index of an occupation index under a mapping
std::vector<uint32_t> decode_rows(int N, int mapping);
uint64_t encode_occupation(int N, int mapping, uint64_t occ);

// Sector-restricted basis: occupation states with n_alpha electrons in the
// even spin orbitals and n_beta in the odd ones, ranked colexicographically
// (rank = rank_alpha * C(n, n_beta) + rank_beta).  A variant of the
// paper's 2^N formulation, not part of it.
struct SectorSpec {
    int n, na, nb, nq, mapping;
    uint32_t dec[32];        // rows of B^-1 (JW: unused)
    int binom[16][16];       // C(i, j)
};
SectorSpec make_sector_spec(int n, int na, int nb, int mapping);

// Commuting families (Sec. III-F, Algorithm 1): terms holds 8 slots per
// generator, nterm[k] of them used; returns the family of each generator.
std::vector<int> pool_families(const std::vector<PauliTerm>& terms, const std::vector<int>& nterm, int mode);
long long sector_dim(int n, int na, int nb);
// qubit indices of the sector in rank order
std::vector<uint32_t> sector_basis(const SectorSpec& s);

// --------------------------------------------------------------- device views

// Pool generators, structure of arrays (one entry per op unless noted).
struct PoolView {
    int M;
    int nq;
    const uint32_t* x;      // X-mask
    const int* nterm;       // 2 or 8
    const uint32_t* z;      // [8 M] Z-masks of the terms
    const float* cf;        // [8 M] coefficients (float32 copy)
    const double* cd;       // [8 M] coefficients (float64)
    const int* fok;         // factored sign form available
    const int* fm;          // number of parity conditions
    const uint32_t* fz0;    // sign mask
    const uint32_t* fd;     // [3 M] condition masks
    const int* ft;          // target parities, bit i for condition i
    const float* fc0f;      // leading coefficient, float32
    const double* fc0d;     // leading coefficient, float64
    const int4* supp;       // [M] support form: (m | target << 8, p0 | p1 << 8 | p2 << 16, -, -)
    const uint32_t* supe;   // [3 M] support masks
    const int2* gitems;     // gradient work items (op, chunk of support rows)
    int n_gitems;
    const int* gfirst;      // [M + 1] first work item of each op
    // sector pools: A_k restricted to the sector, one entry per (op, row):
    // A_k[r][scol] = ssgn (+-1), or ssgn = 0 (A_k annihilates row r)
    long long sdim;         // sector dimension (0: full space)
    const int* scol;        // [M sdim]
    const signed char* ssgn;  // [M sdim]
};

constexpr int XELL_ROWS = 8;   // rows per XOR-ELL block

// Hamiltonian: float64 diagonal + off-diagonal CSR + the same off-diagonal
// entries in XOR-ELL form + X-mask-grouped terms.
struct HamView {
    int nq;
    int prec;
    long long D;
    long long nnz;
    const double* diag;
    const int* rowptr;
    const int* col;
    const void* val;        // double or float
    const uint32_t* sq;     // sector basis: qubit index of each row (null: full space)
    const SectorSpec* sect; // sector spec on the device (null: full space)
    long long n_blocks;     // XOR-ELL row blocks of XELL_ROWS rows, ceil(D / XELL_ROWS)
    long long n_pairs;
    const int* xptr;        // [n_blocks + 1] first pair of each block
    const uint32_t* xmask;  // [n_pairs] X-mask of the pair
    const void* xval;       // [XELL_ROWS n_pairs] values, double or float
                            // (both arrays padded to whole copy chunks)
    int xgrid;              // CTAs of the staged XOR-ELL energy launch
    const int* xsplit;      // [xgrid + 1] first row block of each CTA
    int G;                  // off-diagonal X-mask groups
    const uint32_t* gx;     // [G] group masks
    const int* goff;        // [G + 1] term offsets
    const uint32_t* tz;     // [K_off] term Z-masks
    const double* tc;       // [K_off] term coefficients
    int Kd;                 // diagonal (x = 0) terms
    const uint32_t* dz;
    const double* dc;
};

// Scalars an ADAPT iteration keeps on the device between its kernels.
struct DevStep {
    double e_num, e_den, energy;   // Rayleigh quotient pieces
    double max_grad;
    double theta;
    double norm2;                  // ||psi'||^2 after the update
    double dots[6];                // line-search matrix elements
    int selected;
    int converged;
    int status;                    // TQ_OK, or TQ_ETIMEOUT from a bounded wait
    int iter;                      // steps recorded by a graph-replayed ADAPT run
};

// ------------------------------------------------------------- kernel launchers
// Every launcher enqueues on `stream` and returns the number of launches.

// state
int launch_set_basis(void* psi, int prec, long long D, long long index, cudaStream_t s);

// CSR builder
int launch_csr_count(const HamView& h, double tol, double amb_hi, int* counts,
                     unsigned long long* n_amb, int sms, cudaStream_t s);
int launch_diag(const HamView& h, double* diag, int sms, cudaStream_t s);
int launch_scan(const int* counts, long long D, int* rowptr, long long* total,
                int* max_row, cudaStream_t s);
int launch_csr_fill(const HamView& h, double tol, int max_row, int* col, void* val,
                    int prec, int sms, cudaStream_t s);
int launch_xell_count(const HamView& h, double tol, int* counts, int sms, cudaStream_t s);
int launch_xell_fill(const HamView& h, double tol, uint32_t* xmask, void* xval, int prec, int sms,
                     cudaStream_t s);

// Taylor-5, matrix-free pair path: states back to back, op k[b] / theta[b]
// (device arrays, or the immediates when the pointers are null).  Writes
// taylor5_pair_parts(nq, upt) norm partials per state; `upt` (1, 2, 4, 8)
// is the schedule: pair units (4 amplitudes each) per thread per tile.
int taylor5_pair_parts(int nq, int upt);
bool pair_upt_valid(int upt);
int launch_taylor5_pair(const PoolView& p, int n_states, int prec, int upt, void* psi,
                        const int* k, const double* theta, int k_imm, double theta_imm,
                        double* partials, int sms, cudaStream_t s);
int launch_norm_reduce(const double* partials, int prec, int n_states, int tiles_per_state,
                       double* norm2_out, double* step_norm2, cudaStream_t s);
// The same sum added to base[i] (in/out allowed: norm2_out == base).
int launch_norm_carry(const double* partials, int prec, int n_states, int tiles_per_state, const double* base,
                      double* norm2_out, double* step_norm2, cudaStream_t s);
// Support-only batched Taylor-5 (in place; rows outside each generator's
// support are not touched); partials hold the change of |psi|^2 per tile.
// With one tile per state and norm2 set, the launch adds the change to
// norm2 itself (nothing is left for launch_norm_carry).
// Support-only update of groups of grouped_size(prec) states that share a
// generator, stored amplitude-major within the group (one 32-byte sector
// per support row of the group); k per group, theta and norm2 per state.
int grouped_size(int prec);
bool grouped_schedule_ok(int prec, int lanes_per_row, int pairs_per_thread);
int launch_taylor5_grouped(const PoolView& p, int n_groups, int prec, int lanes_per_row, int pairs_per_thread,
                           void* psi, const int* k, const double* theta, double* norm2, int sms, cudaStream_t s);
int support_tiles(int nq, int n_states, int ppt, int sms);
int support_parts(int tiles);
// sched (device, two counters at zero, left at zero; may be null): with
// one tile per state and norm2 set, the pipelined forms hand out states
// dynamically instead of by a fixed stride.
int launch_taylor5_support(const PoolView& p, int n_states, int prec, int ppt, void* psi, const int* k,
                           const double* theta, double* partials, int tps, double* norm2, int sms,
                           cudaStream_t s, int ctas_per_sm = 0, unsigned* sched = nullptr);
// The same launch with the update taken out (every support row written back
// as read), in the pipelined form with |ppt| pairs per pass: the memory-only
// floor of the support-only update.
int launch_taylor5_support_touch(const PoolView& p, int n_states, int prec, int ppt, void* psi, const int* k,
                                 const double* theta, double* partials, int tps, double* norm2, int sms,
                                 cudaStream_t s, int ctas_per_sm, unsigned* sched);
int launch_scale(void* psi, int prec, long long D, const double* norm2, cudaStream_t s);

// Taylor-5 for a general CSR operator.
int launch_taylor5_csr(int nq, int prec, const int* rowptr, const int* col, const void* val,
                       double theta, void* psi, int renorm, double* scratch_acc,
                       double* scratch_v0, double* scratch_v1, double* partials,
                       double* norm2, int sms, cudaStream_t s);

// Energy, gradients, ADAPT glue
// CTAs (one partial pair each) of the launch launch_energy_csr makes.
int energy_csr_grid(const HamView& h, int psi_prec, int sms);
int launch_energy_csr(const HamView& h, const void* psi, int psi_prec, double2* w,
                      double* partials, unsigned* ticket, DevStep* step, int sms,
                      cudaStream_t s);
int launch_energy_matrix_free(const HamView& h, const void* psi, int psi_prec,
                              double* partials, unsigned* ticket, DevStep* step,
                              int sms, cudaStream_t s);
int launch_energy_xell(const HamView& h, const void* psi, int psi_prec, double2* w, float2* w32,
                       double* partials, unsigned* ticket, DevStep* step, cudaStream_t s, int withhold_chunk = -1);
int xell_grid(long long n_blocks, int prec, int sms);
int xell_chunk_pairs();
int launch_xell_split(const int* xptr, long long n_blocks, int grid, int* split, cudaStream_t s);
int launch_energy_csr2(const HamView& h, const void* psi, int psi_prec, double2* w,
                       float2* w32, double* partials, unsigned* ticket, DevStep* step,
                       int sms, cudaStream_t s, int lanes_per_row);
// gradients read w in float32 (w32) for complex64 states, float64 (w) otherwise
int launch_pool_gradients(const PoolView& p, const double2* w, const float2* w32,
                          const void* psi, int prec, const DevStep* step, double* partials,
                          unsigned* tickets, double* g, int sms, cudaStream_t s);
int launch_select(const double* g, int M, double eps, int prec, DevStep* step,
                  cudaStream_t s);
// Line search: z holds per row the record {psi, A psi, A^2 psi, 0} in the
// state's precision (4 float2 or 4 double2).
int launch_apply_twice(const PoolView& p, const DevStep* step, const void* psi, int prec, void* z, cudaStream_t s);
// The line search's matrix elements from the rows of the selected
// generator's support only (full-space pools; the state itself, no
// records): dots[1..5] divided by <psi|psi>, dots[0] the step's energy.
// Needs line_support_partials(sms) partial slots.
int launch_line_support(const HamView& h, const PoolView& p, const void* psi, DevStep* step, double* partials,
                        unsigned* ticket, int sms, cudaStream_t s);
int line_support_partials(int sms);
int launch_line_dots(const void* z, const double2* w0, const double2* w1, const double2* w2, int prec, long long D,
                     double* partials, unsigned* ticket, DevStep* step, cudaStream_t s);
// sc: sin and cos of the 4096 sample angles (launch_line_table fills it);
// rank: the samples' positions in the order (|theta_m|, m) (host table from
// line_rank_table, copied to the device); se: 4096 + 16 int64 of scratch;
// ticket: zero between calls.
int launch_line_table(double2* sc, cudaStream_t s);
void line_rank_table(int* rank);   // host: rank[4096]
// theta_list (device, optional): the angle of step step->iter (overrides
// theta_given).
int launch_line_search(DevStep* step, double theta_given, const double* theta_list, const double2* sc,
                       const int* rank, long long* se, unsigned* ticket, cudaStream_t s);
// Appends the step's result to rec (6 doubles per step: energy, max|g|,
// theta, selected, converged, bad norm) at step->iter, then advances it.
int launch_step_record(DevStep* step, double* rec, int n, cudaStream_t s);

// gated variants (skip when step->converged) and layout helpers
// Single-state update with the norm (and, if renorm, the rescale) in the
// same launch: one thread-block cluster holds the state in registers.
// k/theta from the arguments, or from the step record when gate is set.
// ready: some cluster shape launches for 2^nq amplitudes in this precision.
// unit_pool: every generator's entries are +-1, so complex128 takes the
// closed-form kernel (norm from the input, update and rescale in one pass).
bool taylor5_single_ready(int nq, int prec);
int launch_taylor5_single(const PoolView& p, int prec, bool unit_pool, int k, double theta, const DevStep* gate,
                          void* psi, int renorm, double* norm2, cudaStream_t s);
int launch_taylor5_pair_gated(const PoolView& p, int prec, int upt, void* psi, const DevStep* step,
                              double* partials, int sms, cudaStream_t s);
int launch_scale_gated(void* psi, int prec, long long D, const double* norm2,
                       const DevStep* gate, cudaStream_t s);
// The line search's three products in one pass over H: y_i = H x_i, x_i
// the three vectors of the records z, y float64.
int launch_line_spmv_gated(const HamView& h, const void* z, double2* y0, double2* y1, double2* y2,
                           const DevStep* gate, int sms, cudaStream_t s);
int energy_grid(long long D, int sms);

// sector-restricted basis
// ADAPT-VQE adjoint sweep: grad_out = 2 Re<chi | A_k T4(theta A_k) phi> / e_den,
// with A T4(theta A) = c4 A - s4 P on A's support (A^2 = -P there),
// c4 = 1 - theta^2/2 + theta^4/24, s4 = theta - theta^3/6; and chi = w - E psi
int launch_ansatz_dot(const PoolView& p, int k, double c4, double s4, const void* chi, const void* phi, int prec,
                      long long D, double* partials, unsigned* ticket, const DevStep* step, double* grad_out,
                      int sms, cudaStream_t s);
int launch_residual(const double2* w, const void* psi, void* chi, int prec, long long D, const DevStep* step,
                    cudaStream_t s);
int sector_tiles(long long dim, int prec);
// true when the sector update finishes the norms itself (no reduction launch)
bool sector_in_smem(long long dim, int prec);
int launch_sector_pool(const PoolView& p, const uint32_t* sq, const SectorSpec* sect, long long dim, int* scol,
                       signed char* ssgn, unsigned long long* bad, int sms, cudaStream_t s);
int launch_taylor5_sector(const PoolView& p, long long n_states, int prec, void* psi, const int* k,
                          const double* theta, int k_fixed, double theta_fixed, const DevStep* gate,
                          double* partials, double* norm2, double* step_norm2, cudaStream_t s);
int launch_sector_gradients(const PoolView& p, const double2* w, const void* psi, int prec, const DevStep* step,
                            double* g, cudaStream_t s);
int launch_apply_twice_sector(const PoolView& p, const DevStep* step, const void* psi, int prec, void* z,
                              cudaStream_t s);

}  // namespace tq

// ------------------------------------------------------------------- handles

// Slots of the context's ticket array (zero between calls): 0 energy, 1
// matrix-free energy, 2 line dots, 3 line search, 4 ansatz gradient, 8-9
// the support update's dynamic state counters, 16.. gradients.
constexpr int TICKET_SUPPORT_SCHED = 8;

struct tq_trace_rec {
    const char* name;
    cudaEvent_t start, stop;
};

struct tq_ctx {
    int device = 0;
    int sm_count = 0;
    long long launches = 0;
    int tracing = 0;
    int pair_upt[2] = {2, 4};              // schedule per precision (C128, C64)
    int supp_ppt[2] = {4, -1};             // support-only update: pairs per thread per pass, < 0 pipelined (C128, C64)
    int supp_ctas[2] = {0, 0};             // its resident CTAs per SM (0: as many as fit)
    int grouped_lanes[2] = {1, 1};         // grouped-layout update: lanes per row (C128, C64)
    int grouped_ppt[2] = {1, 1};           // and pairs per lane
    int l2_fetch_default = 0;              // the CUDA context's L2 fetch granularity at creation (bytes)
    int spmv_lanes = 0;                    // energy SpMV: CSR lanes per row, or 0 for XOR-ELL (default)
    int test_flags = 0;                    // TQ_TEST_* (tests of the failure paths only)
    std::vector<tq_trace_rec> trace;      // recorded, not yet reported
    std::vector<cudaEvent_t> event_pool;  // reusable events
    // device scratch, grown on demand
    static constexpr int kScratch = 16;
    void* scratch[kScratch] = {nullptr};
    size_t scratch_bytes[kScratch] = {0};
    tq::DevStep* step = nullptr;      // device
    unsigned* tickets = nullptr;      // device, zero between calls
    double2* line_sc = nullptr;       // device, sin/cos of the line search's sample angles (filled once)
    long long* line_se = nullptr;     // device, the samples' energy keys and per-block minima (4096 + 16)
    int* line_rank = nullptr;         // device, the samples' tie-rule ranks (4096)
    size_t tickets_n = 0;
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};
};

struct tq_ham {
    tq_ctx* ctx = nullptr;
    int device = 0;            // the context's device, kept for freeing after the context
    int n_spatial = 0, nq = 0, prec = 0, mapping = 0;
    int sector = 0, n_alpha = 0, n_beta = 0;   // sector-restricted basis
    long long D = 0, nnz = 0, n_pauli = 0, n_amb = 0;
    int max_row = 0;
    size_t bytes = 0;
    std::vector<void*> allocs;
    tq::HamView view{};
};

struct tq_pool {
    tq_ctx* ctx = nullptr;
    int device = 0;            // the context's device, kept for freeing after the context
    int n_spatial = 0, n_electrons = 0, nq = 0, mapping = 0, M = 0;
    int sector = 0, n_alpha = 0, n_beta = 0;   // sector-restricted basis
    std::vector<int> idx4;
    std::vector<tq::PauliTerm> terms;   // 8 slots per op (host copy)
    std::vector<int> nterm;
    std::vector<void*> allocs;
    tq::PoolView view{};
    bool unit = false;         // every generator's entries are +-1 (|c0| = 1)
    // on-demand CSR per (op, precision)
    std::vector<void*> csr_alloc[2];
    std::vector<const int*> csr_rowptr[2];
    std::vector<const int*> csr_col[2];
    std::vector<const void*> csr_val[2];
    std::vector<long long> csr_nnz[2];
};

struct tq_state {
    tq_ctx* ctx = nullptr;
    int device = 0;            // the context's device, kept for freeing after the context
    int nq = 0, prec = 0, owned = 0;
    int sector = 0, n_spatial = 0, n_alpha = 0, n_beta = 0;   // sector-restricted basis
    long long D = 0;
    void* data = nullptr;
};
