/*
 * tq.h -- C ABI of the GB300 (sm_103a) library for the ADAPT-VQE fifth-order
 * Taylor hot path of "Alleviating the Sparse Matrix Scaling Bottleneck in
 * Adaptive VQE via High-Order Taylor State Evolution".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status: TQ_OK (0) or a negative TQ_E*
 *    code.  No function throws or aborts.  tq_last_error() returns a
 *    thread-local, human-readable reason for the last failure on the
 *    calling thread (the pointer stays valid until the next failing call on
 *    that thread).
 *  - Qubit j is bit j of a basis index (little-endian).  A state of N qubits
 *    is D = 2^N complex amplitudes stored contiguously, real part first:
 *    TQ_C128 = two float64 per amplitude (16 B), TQ_C64 = two float32 (8 B).
 *  - Spin orbitals are interleaved: spin orbital P = 2p + sigma (sigma 0 is
 *    alpha, 1 is beta); N = 2 * n_spatial qubits.
 *  - Host arrays passed in are read during the call and copied; the caller
 *    keeps ownership.  Handles (tq_ctx, tq_ham, tq_pool, tq_state, ...) are
 *    owned by the library and released by the matching *_free / *_destroy
 *    function, each of which accepts NULL.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it.  Functions that write a HOST scalar or
 *    array synchronise that stream before returning; functions that write
 *    DEVICE memory only are asynchronous.
 *  - A tq_ctx owns device scratch that its calls share: calls on one context
 *    must be issued from one host thread at a time, on one stream (or on
 *    streams the caller orders).  Use one context per concurrent stream.
 *  - Operator values are real: the Jordan-Wigner and Bravyi-Kitaev images of
 *    real integrals and of real excitation generators have real matrix
 *    elements in the computational basis.  States are complex.
 */
#ifndef TQ_H
#define TQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Mappings (Sec. II-A): Jordan-Wigner (Eq. (4), parity string on the lower
 * qubits) and Bravyi-Kitaev (Fenwick-tree encoding: qubit k stores the
 * parity of modes k+1-lowbit(k+1) .. k). */
enum { TQ_JW = 0, TQ_BK = 1 };

/* Ids of relabelled mappings (tq_mapping_relabelled, tq_mapping_linear)
 * start here. */
#define TQ_MAPPING_FIRST_RELABELLED 16

/* Precisions: TQ_C128 runs every product and sum in float64.  TQ_C64 keeps
 * states and sparse products in complex64 (float32) while Hamiltonian
 * diagonals, energy and gradient dot reductions, norms and the convergence
 * test stay in float64. */
enum { TQ_C128 = 0, TQ_C64 = 1 };

enum {
    TQ_OK = 0,
    TQ_EINVAL = -1,    /* invalid argument (range, size, null, mismatch)   */
    TQ_ENOMEM = -2,    /* device or host allocation failed                 */
    TQ_ECUDA = -3,     /* a CUDA runtime call failed                       */
    TQ_ETIMEOUT = -4,  /* a bounded wait ran out                           */
    TQ_EBUSY = -5,     /* admission refused (memory budget or slots)       */
    TQ_ENUMERIC = -6   /* non-finite or inconsistent numerical result      */
};

/* Limits.  States up to 2^26 amplitudes; CSR indices are int32, so a
 * Hamiltonian build fails with TQ_ENOMEM when nnz would reach 2^31. */
#define TQ_MAX_SPATIAL 15
#define TQ_MAX_STATE_QUBITS 26

typedef struct tq_ctx tq_ctx;
typedef struct tq_ham tq_ham;
typedef struct tq_pool tq_pool;
typedef struct tq_state tq_state;

const char* tq_last_error(void);
int tq_version(void); /* 100 * major + minor */

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (makes it current on the calling
 * thread).  Queries the SM count and per-kernel occupancy used to size
 * persistent grids. */
int tq_ctx_create(int device, tq_ctx** out);
int tq_ctx_destroy(tq_ctx* ctx);
/* Number of kernel launches this context has issued since creation. */
int tq_ctx_launch_count(const tq_ctx* ctx, long long* launches);

/* Kernel tracing.  With tracing on, every kernel this context launches is
 * bracketed by two CUDA events recorded on the stream it is launched on.
 * tq_ctx_trace_report synchronises those events and writes one line per
 * kernel name, "name launches total_ms\n", into buf (NUL-terminated,
 * truncated to buf_size), then clears the record.  Tracing adds two event
 * records per launch and nothing else. */
int tq_ctx_trace(tq_ctx* ctx, int enable);
int tq_ctx_trace_report(tq_ctx* ctx, char* buf, size_t buf_size);

/* Launch schedule of the Taylor-5 pair kernel per precision: pair units
 * (4 amplitudes each) per thread per tile, one of 1, 2, 4, 8.  More units
 * per thread put more bytes in flight per thread; fewer raise occupancy.
 * Defaults: 2 (TQ_C128), 4 (TQ_C64). */
int tq_ctx_set_pair_schedule(tq_ctx* ctx, int prec, int units_per_thread);
int tq_ctx_get_pair_schedule(const tq_ctx* ctx, int prec, int* units_per_thread);
/* Autotuner: times each schedule on n_states device scratch states of the
 * pool's qubit count (one warm launch, then the mean of five, CUDA events
 * on the legacy stream), sets the fastest on the context, and returns it
 * with its time per launch.  Synchronises the device; uses context scratch
 * (n_states * 2^N amplitudes). */
int tq_autotune_pair(tq_ctx* ctx, const tq_pool* pool, int prec, int n_states,
                     int* best_units_per_thread, double* best_ms);

/* L2 fetch granularity of the device's CUDA context (the process's primary
 * context, shared by every tq_ctx on that device): 32, 64 or 128 bytes
 * fetched from HBM per L2 miss, or 0 for the value found when the context
 * was created.  Scattered accesses (the support-only update reads 8-byte
 * amplitudes spread over a generator's support) move fewer bytes with 32;
 * streaming kernels read whole lines either way.  It is a hint to the
 * driver, lasts as long as the CUDA context, and changes no setting of the
 * GPU itself. */
int tq_ctx_set_l2_fetch(tq_ctx* ctx, int bytes);
int tq_ctx_get_l2_fetch(tq_ctx* ctx, int* bytes);

/* Schedule of the energy SpMV (the H pass of tq_energy, tq_pool_gradients
 * and tq_adapt_step): 4, 8, 16 or 32 lanes sharing one row of the CSR,
 * or TQ_SPMV_XELL for the XOR-ELL layout (the default; a sector
 * Hamiltonian, which has only the CSR, then uses 8 lanes).  Every Hamiltonian
 * holds both layouts of the same off-diagonal entries: the CSR, and blocks
 * of 8 rows where each X-mask present in the block stores its 8 values
 * H[8R+i][(8R+i)^x] (zero where the CSR has no entry), so one pair's 8
 * gathers read one aligned run of 8 amplitudes.  The autotuner times
 * tq_energy's launch under every schedule on (ham, psi) and keeps the
 * fastest.  Synchronises the device. */
enum { TQ_SPMV_XELL = 0 };
/* Failure-path tests only (no counterpart in the paper).  With
 * TQ_TEST_WITHHOLD_CHUNK set, the XOR-ELL energy pass never copies its
 * first pair chunk into shared memory, so every consumer wait on it runs
 * out after its bound (about 2 s): the call returns TQ_ETIMEOUT with E NaN,
 * nothing faults, and the context stays usable once the flag is cleared. */
enum { TQ_TEST_WITHHOLD_CHUNK = 1 };
int tq_ctx_set_test_flags(tq_ctx* ctx, int flags);
int tq_ctx_set_spmv_schedule(tq_ctx* ctx, int lanes_per_row);
int tq_autotune_spmv(tq_ctx* ctx, const tq_ham* ham, const tq_state* psi,
                     int* best_lanes_per_row, double* best_ms);

/* ------------------------------------------------- host-side construction */

/* Qubit Hamiltonian as a Pauli sum (Eq. (3)) from the fermionic Hamiltonian
 * of Eq. (2).  The paper writes the two-body part with physicist integrals
 * h_ijkl; this entry point takes chemist integrals, (ik|jl) = <ij|kl>, so
 *   H = sum_PQ h_PQ a+_P a_Q + 1/2 sum_PQRS (PQ|RS) a+_P a+_R a_S a_Q + e_const
 * with h_PQ = h1[p*n+q] for equal spins and
 * (PQ|RS) = g2[((p*n+q)*n+r)*n+s] for sigma_P = sigma_Q, sigma_R = sigma_S.
 * Output terms are c * X^x Z^z (Z acts first), i.e. <r|term|c_> =
 * c * (-1)^popcount(c_ & z) when r = c_ xor x, with real c; sorted by
 * (x, z); like terms merged; |c| <= 1e-12 max|c| dropped.  Two-call
 * pattern: with x == NULL only *n_terms is written; otherwise `capacity`
 * must be >= the count.  Host only; needs no GPU. */
int tq_pauli_hamiltonian(int n_spatial, const double* h1, const double* g2,
                         double e_const, int mapping, long long* n_terms,
                         uint64_t* x, uint64_t* z, double* c,
                         long long capacity);

/* Excitation pool (Sec. III-E; sizes of Table II): spin-conserving
 * occupied -> virtual singles (i, a) then doubles (i, j, a, b), i < j,
 * a < b, S_z conserved, each list lexicographic; occupied spin orbitals are
 * P < n_electrons.  idx4 receives 4 ints per op, -1 padded (singles use
 * the first two).  Two-call pattern on idx4 == NULL.  Host only. */
int tq_pool_excitations(int n_spatial, int n_electrons, int* n_ops,
                        int* idx4, int capacity);

/* Generator A_k = tau_k - tau_k^+ of each pool op as a Pauli sum in the
 * same c * X^x Z^z form: x[k], nterm[k] (2 or 8), z[8k + t], c[8k + t]
 * (unused slots zero).  Host only. */
int tq_pauli_pool(int n_spatial, int n_electrons, int mapping, int capacity,
                  uint64_t* x, int* nterm, uint64_t* z, double* c);

/* Support of each pool generator, S_k = {r : A_k[r][r ^ x_k] != 0}, in the
 * reduced form the support-only update and the gradients enumerate: m[k]
 * conditions (1 for a single, 3 for a double), pivot bits pivots[3k + i]
 * ascending (-1 past m[k]) with masks masks[3k + i], each holding its own
 * pivot and no other; r is in S_k iff parity(r & masks[3k + i]) equals bit
 * i of target[k] for every i.  Pair u (0 <= u < 2^(N - m - 1)) of the
 * update is u with a zero inserted at bit rep_pos[k] and at each pivot
 * (ascending), each pivot then set by its condition: the member of the
 * pair {r, r ^ x_k} whose bit rep_bit[k] is 0.  Host only. */
int tq_pool_support_forms(int n_spatial, int n_electrons, int mapping,
                          int capacity, int* m, int* pivots, uint64_t* masks,
                          int* target, int* rep_bit, int* rep_pos);

/* A relabelled mapping: the JW or BK encoding (base_mapping) with its
 * qubit k stored at bit order[k] of the basis index (order: a permutation
 * of 0 .. n_qubits-1).  Relabelling the qubits of an encoding gives another
 * linear encoding of the same occupations (Sec. II-A), so energies,
 * gradients, norms and fidelities are those of the base mapping, and every
 * amplitude sits at the relabelled index.  It changes only how the
 * amplitudes are laid out in memory.  The returned id is accepted wherever
 * a mapping is, for this qubit count only (TQ_EINVAL otherwise);
 * registering the same relabelling again returns the same id.  Ids live
 * until the process exits (at most 4096).  Host only; thread-safe.
 * TQ_EINVAL for a base other than JW/BK, n_qubits outside [1, 30], or an
 * order that is not a permutation. */
int tq_mapping_relabelled(int base_mapping, int n_qubits, const int* order, int* mapping_out);

/* A qubit order for tq_mapping_relabelled that makes the pool's supports
 * (tq_pool_support_forms) dense in the lowest index bits.  An in-place
 * update that touches only a generator's support (the support-only batched
 * update) moves whole memory sectors, 32 bytes = the 2 lowest bits for
 * complex64 amplitudes, and a support whose conditions have rank r on the
 * lowest bits fills 2^-r of every sector it touches.  The lowest low_bits
 * bits (0 .. 2 n_spatial) are filled one at a time, each with the qubit
 * that minimises sum_k |S_k| 2^rank_k over the pool of singles and doubles
 * (ties: the lowest qubit); the other qubits follow in their base order.
 * order_out receives 2 n_spatial entries.  Host only.  TQ_EINVAL for bad
 * sizes or base mapping. */
int tq_pool_sector_order(int n_spatial, int n_electrons, int base_mapping, int low_bits, int* order_out);

/* A linearly relabelled mapping: the JW or BK encoding whose basis index r
 * is carried to r' by an invertible linear map M over GF(2), bit i of r'
 * being the parity of r over rows[i] (a mask over the base index bits; a
 * qubit permutation is the case of one bit per row, and
 * tq_mapping_relabelled registers exactly that).  The encoding matrix
 * becomes M B, another linear encoding of the same occupations (Sec.
 * II-A): energies, gradients, norms and fidelities are the base mapping's
 * and every amplitude sits at index M r.  Ids, lifetime and errors as for
 * tq_mapping_relabelled; TQ_EINVAL for a row with bits at or above
 * n_qubits or a singular map.  Host only; thread-safe. */
int tq_mapping_linear(int base_mapping, int n_qubits, const unsigned long long* rows, int* mapping_out);

/* An index map for tq_mapping_linear that makes the pool's supports dense
 * in the lowest index bits, over all invertible linear maps rather than
 * qubit orders.  New bit l stands for a vector v_l of the base index space
 * (the segments of 2^(l+1) amplitudes are the cosets of span(v_0..v_l)), a
 * support S_k fills |span cap K_k| of each segment it touches, K_k the
 * kernel of its conditions, and v_l is the vector, independent of those
 * before it, that minimises sum_k |S_k| 2^rank_k (rank_k: of the chosen
 * vectors' condition parities; ties: the smallest vector).  Every vector
 * is a candidate while 2^(2 n_spatial) x (pool size) <= 2^26, else the unit
 * vectors and their pairwise sums.  The bits after low_bits take unit
 * vectors in qubit order.  rows_out receives the 2 n_spatial rows of M.
 * For the 14-qubit BK pool the 32-byte sectors a support touches are
 * 0.83 filled against 0.70 for the best qubit order.  Host only.  TQ_EINVAL
 * for bad sizes or base mapping. */
int tq_pool_sector_basis(int n_spatial, int n_electrons, int base_mapping, int low_bits,
                         unsigned long long* rows_out);

/* Qubit-basis index of the Hartree-Fock determinant (spin orbitals
 * P < n_electrons occupied) under `mapping`.  Host only. */
int tq_hf_index(int n_qubits, int n_electrons, int mapping, long long* index);

/* ------------------------------------------------------------ Hamiltonian */

/* Build the Hamiltonian on the device (Sec. III-D step 1; CSR compilation
 * of Sec. III-E step 3).  The Pauli sum is formed on the host, uploaded once,
 * and compiled on the GPU into
 *   - diag:   float64[D], H[r][r] (the X-mask-0 group);
 *   - CSR of the off-diagonal part: rowptr int32[D+1], col int32[nnz]
 *     ascending within each row, val float64 (TQ_C128) or float32 (TQ_C64)
 *     [nnz].  An entry H[r][r^x] is the sum, in (x, z) order, of
 *     c_p (-1)^popcount((r^x) & z_p) over the terms of X-mask x; entries with
 *     |v| <= 1e-12 max|c| are dropped;
 *   - the X-mask-grouped matrix-free layout (group masks, term offsets,
 *     z masks, coefficients) used by tq_energy_matrix_free.
 * Synchronises the device.  Errors: TQ_EINVAL (sizes, mapping, precision,
 * null), TQ_ENOMEM, TQ_ECUDA, TQ_ENUMERIC (a term with an odd number of Y
 * survived, which real symmetric integrals cannot produce). */
int tq_build_hamiltonian(tq_ctx* ctx, int n_spatial, const double* h1,
                         const double* g2, double e_const, int mapping,
                         int prec, tq_ham** out);
/* Any output pointer may be NULL.  n_ambiguous counts CSR entries whose
 * magnitude fell in (1e-12, 1e-9] * max|c|, where the zero-drop decision
 * would be fragile (expected 0). */
int tq_ham_info(const tq_ham* ham, int* n_qubits, int* prec, long long* nnz,
                long long* n_pauli, long long* n_xgroups, long long* n_ambiguous,
                size_t* device_bytes);
/* Borrowed device pointers (valid until tq_ham_free). */
int tq_ham_csr(const tq_ham* ham, const int** rowptr, const int** col,
               const void** val, const double** diag);
/* Borrowed device pointers to the XOR-ELL layout of the same off-diagonal
 * entries (no counterpart in the paper; it is a second storage order of
 * the CSR's values).  Rows come in blocks of 8; block R's pairs are
 * xptr[R] .. xptr[R+1]-1 (int32, n_blocks + 1 = ceil(2^N / 8) + 1 entries),
 * pair p has X-mask xmask[p] (uint32) and values xval[8p + i] =
 * H[8R+i][(8R+i) ^ xmask[p]] (double for TQ_C128, float for TQ_C64, zero
 * where the CSR drops the entry); a block's pairs are the X-mask groups
 * with a kept entry in any of its rows, in ascending group order.  Any
 * output pointer may be NULL. */
int tq_ham_xell(const tq_ham* ham, long long* n_blocks, long long* n_pairs,
                const int** xptr, const unsigned** xmask, const void** xval);
int tq_ham_free(tq_ham* ham);

/* ------------------------------------------------------------------- pool */

/* Build the pool (Sec. III-D step 2) in the vectorised device layout of
 * Sec. III-E: structure-of-arrays x[M], nterm[M], z[8M], c[8M].  Every
 * generator has one X-mask, at most one non-zero per row and column, and
 * entries in {0, +1, -1}. */
int tq_build_pool(tq_ctx* ctx, int n_spatial, int n_electrons, int mapping,
                  tq_pool** out);
/* M, qubit count, and (if idx4 != NULL) 4 ints per op as in
 * tq_pool_excitations. */
int tq_pool_info(const tq_pool* pool, int* n_ops, int* n_qubits, int* idx4);
/* On-the-fly sparse compilation (Sec. III-E step 3): CSR of generator k,
 * built on the device the first time it is asked for and cached.  Values
 * are float64 (TQ_C128) or float32 (TQ_C64).  Borrowed device pointers. */
int tq_pool_csr(tq_ctx* ctx, tq_pool* pool, int k, int prec,
                const int** rowptr, const int** col, const void** val,
                long long* nnz);
int tq_pool_free(tq_pool* pool);

/* ------------------------------------------------------------------ state */

int tq_state_create(tq_ctx* ctx, int n_qubits, int prec, tq_state** out);
/* Borrow caller memory (e.g. a torch tensor's data_ptr()): D amplitudes,
 * 16-byte aligned.  The caller keeps it alive and orders streams. */
int tq_state_wrap(tq_ctx* ctx, int n_qubits, int prec, void* dev_ptr,
                  tq_state** out);
int tq_state_data(const tq_state* st, void** dev_ptr, int* n_qubits, int* prec);
/* |HF>: the basis state of tq_hf_index, amplitude 1 (async). */
int tq_state_set_hf(tq_state* st, int n_electrons, int mapping, void* stream);
int tq_state_free(tq_state* st);

/* ------------------------------------------------- integrals and checkpoints */
/* FCIDUMP integral files (host only; the paper's molecular integrals are
 * not available, so real ones are supplied this way).  Format: a namelist
 * header "&FCI NORB=n, NELEC=ne, MS2=m, ... &END" (or "/"), then lines
 * "value i j k l" with 1-based orbitals: all non-zero -> chemist (ij|kl),
 * k = l = 0 -> h_ij, all zero -> core energy, other patterns skipped; each
 * (ij|kl) line fills its 8 real-orbital symmetry partners and each h_ij
 * line also h_ji; a Fortran D exponent is accepted.
 * tq_read_fcidump: header values into n_spatial, n_electrons, ms2 (any may
 * be NULL); with h1 (n*n, row-major) and/or g2 (n^4, [((p*n+q)*n+r)*n+s] =
 * (pq|rs), the layout tq_build_hamiltonian takes) and/or e_core non-NULL,
 * also the integrals (entries not in the file are 0; capacity_n >= n).
 * TQ_EINVAL: unreadable file, missing header key, NORB outside [1, 15],
 * an orbital index above NORB, a malformed line.
 * tq_write_fcidump: the symmetry-unique entries with |v| > tol (i >= j,
 * k >= l, pair(ij) >= pair(kl); then h_ij with i >= j; then the core
 * energy), %.16E: a read-back is exact. */
int tq_read_fcidump(const char* path, int* n_spatial, int* n_electrons, int* ms2,
                    double* e_core, double* h1, double* g2, int capacity_n);
int tq_write_fcidump(const char* path, int n_spatial, int n_electrons, int ms2,
                     const double* h1, const double* g2, double e_core, double tol);
/* State checkpoints: a 40-byte header (magic "TQSTATE1", int32 precision,
 * qubits, sector flag, n_alpha, n_beta, 0, int64 amplitude count) and the
 * amplitudes as stored on the device.  tq_state_load requires the header
 * to match the target state (TQ_EINVAL otherwise).  Both synchronise the
 * device. */
int tq_state_save(const tq_state* st, const char* path);
int tq_state_load(tq_state* st, const char* path);

/* -------------------------------------- ADAPT-VQE with re-optimised angles */
/* Not in the paper, whose loop (Sec. III-D) sets only the newest angle: the
 * standard ADAPT-VQE form of that loop on the same Taylor-5 factors
 * U_j(t) = sum_{m<=5} (t A_j)^m / m! of Eqs. (6)-(8).
 *
 * tq_ansatz_energy_grad: for psi(theta) = U_n(theta_n) ... U_1(theta_1) psi0
 * (no renormalisation), E = Re<psi|H|psi>/<psi|psi> (Eq. (1)) into *E and,
 * if grad is not NULL, dE/dtheta_j into grad[0 .. n_ops-1], exact for the
 * product (one forward sweep that keeps the n_ops + 1 states in context
 * scratch, one adjoint sweep: chi = (H - E) psi, grad_j =
 * 2 Re<chi_j | U_j'(theta_j) phi_{j-1}> / <psi|psi>, chi_{j-1} =
 * U_j(-theta_j) chi_j).  ops, thetas, E, grad: host arrays; psi0 (not
 * modified) and psi_out (optional, receives psi(theta)) are states of the
 * pool's space (full or sector).  Synchronises the stream.  TQ_EINVAL for
 * an op index out of range, a non-finite angle or mismatched spaces.
 *
 * tq_adapt_vqe: from psi0, repeat up to max_ops times: pool gradients at
 * psi(theta), the operator with the largest |g| (tie rule of
 * tq_adapt_step), stop if max|g| < eps, else append it with angle 0 and
 * re-optimise every angle by BFGS (inverse-Hessian update, backtracking
 * line search; stop at max |dE/dtheta| < gtol or max_iter iterations).
 * Writes n_ops and ops_out, thetas_out, energies_out (host arrays of
 * max_ops; energies_out[i] = the optimised energy with i + 1 operators),
 * and psi(theta) into psi_out if not NULL.  Runs on the legacy stream. */
int tq_ansatz_energy_grad(tq_ctx* ctx, const tq_ham* ham, const tq_pool* pool,
                          const tq_state* psi0, int n_ops, const int* ops,
                          const double* thetas, double* E, double* grad,
                          tq_state* psi_out, void* stream);
int tq_adapt_vqe(tq_ctx* ctx, const tq_ham* ham, const tq_pool* pool,
                 const tq_state* psi0, double eps, int max_ops, double gtol,
                 int max_iter, int* n_ops, int* ops_out, double* thetas_out,
                 double* energies_out, tq_state* psi_out);

/* ----------------------------------------------------- commuting families */
/* Sec. III-F, Algorithm 1: partition of the pool into families of mutually
 * commuting generators by a largest-first greedy colouring of the
 * non-commutativity graph (vertices by descending degree, ties by pool
 * index; each joins the lowest-indexed family holding none of its
 * neighbours, else opens a new one).  The paper names the relation two
 * ways; `mode` picks one:
 *   TQ_COMMUTE_FULL: an edge where [A_i, A_j] != 0 as operators (exact:
 *     the commutator's Pauli expansion has dyadic coefficients);
 *   TQ_COMMUTE_QWC:  an edge unless every Pauli string of A_i commutes
 *     qubit-wise with every string of A_j.
 * Outputs (host arrays of M = pool size, any may be NULL): family[k] in
 * [0, n_families); order = pool indices family by family, ascending inside
 * a family (the family-contiguous layout of the pool).  Host only: the
 * _host variant builds the pool's strings itself (no device, no context);
 * TQ_EINVAL if capacity < M or mode is unknown. */
enum { TQ_COMMUTE_FULL = 0, TQ_COMMUTE_QWC = 1 };
int tq_pool_families(const tq_pool* pool, int mode, int* family, int* order,
                     int* n_families);
int tq_pool_families_host(int n_spatial, int n_electrons, int mapping, int mode,
                          int capacity, int* family, int* order, int* n_families);

/* ---------------------------------------------- sector-restricted basis */
/* Not in the paper, which works in the full 2^N space: the same operators
 * restricted to the occupation states with n_alpha electrons in the even
 * spin orbitals (alpha, P = 2p) and n_beta in the odd ones (beta).  H of
 * Eq. (2) and every spin-conserving pool generator map this subspace into
 * itself, so energies, gradients and Taylor-5 updates of a state in it are
 * those of the full space, with C(n, n_alpha) C(n, n_beta) amplitudes
 * instead of 2^(2n) (14 qubits, 3 + 3 electrons: 1225 instead of 16384).
 * Basis order: rank = rank_alpha * C(n, n_beta) + rank_beta, rank_x the
 * colexicographic rank of the occupied x-spin spatial orbitals
 * {c_1 < ... < c_k}: sum_j C(c_j, j).  The matrices in this order do not
 * depend on the mapping; the mapping fixes only the qubit-space index of
 * each basis state.  1 <= n_spatial <= 13, 0 <= n_alpha, n_beta <=
 * n_spatial, else TQ_EINVAL. */
int tq_sector_dim(int n_spatial, int n_alpha, int n_beta, long long* dim);
/* Host: qubit-space index (under `mapping`) of every basis state, in rank
 * order, into qubit_index[0 .. dim-1]; TQ_EINVAL if capacity < dim. */
int tq_sector_basis(int n_spatial, int n_alpha, int n_beta, int mapping,
                    long long capacity, unsigned* qubit_index);
/* As tq_build_hamiltonian, restricted to the sector: float64 diagonal and
 * CSR (rowptr int32[dim+1], col int32 ascending, real values) over ranks,
 * read with tq_ham_csr; no XOR-ELL layout (tq_energy uses the CSR). */
int tq_build_hamiltonian_sector(tq_ctx* ctx, int n_spatial, const double* h1,
                                const double* g2, double e_const, int mapping,
                                int prec, int n_alpha, int n_beta, tq_ham** out);
/* As tq_build_pool, plus each generator restricted to the sector: per op k
 * and row r, col[k*dim + r] (int32) and sgn[k*dim + r] (int8) with
 * A_k[r][col] = sgn = +-1, or sgn = 0 where A_k annihilates row r (then
 * col = r).  TQ_ENUMERIC if a generator leaves the sector.  The sector pool
 * drives tq_evolve_taylor5, tq_evolve_taylor5_batch(_host) (states of dim
 * amplitudes), tq_pool_gradients and tq_adapt_step with sector
 * Hamiltonians and states; the trajectory batch, the request loop and the
 * pair autotuner take full-space objects only. */
int tq_build_pool_sector(tq_ctx* ctx, int n_spatial, int n_electrons,
                         int mapping, int n_alpha, int n_beta, tq_pool** out);
/* Borrowed device pointers to a sector pool's tables (dim = 0 and NULL
 * tables for a full-space pool). */
int tq_pool_sector_table(const tq_pool* pool, long long* dim, const int** col,
                         const signed char** sgn);
/* Sector states: dim amplitudes in rank order, owned (zeroed) or borrowed
 * (16-byte aligned).  tq_state_set_hf puts the lowest determinant (spin
 * orbitals P < n_electrons; rank 0) and fails with TQ_EINVAL unless
 * n_alpha = ceil(n_electrons/2) and n_beta = floor(n_electrons/2).  Every
 * hot-path call checks that Hamiltonian, pool and state describe the same
 * space (full, or the same sector): TQ_EINVAL otherwise. */
int tq_state_create_sector(tq_ctx* ctx, int n_spatial, int n_alpha, int n_beta,
                           int prec, tq_state** out);
int tq_state_wrap_sector(tq_ctx* ctx, int n_spatial, int n_alpha, int n_beta,
                         int prec, void* dev_ptr, tq_state** out);

/* ------------------------------------------------------------- hot path */

/* Fifth-order Taylor update of Sec. III-C, Eqs. (6)-(8):
 *   v_0 = psi, v_k = A v_{k-1} (k = 1..5),
 *   psi <- psi + theta v_1 + theta^2/2 v_2 + ... + theta^5/120 v_5,
 * with A = pool generator k, applied matrix-free from the pool layout.  The
 * five products and the running sum stay in registers; psi is read once
 * and written once.  If renormalize != 0 the result is divided by its
 * float64 norm: for states of up to 2^16 amplitudes in the same launch (a
 * thread-block cluster holds the state while the norm is reduced), for
 * larger ones in a second, L2-resident pass.  Async.  Errors: TQ_EINVAL
 * (k out of range, qubit mismatch, non-finite theta). */
int tq_evolve_taylor5(tq_ctx* ctx, const tq_pool* pool, int k, double theta,
                      tq_state* psi, int renormalize, void* stream);

/* The same update for an arbitrary CSR operator A (rowptr int32[D+1], col
 * int32[nnz], val float64 for TQ_C128 / float32 for TQ_C64 states, device
 * pointers).  The caller guarantees rowptr is non-decreasing with
 * rowptr[0] = 0 and rowptr[D] = nnz; column indices outside [0, D) are
 * skipped (treated as zero entries).  The state is staged in shared
 * memory -- across a thread-block cluster of up to 16 CTAs, read through
 * distributed shared memory, up to 2^17 complex64 or 2^16 complex128
 * amplitudes -- and never returns to global memory between the five
 * products; the lanes per row follow the operator's mean row length; the
 * float64 norm is reduced across the cluster and, if renormalize != 0,
 * applied before the single store.  Larger states use one L2-resident pass
 * per product.  Async. */
int tq_evolve_taylor5_csr(tq_ctx* ctx, int n_qubits, const int* rowptr,
                          const int* col, const void* val, double theta,
                          tq_state* psi, int renormalize, void* stream);

/* Energy of Eq. (1): E = Re<psi|H|psi> / <psi|psi>, float64.  One fused
 * pass: SpMV over the CSR or the XOR-ELL layout (the context's SpMV
 * schedule; w = H psi, kept in context scratch for tq_pool_gradients) and
 * float64 warp-shuffle dot products.  The XOR-ELL pass streams its pairs
 * through shared memory with bulk copies; its waits are bounded, and a
 * wait that runs out returns TQ_ETIMEOUT (E is then NaN).  Writes the host
 * scalar *E (synchronises the stream). */
int tq_energy(tq_ctx* ctx, const tq_ham* ham, const tq_state* psi, double* E,
              void* stream);
/* Energy that allocates nothing (the paper has no counterpart: it serves
 * callers that cannot call cudaMalloc or cudaFree where they need an energy,
 * such as serving loops that reserved their memory up front and must not
 * stall the device on an allocation, or hosts whose own allocator owns the
 * device heap).  Same arithmetic as tq_energy (float64 warp-shuffle sums of
 * the fused CSR SpMV), on the calling thread's current device, with inputs
 * given as device pointers: the off-diagonal CSR (rowptr int32[D+1], col
 * int32, val float64 for TQ_C128 / float32 for TQ_C64), the float64
 * diagonal[D], and the state psi (D amplitudes of `prec`).  The energy is
 * written to energy_out (one float64 in device memory), stream-ordered on
 * `stream`; the call does not synchronise.
 * Its scratch is one fixed 64 KiB array in device global memory that every
 * GPU loading the library holds until the process exits; it bounds the
 * reduction to 4064 CTA partials.  The first call on a device resolves that
 * array's device address (cudaGetSymbolAddress) and the SM count, so make
 * the first call before any stream capture.  Every call shares the array:
 * calls that overlap on the GPU (other streams, other threads) race and
 * must be ordered by the caller.  Errors: TQ_EINVAL (null pointer,
 * precision, n_qubits outside [1, 26], or a reduction larger than the
 * scratch holds), TQ_ECUDA. */
int tq_energy_noalloc(int n_qubits, int prec, const int* rowptr, const int* col,
                      const void* val, const double* diag, const void* psi,
                      double* energy_out, void* stream);

/* Same energy, computed from the X-mask-grouped Pauli layout without the
 * CSR (cross-check of the CSR build).  Each row's terms are evaluated and
 * summed in float64, an add per term and row, so the float64 pipe bounds
 * it (see tq_fp64_fma_rate).  Full space only (TQ_EINVAL for a sector
 * Hamiltonian or a state of another space).  Synchronises the stream. */
int tq_energy_matrix_free(tq_ctx* ctx, const tq_ham* ham, const tq_state* psi,
                          double* E, void* stream);

/* Pool gradients of Eq. (5): g_k = <psi|[H, A_k]|psi> / <psi|psi>
 *                                = 2 Re<H psi|A_k psi> / <psi|psi>
 * for all k in one persistent launch after one H pass; float64 sums.
 * `g` has M entries; g_on_device != 0 means `g` is a device pointer (async),
 * otherwise a host pointer (synchronises). */
int tq_pool_gradients(tq_ctx* ctx, const tq_ham* ham, const tq_pool* pool,
                      const tq_state* psi, double* g, int g_on_device,
                      void* stream);

/* One ADAPT iteration (Sec. III-D steps 3-4) entirely on the device:
 * energy, all gradients, k* = argmax |g_k| (tie rule: the lowest k with
 * |g_k| >= max|g| - tau, tau = 1e-9 max(1, max|g|) in TQ_C128 and 1e-5 in
 * TQ_C64), converged = max|g| < eps; if not converged, the Taylor-5 update
 * with A_{k*} and angle `theta`, or, when theta is NaN, the angle that
 * minimises the energy along exp(theta A_{k*}) psi on (-pi, pi] (4096
 * samples, ties within 1e-10 to the smallest |theta|, Newton polish), then
 * renormalisation.  `energy` is the energy before the update.  Writes *out
 * (synchronises). */
typedef struct {
    double energy;
    double max_grad;
    double theta;
    int selected;
    int converged;
} tq_adapt_result;
int tq_adapt_step(tq_ctx* ctx, const tq_ham* ham, const tq_pool* pool,
                  tq_state* psi, double eps, double theta,
                  tq_adapt_result* out, void* stream);

/* n_iter ADAPT steps in a row (the loop of Sec. III-D) without a host round
 * trip between them: the first step is launched directly, the next ones
 * replay one captured CUDA graph of a step.  thetas (host, n_iter finite
 * angles, copied) gives step i its angle; NULL runs the line search at every
 * step (as tq_adapt_step with theta = NaN).  results[i] receives step i's
 * result as tq_adapt_step reports it; *n_done is the number of steps up to
 * and including the first converged one (n_iter if none converged).  Steps
 * after convergence leave the state as it is (their records repeat the
 * converged result).  TQ_ENUMERIC with *n_done = i + 1 if the update of
 * step i left a non-finite or zero norm.  Runs on a stream of the context
 * after the caller's stream is idle; synchronises.  Bit-identical to n_iter
 * calls of tq_adapt_step. */
int tq_adapt_run(tq_ctx* ctx, const tq_ham* ham, const tq_pool* pool,
                 tq_state* psi, double eps, const double* thetas, int n_iter,
                 tq_adapt_result* results, int* n_done, void* stream);

/* ------------------------------------------------------------ batched */

/* Batched Taylor-5: n_states states of the pool's qubit count, stored
 * back to back from psi (device, D amplitudes each, in place); state b is
 * updated with generator k[b] and angle theta[b] (device arrays).  If norm2
 * is not NULL it receives float64 ||psi_b'||^2 per state (renormalisation
 * is left to the consumer: every energy and gradient here is a Rayleigh
 * quotient).  A state whose k[b] is outside [0, M) is left unchanged and
 * its norm2 is NaN.  One streaming launch plus a per-state reduction.
 * Async. */
int tq_evolve_taylor5_batch(tq_ctx* ctx, const tq_pool* pool, int n_states,
                            int prec, void* psi, const int* k,
                            const double* theta, double* norm2, void* stream);

/* Support-only batched Taylor-5 (Sec. III-C: each product of Eq. (7) is
 * O(nnz(A))).  Same states, generators and angles as
 * tq_evolve_taylor5_batch, and the same amplitudes out, but only the rows
 * on the support of A_k[b] (D/2 for a single excitation, D/8 for a double)
 * are read and written: A annihilates every other row, so all terms of
 * Eq. (6) past the first leave it unchanged.  norm2 (device, optional) is
 * IN/OUT: on entry ||psi_b||^2, on exit ||psi_b'||^2, carried as the entry
 * value plus the change over the support (a state whose norm is not known
 * can take it from tq_evolve_taylor5_batch or a dot product first).  A
 * state whose k[b] is outside [0, M) is left unchanged and its norm2 set to
 * NaN.  Full-space pools only (TQ_EINVAL for a sector pool).  One
 * streaming launch plus a per-state reduction.  Async. */
int tq_evolve_taylor5_batch_support(tq_ctx* ctx, const tq_pool* pool,
                                    int n_states, int prec, void* psi,
                                    const int* k, const double* theta,
                                    double* norm2, void* stream);

/* The support-only update on states in HOST memory, read and written in
 * place by the kernel over the host link (NVLink-C2C on Grace-Blackwell):
 * only the support sectors cross it.  psi_host must be page-locked and
 * mapped for the device (cudaHostAlloc, or cudaHostRegister with the
 * mapped flag), else TQ_EINVAL before any launch.  k_host, theta_host and
 * norm2_host (in/out as above, optional) are ordinary host arrays, copied.
 * Synchronises. */
int tq_evolve_taylor5_batch_support_host(tq_ctx* ctx, const tq_pool* pool,
                                         int n_states, int prec,
                                         void* psi_host, const int* k_host,
                                         const double* theta_host,
                                         double* norm2_host);

/* Schedule of the support-only update: support pairs per thread per pass,
 * 1, 2, 4 or 8 with the amplitudes held in registers, or -1, -2, -4, -8
 * with them staged in shared memory by asynchronous copies that run one
 * pass ahead (across states).  Defaults: 4 for TQ_C128, -1 for TQ_C64. */
int tq_ctx_set_support_schedule(tq_ctx* ctx, int prec, int pairs_per_thread);
/* A measurement aid with no counterpart in the paper: the support-only
 * batched update's launch (the pipelined form with the context's pairs per
 * pass, the same tile set-up, state queue, barriers and norm finish) with
 * the update taken out.  Every support row it would touch is read and
 * written back unchanged, so psi keeps its bits, and norm2 (may be null;
 * then the states are taken in a fixed stride) keeps its values (an op
 * index outside [0, M) makes that state's norm NaN, as in the update).  Timing
 * it gives the floor that this access pattern sets for the update.  Async.
 * Errors as tq_evolve_taylor5_batch_support. */
int tq_evolve_taylor5_batch_support_touch(tq_ctx* ctx, const tq_pool* pool, int n_states, int prec, void* psi,
                                          const int* k, double* norm2, void* stream);
/* The support-only batched update for groups of states that share a
 * generator, in an interleaved layout (a layout choice with no counterpart
 * in the paper; the update is that of Eqs. (6)-(8) as above).  A group is
 * TQ_GROUP_C64 = 4 complex64 or TQ_GROUP_C128 = 2 complex128 states, the
 * 32 bytes of one memory sector: element (g, r, s) -- group g, amplitude r
 * (0 <= r < D), state s of the group -- is at psi[(g D + r) G + s], so one
 * support row of a group is one whole sector and every touched sector is
 * used in full.  k: int32[n_groups] device, the generator of each group;
 * theta, norm2: [n_groups G] device, per state (norm2 may be null; else
 * in/out as in tq_evolve_taylor5_batch_support).  Each state's amplitudes
 * equal what tq_evolve_taylor5_batch_support gives it; its norm agrees to
 * rounding (another summation order).  psi 32-byte aligned.  Async.
 * TQ_EINVAL for a sector pool, bad sizes or alignment; an op index outside
 * [0, M) leaves its group untouched and its norms NaN. */
#define TQ_GROUP_C64 4
#define TQ_GROUP_C128 2
int tq_evolve_taylor5_batch_grouped(tq_ctx* ctx, const tq_pool* pool, int n_groups, int prec, void* psi,
                                    const int* k, const double* theta, double* norm2, void* stream);
/* Schedule of that update: lanes_per_row threads share each support row
 * of a group, each holding G / lanes_per_row of its states (1 or 2, and 4
 * for TQ_C64), with pairs_per_thread pairs each (1, 2 or 4).  Default
 * (1, 1).  Every schedule gives the same amplitudes.  TQ_EINVAL
 * otherwise. */
int tq_ctx_set_grouped_schedule(tq_ctx* ctx, int prec, int lanes_per_row, int pairs_per_thread);

/* Resident CTAs per SM of the support-only update (its persistent grid is
 * that many CTAs per SM): 0 (the default) takes as many as fit, 1..32
 * fewer.  Fewer concurrent states per SM can raise DRAM locality for the
 * scattered support runs; a tuning knob with no counterpart in the paper.
 * TQ_EINVAL for a bad precision or count. */
int tq_ctx_set_support_occupancy(tq_ctx* ctx, int prec, int ctas_per_sm);
/* Autotuner of that schedule, as tq_autotune_pair: times each on n_states
 * device scratch states (the update and its norm), keeps the fastest on
 * the context and returns it with its time per launch.  Synchronises. */
int tq_autotune_support(tq_ctx* ctx, const tq_pool* pool, int prec,
                        int n_states, int* best_pairs_per_thread,
                        double* best_ms);

/* Measured float64 FMA rate of the context's device, in float64 lane
 * operations per second (one fused multiply-add, two flops, on one lane
 * each): the roofline of the complex128 updates, which the float64 pipe
 * bounds on this part rather than HBM.  Launches a microbenchmark of
 * independent FMA chains (iters steps of 8 chains per thread, 8 CTAs of
 * 256 threads per SM; 1 <= iters <= 2^20, about 4096 for a 20 ms launch)
 * on the legacy default stream and keeps the fastest of three timed
 * launches.  Synchronises.  TQ_EINVAL for a null argument or iters out of
 * range. */
int tq_fp64_fma_rate(tq_ctx* ctx, int iters, double* lane_ops_per_s);

/* The device's L2 read rate (no passage of the paper; the roofline of the
 * kernels whose working set stays in L2, such as the pool gradients, which
 * read H psi and psi at every support row of every generator).  A buffer
 * of `bytes` (1 MiB to 256 MiB, a multiple of 16; keep it well inside
 * the L2) from the context's scratch is zeroed, read once to bring it into
 * L2, then read `reps` times (1 to 4096) by 4 CTAs of 512 threads per SM
 * with 16-byte loads that bypass L1; the fastest of three launches gives
 * *bytes_per_s.  Runs on the legacy default stream and synchronises.
 * TQ_EINVAL for a null argument or a size out of range. */
int tq_l2_read_rate(tq_ctx* ctx, long long bytes, int reps, double* bytes_per_s);

/* The same batch with HOST buffers (psi, k, theta, norm2 in host memory;
 * pinned memory gives full copy speed): the batch is cut into chunks whose
 * host-to-device copy, update and device-to-host copy overlap on three
 * streams.  Synchronises.  Device staging comes from the context. */
int tq_evolve_taylor5_batch_host(tq_ctx* ctx, const tq_pool* pool,
                                 int n_states, int prec, void* psi_host,
                                 const int* k_host, const double* theta_host,
                                 double* norm2_host);

/* --------------------------------------------------- trajectory batches */

/* Many independent ADAPT trajectories (the loop of Sec. III-D) advanced
 * together.  Trajectory t uses Hamiltonian hams[t] and pool pools[t] (same
 * qubit count; every Hamiltonian of one batch has the same precision, which
 * is the states' precision), starts from the Hartree-Fock state of
 * n_electrons[t] under mappings[t], and runs at most lengths[t] iterations,
 * iteration i using angle thetas[off_t + i] (off_t = sum of the earlier
 * lengths) unless max|g| < eps stops it first.  Each iteration is energy,
 * all gradients, selection (tie rule of tq_adapt_step) and the Taylor-5
 * update; the energy and gradients are divided by <psi|psi>, so the state
 * is renormalised once, after the last iteration, which changes only
 * rounding against renormalising every step.  The batch owns its states and
 * keeps the handles it was given (they must outlive it).  Every iteration of
 * every trajectory is four persistent launches over static work tables, and
 * the run ends with one renormalisation launch; finished trajectories are
 * left out on the device (the energy launch runs over the active
 * trajectories' items, numbered by the previous iteration; the others test
 * a flag), so a run needs no host round trip. */
typedef struct tq_batch tq_batch;
int tq_batch_create(tq_ctx* ctx, int n_traj, tq_ham* const* hams,
                    tq_pool* const* pools, const int* n_electrons,
                    const int* mappings, const int* lengths,
                    const double* thetas, double eps, tq_batch** out);
/* The energy SpMV's schedule: lanes that share one CSR row (4, 8, 16,
 * 32), or TQ_SPMV_XELL for the XOR-ELL layout (8-row blocks, each X-mask's
 * 8 values stored together, so a pair's gathers read one aligned run). */
int tq_batch_set_schedule(tq_batch* b, int lanes_per_row);
/* Autotuner: times the energy launch under each schedule (TQ_SPMV_XELL, 4,
 * 8, 16, 32) on the batch's own states (reset to Hartree-Fock), keeps the
 * fastest. */
int tq_batch_autotune(tq_batch* b, int* lanes_per_row, double* best_ms);
/* Reset every state to Hartree-Fock and run all iterations, enqueued on
 * `stream`.  use_graph != 0 replays one CUDA graph holding every iteration
 * (captured on the first such call and after a schedule change).  Async. */
int tq_batch_run(tq_batch* b, int use_graph, void* stream);
/* Per trajectory: iterations evaluated and the converged flag; per
 * iteration (laid out like `thetas`): energy before the update, max|g|,
 * selected op, angle used (0 on the converged iteration).  Any output may
 * be NULL.  Synchronises the device. */
int tq_batch_results(const tq_batch* b, int* n_iter, int* converged,
                     double* energy, double* max_grad, int* selected,
                     double* theta);
/* Borrowed device pointer to trajectory t's state. */
int tq_batch_state(const tq_batch* b, int t, void** dev_ptr, int* n_qubits);
int tq_batch_free(tq_batch* b);

/* ----------------------------------------------------------- request loop */

/* A request loop that batches evolve, energy and gradient requests on
 * resident sessions continuously (the paper runs one trajectory at a time;
 * this serves many at once).  Each session is a state of one registered
 * Hamiltonian and its pool, created at the Hartree-Fock state.  A server
 * thread forms ticks from the queue in arrival order -- at most one request
 * per session per tick (a session's requests complete in submission order),
 * at most max_batch per tick, and only while the per-request working memory
 * (w = H psi, gradients, their partials) fits the arena: admission is by
 * HBM footprint -- and runs each tick as one batched launch per step; the
 * next tick is formed while the current one runs.  Evolve applies the
 * Taylor-5 update of the given op and angle and renormalises; energy is
 * Eq. (1); gradients returns max |g| and its op (the ADAPT selection rule)
 * and the energy.  A request's result does not depend on the other
 * requests of its tick.  While the server runs it owns its context: issue
 * no other call on that context until tq_server_stop. */
enum { TQ_REQ_EVOLVE = 0, TQ_REQ_ENERGY = 1, TQ_REQ_GRADIENTS = 2 };
typedef struct {
    int kind;                 /* TQ_REQ_*                                  */
    int session;              /* session id                                */
    int op;                   /* pool op (evolve)                          */
    int pad;
    double theta;             /* angle (evolve)                            */
    unsigned long long tag;   /* caller's id, returned in the completion   */
} tq_request;
typedef struct {
    unsigned long long tag;
    int kind, session, status, argmax;   /* argmax: gradients, else -1     */
    double energy;            /* energy and gradients requests             */
    double max_grad;          /* gradients requests                        */
    double norm2;             /* evolve: ||psi'||^2 before renormalising;
                                 others: <psi|psi>                         */
    double t_submit, t_done;  /* steady-clock seconds, for latency         */
} tq_completion;
typedef struct tq_server tq_server;
/* hbm_budget covers session states (at most half of it) and the working
 * arena (the rest, allocated at start). */
int tq_server_create(tq_ctx* ctx, int prec, size_t hbm_budget, int max_batch,
                     tq_server** out);
int tq_server_add_hamiltonian(tq_server* s, const tq_ham* ham, const tq_pool* pool,
                              int* ham_id);
/* TQ_EBUSY when the session's state would exceed half of the budget. */
int tq_server_add_session(tq_server* s, int ham_id, int n_electrons, int mapping,
                          int* session_id);
int tq_server_start(tq_server* s);
/* Thread-safe enqueue; TQ_EBUSY when the queue is full. */
int tq_server_submit(tq_server* s, const tq_request* req);
/* Up to max completions; waits at most timeout_us for the first one and
 * returns TQ_ETIMEOUT if none arrived. */
int tq_server_poll(tq_server* s, tq_completion* out, int max, int* n_out,
                   int timeout_us);
int tq_server_stats(const tq_server* s, long long* ticks, long long* completed,
                    long long* queued);
/* Borrowed device pointer to a session's state (read it only when idle). */
int tq_server_session_state(const tq_server* s, int session, void** dev_ptr,
                            int* n_qubits);
/* Stop the server thread after the ticks in flight; queued requests stay. */
int tq_server_stop(tq_server* s);
int tq_server_free(tq_server* s);

#ifdef __cplusplus
}
#endif

#endif /* TQ_H */
