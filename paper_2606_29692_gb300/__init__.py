"""GB300 (sm_103a) library for the ADAPT-VQE fifth-order Taylor hot path.

Thin Python binding over the C ABI of ``include/tq.h``: every function here
only marshals arguments (numpy arrays for host data, torch tensors for device
memory, torch streams) and calls the native library, where all of the
method's steps run.  Names follow the C entry points without the ``tq_``
prefix.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from ._native import (TQ_BK, TQ_C64, TQ_C128, TQ_JW, AdaptResult, Completion, Request, TQError, call,
                      lib)

TQ_REQ_EVOLVE, TQ_REQ_ENERGY, TQ_REQ_GRADIENTS = 0, 1, 2
TQ_SPMV_XELL = 0      # energy-SpMV schedule: the XOR-ELL layout (else CSR lanes per row)
TQ_TEST_WITHHOLD_CHUNK = 1

__all__ = [
    "TQ_JW", "TQ_BK", "TQ_C128", "TQ_C64", "TQError", "Context", "Hamiltonian", "Pool", "State",
    "pauli_hamiltonian", "pool_excitations", "pauli_pool", "hf_index", "build_hamiltonian",
    "build_pool", "evolve_taylor5", "evolve_taylor5_csr", "energy", "energy_matrix_free",
    "pool_gradients", "adapt_step", "evolve_taylor5_batch", "evolve_taylor5_batch_host",
    "state_set_hf", "pool_csr", "ham_csr", "lib", "autotune_pair", "fp64_fma_rate", "energy_noalloc", "Batch", "autotune_spmv", "Server",
    "TQ_REQ_EVOLVE", "TQ_REQ_ENERGY", "TQ_REQ_GRADIENTS", "TQ_SPMV_XELL", "ham_xell",
    "sector_dim", "sector_basis", "build_hamiltonian_sector", "build_pool_sector", "pool_sector_table",
    "TQ_COMMUTE_FULL", "TQ_COMMUTE_QWC", "pool_families", "pool_families_host",
    "ansatz_energy_grad", "adapt_vqe", "read_fcidump", "write_fcidump", "state_save", "state_load", "replay",
]


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return C.c_void_p(a.ctypes.data)
    return C.c_void_p(a.data_ptr())      # torch tensor


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _torch_dtype(prec):
    import torch
    return torch.complex128 if prec == TQ_C128 else torch.complex64


# ------------------------------------------------------------- host algebra

def pauli_hamiltonian(h1, g2, e_const, mapping):
    """Pauli sum of the qubit Hamiltonian: arrays (x, z, c) of ``c X^x Z^z``."""
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    g2 = np.ascontiguousarray(g2, dtype=np.float64)
    n = h1.shape[0]
    cnt = C.c_longlong()
    call("tq_pauli_hamiltonian", n, _ptr(h1), _ptr(g2), float(e_const), mapping, C.byref(cnt),
         None, None, None, 0)
    x = np.zeros(cnt.value, dtype=np.uint64)
    z = np.zeros(cnt.value, dtype=np.uint64)
    c = np.zeros(cnt.value, dtype=np.float64)
    call("tq_pauli_hamiltonian", n, _ptr(h1), _ptr(g2), float(e_const), mapping, C.byref(cnt),
         _ptr(x), _ptr(z), _ptr(c), cnt.value)
    return x, z, c


def pool_excitations(n_spatial, n_electrons):
    """Pool excitations as an (M, 4) int array, -1 padded."""
    m = C.c_int()
    call("tq_pool_excitations", n_spatial, n_electrons, C.byref(m), None, 0)
    idx = np.zeros((m.value, 4), dtype=np.int32)
    call("tq_pool_excitations", n_spatial, n_electrons, C.byref(m), _ptr(idx), m.value)
    return idx


def pauli_pool(n_spatial, n_electrons, mapping):
    """Generators as Pauli sums: x[M], nterm[M], z[M, 8], c[M, 8]."""
    M = pool_excitations(n_spatial, n_electrons).shape[0]
    x = np.zeros(M, dtype=np.uint64)
    nt = np.zeros(M, dtype=np.int32)
    z = np.zeros((M, 8), dtype=np.uint64)
    c = np.zeros((M, 8), dtype=np.float64)
    call("tq_pauli_pool", n_spatial, n_electrons, mapping, M, _ptr(x), _ptr(nt), _ptr(z), _ptr(c))
    return x, nt, z, c


def pool_support_forms(n_spatial, n_electrons, mapping):
    """Support of each generator in reduced form: dict of m[M], pivots[M, 3],
    masks[M, 3], target[M], rep_bit[M], rep_pos[M]."""
    M = pool_excitations(n_spatial, n_electrons).shape[0]
    out = {"m": np.zeros(M, np.int32), "pivots": np.zeros((M, 3), np.int32),
           "masks": np.zeros((M, 3), np.uint64), "target": np.zeros(M, np.int32),
           "rep_bit": np.zeros(M, np.int32), "rep_pos": np.zeros(M, np.int32)}
    call("tq_pool_support_forms", n_spatial, n_electrons, mapping, M, _ptr(out["m"]), _ptr(out["pivots"]),
         _ptr(out["masks"]), _ptr(out["target"]), _ptr(out["rep_bit"]), _ptr(out["rep_pos"]))
    return out


def mapping_relabelled(base_mapping, order):
    """Id of the JW/BK encoding with qubit k stored at bit order[k] of the
    basis index (a memory layout; every result is the base mapping's)."""
    o = np.ascontiguousarray(order, dtype=np.int32)
    out = C.c_int()
    call("tq_mapping_relabelled", int(base_mapping), int(o.size), _ptr(o), C.byref(out))
    return out.value


def pool_sector_order(n_spatial, n_electrons, base_mapping, low_bits=4):
    """Qubit order (for mapping_relabelled) that packs the pool's supports
    into the lowest index bits."""
    o = np.zeros(2 * n_spatial, dtype=np.int32)
    call("tq_pool_sector_order", int(n_spatial), int(n_electrons), int(base_mapping), int(low_bits), _ptr(o))
    return o


def relabel_index(order):
    """Relabelled index of every base-mapping basis index: out[b] has bit
    order[k] set where b has bit k (a state moves by psi_new[out] = psi)."""
    order = np.asarray(order, dtype=np.int64)
    b = np.arange(1 << order.size, dtype=np.int64)
    out = np.zeros_like(b)
    for k, o in enumerate(order):
        out |= ((b >> k) & 1) << o
    return out


def mapping_linear(base_mapping, rows):
    """Id of the JW/BK encoding whose basis index r is carried to r' by the
    invertible GF(2) map with the given rows (bit i of r' = parity of r over
    rows[i]); a memory layout, every result is the base mapping's."""
    r = np.ascontiguousarray(rows, dtype=np.uint64)
    out = C.c_int()
    call("tq_mapping_linear", int(base_mapping), int(r.size), _ptr(r), C.byref(out))
    return out.value


def pool_sector_basis(n_spatial, n_electrons, base_mapping, low_bits=None):
    """Rows of an index map for mapping_linear that packs the pool's
    supports into whole 32-byte sectors (greedy over all GF(2) vectors)."""
    n = 2 * n_spatial
    r = np.zeros(n, dtype=np.uint64)
    call("tq_pool_sector_basis", int(n_spatial), int(n_electrons), int(base_mapping),
         int(n if low_bits is None else low_bits), _ptr(r))
    return r


def linear_index(rows):
    """New index of every base-mapping basis index under mapping_linear's
    map: bit i of out[b] is the parity of b over rows[i] (a state moves by
    psi_new[out] = psi)."""
    rows = np.asarray(rows, dtype=np.int64)
    b = np.arange(1 << rows.size, dtype=np.int64)
    out = np.zeros_like(b)
    for i, r in enumerate(rows):
        v = b & r
        for s in (32, 16, 8, 4, 2, 1):
            v ^= v >> s
        out |= (v & 1) << i
    return out


def hf_index(n_qubits, n_electrons, mapping):
    out = C.c_longlong()
    call("tq_hf_index", n_qubits, n_electrons, mapping, C.byref(out))
    return out.value


# ----------------------------------------------------------------- handles

class Context:
    """Device context (owns scratch); one per concurrent stream."""

    def __init__(self, device=0):
        h = C.c_void_p()
        call("tq_ctx_create", int(device), C.byref(h))
        self.handle = h
        self.device = device

    def launches(self):
        n = C.c_longlong()
        call("tq_ctx_launch_count", self.handle, C.byref(n))
        return n.value

    def set_pair_schedule(self, prec, units_per_thread):
        call("tq_ctx_set_pair_schedule", self.handle, prec, int(units_per_thread))

    def pair_schedule(self, prec):
        u = C.c_int()
        call("tq_ctx_get_pair_schedule", self.handle, prec, C.byref(u))
        return u.value

    def set_test_flags(self, flags):
        """Failure-path tests only: TQ_TEST_WITHHOLD_CHUNK makes the XOR-ELL
        energy's bounded waits run out (TQ_ETIMEOUT)."""
        call("tq_ctx_set_test_flags", self.handle, int(flags))

    def set_spmv_schedule(self, lanes_per_row):
        """4, 8, 16 or 32 CSR lanes per row, or TQ_SPMV_XELL (the default)."""
        call("tq_ctx_set_spmv_schedule", self.handle, int(lanes_per_row))

    def set_support_schedule(self, prec, pairs_per_thread):
        """Support-only update: 1, 2, 4 or 8 support pairs per thread per pass
        (registers), or -1, -2, -4, -8 (shared-memory staging, pipelined)."""
        call("tq_ctx_set_support_schedule", self.handle, prec, int(pairs_per_thread))

    def set_grouped_schedule(self, prec, lanes_per_row, pairs_per_thread):
        """Schedule of the grouped-layout update: lanes sharing a row (1, 2,
        or 4 for complex64) and pairs per lane (1, 2 or 4)."""
        call("tq_ctx_set_grouped_schedule", self.handle, prec, int(lanes_per_row), int(pairs_per_thread))

    def set_support_occupancy(self, prec, ctas_per_sm):
        """Resident CTAs per SM of the support-only update (0: as many as fit)."""
        call("tq_ctx_set_support_occupancy", self.handle, prec, int(ctas_per_sm))

    def set_l2_fetch(self, nbytes):
        """L2 fetch granularity of the CUDA context: 32, 64, 128, or 0 (initial)."""
        call("tq_ctx_set_l2_fetch", self.handle, int(nbytes))

    def l2_fetch(self):
        out = C.c_int()
        call("tq_ctx_get_l2_fetch", self.handle, C.byref(out))
        return out.value

    def trace(self, enable=True):
        """Bracket every kernel launch with CUDA events on its stream."""
        call("tq_ctx_trace", self.handle, 1 if enable else 0)

    def trace_report(self):
        """{kernel name: (launches, total ms)} since the last report (synchronises)."""
        buf = C.create_string_buffer(1 << 16)
        call("tq_ctx_trace_report", self.handle, buf, len(buf))
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms = line.split()
            out[name] = (int(n), float(ms))
        return out

    def close(self):
        if self.handle:
            lib().tq_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Hamiltonian:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle
        nq, prec, nnz, npl, ng, namb, nb = (C.c_int(), C.c_int(), C.c_longlong(), C.c_longlong(),
                                            C.c_longlong(), C.c_longlong(), C.c_size_t())
        call("tq_ham_info", handle, C.byref(nq), C.byref(prec), C.byref(nnz), C.byref(npl),
             C.byref(ng), C.byref(namb), C.byref(nb))
        self.n_qubits, self.prec, self.nnz = nq.value, prec.value, nnz.value
        self.n_pauli, self.n_xgroups, self.n_ambiguous = npl.value, ng.value, namb.value
        self.device_bytes = nb.value

    def __del__(self):
        try:
            if self.handle:
                lib().tq_ham_free(self.handle)
                self.handle = None
        except Exception:
            pass


class Pool:
    def __init__(self, ctx, handle):
        self.ctx = ctx
        self.handle = handle
        m, nq = C.c_int(), C.c_int()
        call("tq_pool_info", handle, C.byref(m), C.byref(nq), None)
        self.M, self.n_qubits = m.value, nq.value
        self.idx4 = np.zeros((self.M, 4), dtype=np.int32)
        call("tq_pool_info", handle, None, None, _ptr(self.idx4))

    def __del__(self):
        try:
            if self.handle:
                lib().tq_pool_free(self.handle)
                self.handle = None
        except Exception:
            pass


class State:
    """A state backed by a torch tensor (device memory comes from torch).

    With ``sector=(n_alpha, n_beta)`` it holds the sector's amplitudes in rank
    order (``sector_dim`` of them) instead of all 2^n_qubits."""

    def __init__(self, ctx, n_qubits, prec=TQ_C128, tensor=None, sector=None):
        import torch
        self.ctx = ctx
        self.n_qubits = n_qubits
        self.prec = prec
        self.sector = tuple(sector) if sector is not None else None
        n = sector_dim(n_qubits // 2, *self.sector) if self.sector else 1 << n_qubits
        if tensor is None:
            tensor = torch.zeros(n, dtype=_torch_dtype(prec), device=f"cuda:{ctx.device}")
        assert tensor.is_contiguous() and tensor.numel() == n
        assert tensor.dtype == _torch_dtype(prec)
        self.tensor = tensor
        h = C.c_void_p()
        if self.sector:
            call("tq_state_wrap_sector", ctx.handle, n_qubits // 2, self.sector[0], self.sector[1], prec,
                 _ptr(tensor), C.byref(h))
        else:
            call("tq_state_wrap", ctx.handle, n_qubits, prec, _ptr(tensor), C.byref(h))
        self.handle = h

    def numpy(self):
        import torch
        torch.cuda.synchronize()
        return self.tensor.cpu().numpy().astype(np.complex128)

    def __del__(self):
        try:
            if self.handle:
                lib().tq_state_free(self.handle)
                self.handle = None
        except Exception:
            pass


# ------------------------------------------------------------------ builders

def build_hamiltonian(ctx, h1, g2, e_const=0.0, mapping=TQ_JW, prec=TQ_C128):
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    g2 = np.ascontiguousarray(g2, dtype=np.float64)
    h = C.c_void_p()
    call("tq_build_hamiltonian", ctx.handle, h1.shape[0], _ptr(h1), _ptr(g2), float(e_const), mapping,
         prec, C.byref(h))
    return Hamiltonian(ctx, h)


def build_pool(ctx, n_spatial, n_electrons, mapping=TQ_JW):
    h = C.c_void_p()
    call("tq_build_pool", ctx.handle, n_spatial, n_electrons, mapping, C.byref(h))
    return Pool(ctx, h)


# ------------------------------------------------- integrals and checkpoints

class FcidumpIntegrals:
    """Integrals read from a FCIDUMP file: h (n, n), g (n, n, n, n) chemist
    (pq|rs), e_const (core energy), n_spatial, n_electrons, ms2."""

    def __init__(self, h, g, e_const, n_electrons, ms2):
        self.h, self.g, self.e_const = h, g, e_const
        self.n_spatial = h.shape[0]
        self.n_electrons, self.ms2 = n_electrons, ms2


def read_fcidump(path):
    n, ne, ms2 = C.c_int(), C.c_int(), C.c_int()
    call("tq_read_fcidump", str(path).encode(), C.byref(n), C.byref(ne), C.byref(ms2), None, None, None, 0)
    h = np.zeros((n.value, n.value))
    g = np.zeros((n.value,) * 4)
    e = C.c_double()
    call("tq_read_fcidump", str(path).encode(), None, None, None, C.byref(e), _ptr(h), _ptr(g), n.value)
    return FcidumpIntegrals(h, g, e.value, ne.value, ms2.value)


def write_fcidump(path, h, g, e_const, n_electrons, ms2=0, tol=0.0):
    h = np.ascontiguousarray(h, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    call("tq_write_fcidump", str(path).encode(), h.shape[0], int(n_electrons), int(ms2), _ptr(h), _ptr(g),
         float(e_const), float(tol))


def state_save(state, path):
    call("tq_state_save", state.handle, str(path).encode())


def state_load(state, path):
    call("tq_state_load", state.handle, str(path).encode())


def replay(ctx, pool, state, ops, thetas, renormalize=True, stream=None):
    """Re-apply a recorded sequence of (operator, angle) updates to ``state``
    (e.g. from Hartree-Fock), as the ADAPT step applied them."""
    for k, th in zip(ops, thetas):
        evolve_taylor5(ctx, pool, int(k), float(th), state, renormalize=renormalize, stream=stream)


# ----------------------------------------------- ADAPT-VQE with re-optimised angles

def ansatz_energy_grad(ctx, ham, pool, psi0, ops, thetas, psi_out=None, gradient=True, stream=None):
    """E and dE/dtheta of the Taylor-5 product ansatz U_n ... U_1 psi0."""
    ops = np.ascontiguousarray(ops, dtype=np.int32)
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    E = C.c_double()
    g = np.zeros(max(ops.size, 1), dtype=np.float64)
    call("tq_ansatz_energy_grad", ctx.handle, ham.handle, pool.handle, psi0.handle, int(ops.size),
         _ptr(ops) if ops.size else None, _ptr(th) if th.size else None, C.byref(E),
         _ptr(g) if gradient else None, psi_out.handle if psi_out is not None else None, _stream(stream))
    return E.value, g[: ops.size]


def adapt_vqe(ctx, ham, pool, psi0, eps=1e-3, max_ops=20, gtol=1e-8, max_iter=200, psi_out=None):
    """ADAPT-VQE with every angle re-optimised: (ops, thetas, energies)."""
    n = C.c_int()
    ops = np.zeros(max(max_ops, 1), dtype=np.int32)
    th = np.zeros(max(max_ops, 1), dtype=np.float64)
    en = np.zeros(max(max_ops, 1), dtype=np.float64)
    call("tq_adapt_vqe", ctx.handle, ham.handle, pool.handle, psi0.handle, float(eps), int(max_ops), float(gtol),
         int(max_iter), C.byref(n), _ptr(ops), _ptr(th), _ptr(en),
         psi_out.handle if psi_out is not None else None)
    k = n.value
    return ops[:k].copy(), th[:k].copy(), en[:k].copy()


# ------------------------------------------------------------ commuting families

TQ_COMMUTE_FULL, TQ_COMMUTE_QWC = 0, 1


def pool_families(pool, mode=TQ_COMMUTE_FULL):
    """Algorithm 1 on a built pool: (family per generator, family-major order, count)."""
    fam = np.zeros(pool.M, dtype=np.int32)
    order = np.zeros(pool.M, dtype=np.int32)
    k = C.c_int()
    call("tq_pool_families", pool.handle, int(mode), _ptr(fam), _ptr(order), C.byref(k))
    return fam, order, k.value


def pool_families_host(n_spatial, n_electrons, mapping=TQ_JW, mode=TQ_COMMUTE_FULL):
    """Algorithm 1 on the host, from (n_spatial, n_electrons, mapping); no device needed."""
    M = len(pool_excitations(n_spatial, n_electrons))
    fam = np.zeros(M, dtype=np.int32)
    order = np.zeros(M, dtype=np.int32)
    k = C.c_int()
    call("tq_pool_families_host", int(n_spatial), int(n_electrons), mapping, int(mode), M, _ptr(fam), _ptr(order),
         C.byref(k))
    return fam, order, k.value


# ------------------------------------------------------- sector-restricted basis

def sector_dim(n_spatial, n_alpha, n_beta):
    """C(n, n_alpha) * C(n, n_beta): amplitudes of the fixed-(n_alpha, n_beta) sector."""
    d = C.c_longlong()
    call("tq_sector_dim", int(n_spatial), int(n_alpha), int(n_beta), C.byref(d))
    return d.value


def sector_basis(n_spatial, n_alpha, n_beta, mapping=TQ_JW):
    """Qubit-space index of every sector basis state, in rank order (host)."""
    out = np.zeros(sector_dim(n_spatial, n_alpha, n_beta), dtype=np.uint32)
    call("tq_sector_basis", int(n_spatial), int(n_alpha), int(n_beta), mapping, out.size, _ptr(out))
    return out


def build_hamiltonian_sector(ctx, h1, g2, e_const=0.0, mapping=TQ_JW, prec=TQ_C128, n_alpha=0, n_beta=0):
    h1 = np.ascontiguousarray(h1, dtype=np.float64)
    g2 = np.ascontiguousarray(g2, dtype=np.float64)
    h = C.c_void_p()
    call("tq_build_hamiltonian_sector", ctx.handle, h1.shape[0], _ptr(h1), _ptr(g2), float(e_const), mapping,
         prec, int(n_alpha), int(n_beta), C.byref(h))
    ham = Hamiltonian(ctx, h)
    ham.sector = (int(n_alpha), int(n_beta))
    ham.dim = sector_dim(h1.shape[0], n_alpha, n_beta)
    return ham


def build_pool_sector(ctx, n_spatial, n_electrons, mapping=TQ_JW, n_alpha=0, n_beta=0):
    h = C.c_void_p()
    call("tq_build_pool_sector", ctx.handle, n_spatial, n_electrons, mapping, int(n_alpha), int(n_beta),
         C.byref(h))
    pool = Pool(ctx, h)
    pool.sector = (int(n_alpha), int(n_beta))
    pool.dim = sector_dim(n_spatial, n_alpha, n_beta)
    return pool


def pool_sector_table(pool):
    """(dim, col, sgn) borrowed device pointers of a sector pool's tables."""
    d, cl, sg = C.c_longlong(), C.c_void_p(), C.c_void_p()
    call("tq_pool_sector_table", pool.handle, C.byref(d), C.byref(cl), C.byref(sg))
    return d.value, cl.value, sg.value


def ham_csr(ham):
    """(rowptr, col, val, diag) device pointers of the Hamiltonian (borrowed)."""
    rp, cl, vl, dg = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    call("tq_ham_csr", ham.handle, C.byref(rp), C.byref(cl), C.byref(vl), C.byref(dg))
    return rp.value, cl.value, vl.value, dg.value


def ham_xell(ham):
    """(n_blocks, n_pairs, xptr, xmask, xval) of the XOR-ELL layout (borrowed device pointers)."""
    nb, npairs = C.c_longlong(), C.c_longlong()
    xp, xm, xv = C.c_void_p(), C.c_void_p(), C.c_void_p()
    call("tq_ham_xell", ham.handle, C.byref(nb), C.byref(npairs), C.byref(xp), C.byref(xm), C.byref(xv))
    return nb.value, npairs.value, xp.value, xm.value, xv.value


def pool_csr(ctx, pool, k, prec=TQ_C128):
    """(rowptr, col, val, nnz) of generator k (device pointers, built on demand)."""
    rp, cl, vl, nnz = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_longlong()
    call("tq_pool_csr", ctx.handle, pool.handle, k, prec, C.byref(rp), C.byref(cl), C.byref(vl),
         C.byref(nnz))
    return rp.value, cl.value, vl.value, nnz.value


def state_set_hf(state, n_electrons, mapping, stream=None):
    call("tq_state_set_hf", state.handle, n_electrons, mapping, _stream(stream))


# ------------------------------------------------------------------ hot path

def evolve_taylor5(ctx, pool, k, theta, state, renormalize=False, stream=None):
    call("tq_evolve_taylor5", ctx.handle, pool.handle, int(k), float(theta), state.handle,
         1 if renormalize else 0, _stream(stream))


def evolve_taylor5_csr(ctx, n_qubits, rowptr, col, val, theta, state, renormalize=False, stream=None):
    call("tq_evolve_taylor5_csr", ctx.handle, n_qubits, C.c_void_p(rowptr), C.c_void_p(col),
         C.c_void_p(val), float(theta), state.handle, 1 if renormalize else 0, _stream(stream))


def energy(ctx, ham, state, stream=None):
    e = C.c_double()
    call("tq_energy", ctx.handle, ham.handle, state.handle, C.byref(e), _stream(stream))
    return e.value


def energy_noalloc(n_qubits, prec, rowptr, col, val, diag, psi, energy_out, stream=None):
    """Energy without any allocation; every argument is a device pointer (int)
    and the result lands in ``energy_out`` (one float64 on the device)."""
    call("tq_energy_noalloc", n_qubits, prec, C.c_void_p(rowptr), C.c_void_p(col), C.c_void_p(val),
         C.c_void_p(diag), C.c_void_p(psi), C.c_void_p(energy_out), _stream(stream))


def energy_matrix_free(ctx, ham, state, stream=None):
    e = C.c_double()
    call("tq_energy_matrix_free", ctx.handle, ham.handle, state.handle, C.byref(e), _stream(stream))
    return e.value


def pool_gradients(ctx, ham, pool, state, out=None, stream=None):
    """Gradients of every pool op; ``out`` may be a float64 CUDA tensor (async)."""
    if out is not None:
        call("tq_pool_gradients", ctx.handle, ham.handle, pool.handle, state.handle, _ptr(out), 1,
             _stream(stream))
        return out
    g = np.zeros(pool.M, dtype=np.float64)
    call("tq_pool_gradients", ctx.handle, ham.handle, pool.handle, state.handle, _ptr(g), 0,
         _stream(stream))
    return g


def adapt_step(ctx, ham, pool, state, eps, theta=float("nan"), stream=None):
    r = AdaptResult()
    call("tq_adapt_step", ctx.handle, ham.handle, pool.handle, state.handle, float(eps),
         float(theta), C.byref(r), _stream(stream))
    return {"energy": r.energy, "max_grad": r.max_grad, "theta": r.theta,
            "selected": r.selected, "converged": bool(r.converged)}


def adapt_run(ctx, ham, pool, state, eps, n_iter, thetas=None, stream=None):
    """n_iter ADAPT steps replayed from one CUDA graph; thetas (length
    n_iter) or None for the line search.  Returns (results, n_done)."""
    res = (AdaptResult * max(int(n_iter), 1))()
    th = None if thetas is None else np.ascontiguousarray(thetas, dtype=np.float64)
    done = C.c_int()
    call("tq_adapt_run", ctx.handle, ham.handle, pool.handle, state.handle, float(eps), _ptr(th), int(n_iter),
         C.cast(res, C.c_void_p), C.byref(done), _stream(stream))
    out = [{"energy": r.energy, "max_grad": r.max_grad, "theta": r.theta, "selected": r.selected,
            "converged": bool(r.converged)} for r in res[:int(n_iter)]]
    return out, done.value


def autotune_support(ctx, pool, prec=TQ_C64, n_states=1024):
    """Time every support-update schedule; set and return (pairs_per_thread, ms)."""
    u, ms = C.c_int(), C.c_double()
    call("tq_autotune_support", ctx.handle, pool.handle, prec, int(n_states), C.byref(u), C.byref(ms))
    return u.value, ms.value


def fp64_fma_rate(ctx, iters=4096):
    """Measured float64 FMA rate of the device, float64 lane operations per
    second (one FMA per lane each; twice that in flops)."""
    r = C.c_double()
    call("tq_fp64_fma_rate", ctx.handle, int(iters), C.byref(r))
    return r.value


def l2_read_rate(ctx, nbytes=32 << 20, reps=64):
    """Measured L2 read rate of the device in bytes per second (a buffer of
    ``nbytes`` read ``reps`` times with loads that bypass L1)."""
    r = C.c_double()
    call("tq_l2_read_rate", ctx.handle, int(nbytes), int(reps), C.byref(r))
    return r.value


def autotune_pair(ctx, pool, prec=TQ_C64, n_states=1024):
    """Time every pair-kernel schedule; set and return (units_per_thread, ms)."""
    u, ms = C.c_int(), C.c_double()
    call("tq_autotune_pair", ctx.handle, pool.handle, prec, int(n_states), C.byref(u), C.byref(ms))
    return u.value, ms.value


def autotune_spmv(ctx, ham, state):
    """Time every energy-SpMV schedule on (ham, state); set and return (schedule, ms).

    The schedule is a CSR lanes-per-row count or TQ_SPMV_XELL."""
    l, ms = C.c_int(), C.c_double()
    call("tq_autotune_spmv", ctx.handle, ham.handle, state.handle, C.byref(l), C.byref(ms))
    return l.value, ms.value


def evolve_taylor5_batch(ctx, pool, psi, k, theta, norm2=None, prec=TQ_C64, stream=None):
    """In-place batched update of ``psi`` (CUDA tensor, n_states x 2^N)."""
    n_states = psi.shape[0]
    call("tq_evolve_taylor5_batch", ctx.handle, pool.handle, n_states, prec, _ptr(psi), _ptr(k),
         _ptr(theta), _ptr(norm2), _stream(stream))


def evolve_taylor5_batch_support(ctx, pool, psi, k, theta, norm2=None, prec=TQ_C64, stream=None):
    """In-place batched update touching only each generator's support rows;
    ``norm2`` (float64 CUDA tensor) is in/out: ||psi_b||^2 in, ||psi_b'||^2 out."""
    n_states = psi.shape[0]
    call("tq_evolve_taylor5_batch_support", ctx.handle, pool.handle, n_states, prec, _ptr(psi), _ptr(k),
         _ptr(theta), _ptr(norm2), _stream(stream))


TQ_GROUP_C64 = 4      # states per group of the grouped layout (one 32-byte sector)
TQ_GROUP_C128 = 2


def evolve_taylor5_batch_grouped(ctx, pool, psi, k, theta, norm2=None, prec=TQ_C64, stream=None):
    """Support-only update of groups of states sharing a generator, stored
    amplitude-major within each group: psi of shape (n_groups, D, G) (G = 4
    complex64 or 2 complex128 states), k int32 [n_groups], theta and norm2
    float64 [n_groups * G], all CUDA tensors."""
    G = TQ_GROUP_C128 if prec == TQ_C128 else TQ_GROUP_C64
    n_groups = int(k.numel())
    assert psi.numel() == n_groups * (1 << pool.n_qubits) * G and theta.numel() == n_groups * G
    call("tq_evolve_taylor5_batch_grouped", ctx.handle, pool.handle, n_groups, prec, _ptr(psi), _ptr(k),
         _ptr(theta), _ptr(norm2), _stream(stream))


def evolve_taylor5_batch_support_touch(ctx, pool, psi, k, norm2=None, prec=TQ_C64, stream=None):
    """The support-only update's launch with the update taken out: every
    support row read and written back unchanged (a measurement aid: the
    access pattern's own floor)."""
    call("tq_evolve_taylor5_batch_support_touch", ctx.handle, pool.handle, int(psi.shape[0]), prec, _ptr(psi),
         _ptr(k), _ptr(norm2), _stream(stream))


def evolve_taylor5_batch_support_host(ctx, pool, psi, k, theta, norm2=None, prec=TQ_C64):
    """Support-only update of states in page-locked HOST memory (a pinned
    torch CPU tensor), read and written in place by the kernel; k, theta and
    norm2 (in/out) are host arrays."""
    n_states = psi.shape[0]
    call("tq_evolve_taylor5_batch_support_host", ctx.handle, pool.handle, n_states, prec, _ptr(psi), _ptr(k),
         _ptr(theta), _ptr(norm2))


def evolve_taylor5_batch_host(ctx, pool, psi, k, theta, norm2=None, prec=TQ_C64):
    """Batched update of HOST arrays (numpy or pinned torch CPU tensors)."""
    n_states = psi.shape[0]
    call("tq_evolve_taylor5_batch_host", ctx.handle, pool.handle, n_states, prec, _ptr(psi), _ptr(k),
         _ptr(theta), _ptr(norm2))


# ----------------------------------------------------------- trajectory batch

class Batch:
    """Independent ADAPT trajectories advanced together (graph-replayed)."""

    def __init__(self, ctx, hams, pools, n_electrons, mappings, thetas, eps=1e-3):
        self.ctx, self.hams, self.pools = ctx, list(hams), list(pools)
        n = len(self.hams)
        self.lengths = np.array([len(t) for t in thetas], dtype=np.int32)
        flat = np.concatenate([np.asarray(t, dtype=np.float64) for t in thetas]) if n else np.zeros(0)
        self._flat = np.ascontiguousarray(flat if flat.size else np.zeros(1))
        hh = (C.c_void_p * n)(*[h.handle.value for h in self.hams])
        pp = (C.c_void_p * n)(*[p.handle.value for p in self.pools])
        ne = np.ascontiguousarray(n_electrons, dtype=np.int32)
        mp = np.ascontiguousarray(mappings, dtype=np.int32)
        h = C.c_void_p()
        call("tq_batch_create", ctx.handle, n, hh, pp, _ptr(ne), _ptr(mp), _ptr(self.lengths),
             _ptr(self._flat), float(eps), C.byref(h))
        self.handle = h
        self.n = n

    def set_schedule(self, lanes_per_row):
        call("tq_batch_set_schedule", self.handle, int(lanes_per_row))

    def autotune(self):
        l, ms = C.c_int(), C.c_double()
        call("tq_batch_autotune", self.handle, C.byref(l), C.byref(ms))
        return l.value, ms.value

    def run(self, use_graph=True, stream=None):
        call("tq_batch_run", self.handle, 1 if use_graph else 0, _stream(stream))

    def results(self):
        L = int(self.lengths.sum())
        n_iter = np.zeros(self.n, dtype=np.int32)
        conv = np.zeros(self.n, dtype=np.int32)
        e, g, th = (np.zeros(max(L, 1)) for _ in range(3))
        sel = np.zeros(max(L, 1), dtype=np.int32)
        call("tq_batch_results", self.handle, _ptr(n_iter), _ptr(conv), _ptr(e), _ptr(g), _ptr(sel), _ptr(th))
        out, off = [], 0
        for t in range(self.n):
            n = int(self.lengths[t])
            k = int(n_iter[t])
            out.append({"n_iter": k, "converged": bool(conv[t]), "energy": e[off:off + k].copy(),
                        "max_grad": g[off:off + k].copy(), "selected": sel[off:off + k].copy(),
                        "theta": th[off:off + k].copy()})
            off += n
        return out

    def state(self, t):
        """Copy of trajectory t's state as a complex128 numpy array."""
        import torch
        ptr, nq = C.c_void_p(), C.c_int()
        call("tq_batch_state", self.handle, int(t), C.byref(ptr), C.byref(nq))
        prec = self.hams[0].prec
        n = 1 << nq.value
        typestr = "<c16" if prec == TQ_C128 else "<c8"

        class _View:
            __cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                        "data": (ptr.value, False), "version": 3}

        torch.cuda.synchronize()
        return torch.as_tensor(_View(), device="cuda").cpu().numpy().astype(np.complex128)

    def __del__(self):
        try:
            if self.handle:
                lib().tq_batch_free(self.handle)
                self.handle = None
        except Exception:
            pass


# --------------------------------------------------------------- request loop

class Server:
    """Continuous-batching request loop over resident sessions (owns ``ctx`` while running)."""

    def __init__(self, ctx, prec=TQ_C64, hbm_budget=4 << 30, max_batch=512):
        self.ctx, self.prec = ctx, prec
        h = C.c_void_p()
        call("tq_server_create", ctx.handle, prec, C.c_size_t(int(hbm_budget)), int(max_batch), C.byref(h))
        self.handle = h
        self._keep = []
        self._out = (Completion * 4096)()

    def add_hamiltonian(self, ham, pool):
        i = C.c_int()
        call("tq_server_add_hamiltonian", self.handle, ham.handle, pool.handle, C.byref(i))
        self._keep += [ham, pool]
        return i.value

    def add_session(self, ham_id, n_electrons, mapping):
        i = C.c_int()
        call("tq_server_add_session", self.handle, int(ham_id), int(n_electrons), int(mapping), C.byref(i))
        return i.value

    def start(self):
        call("tq_server_start", self.handle)

    def submit(self, kind, session, op=0, theta=0.0, tag=0):
        r = Request(int(kind), int(session), int(op), 0, float(theta), int(tag))
        call("tq_server_submit", self.handle, C.byref(r))

    def poll(self, timeout_us=1000):
        """Completions as dicts (empty list on timeout)."""
        n = C.c_int()
        rc = lib().tq_server_poll(self.handle, self._out, len(self._out), C.byref(n), int(timeout_us))
        if rc == -4:
            return []
        if rc != 0:
            raise TQError(rc, "tq_server_poll", lib().tq_last_error().decode())
        return [{f: getattr(self._out[i], f) for f, _ in Completion._fields_} for i in range(n.value)]

    def stats(self):
        t, c, q = C.c_longlong(), C.c_longlong(), C.c_longlong()
        call("tq_server_stats", self.handle, C.byref(t), C.byref(c), C.byref(q))
        return {"ticks": t.value, "completed": c.value, "queued": q.value}

    def state(self, session):
        """Copy of a session's state (call when idle), complex128 numpy."""
        import torch
        ptr, nq = C.c_void_p(), C.c_int()
        call("tq_server_session_state", self.handle, int(session), C.byref(ptr), C.byref(nq))
        n = 1 << nq.value
        typestr = "<c16" if self.prec == TQ_C128 else "<c8"

        class _View:
            __cuda_array_interface__ = {"shape": (n,), "typestr": typestr,
                                        "data": (ptr.value, False), "version": 3}

        torch.cuda.synchronize()
        return torch.as_tensor(_View(), device="cuda").cpu().numpy().astype(np.complex128)

    def stop(self):
        call("tq_server_stop", self.handle)

    def __del__(self):
        try:
            if self.handle:
                lib().tq_server_free(self.handle)
                self.handle = None
        except Exception:
            pass
